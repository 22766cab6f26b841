"""BB-Base (Algorithm 1) on the GPU (bb_count_base): explicit pair tests
must give exactly the oracle's counts, like the bucket method."""
import numpy as np
import pytest

import oracle
import paper_2308_07932_gb300 as pkg
from paper_2308_07932_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pkg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("make", [
    lambda: synth.uniform_2k_1k(),
    lambda: synth.chung_lu_scaled(41, 200_000),
    lambda: synth.vote(7, 40, 3_000, 0.4, 2, 0.55, 0.8),
    lambda: synth.from_dense(np.ones((9, 11), dtype=np.int8)),
    lambda: synth.chung_lu_scaled(43, 2_000_000),
])
def test_base_matches_oracle(ctx, make):
    g = make()
    r = ctx.upload(g)
    want = oracle.count(g, threads=8)
    assert r.count_base() == want, g.name
    c = r.count()
    assert (c.balanced, c.total) == want
    r.free()


def test_base_tiny_graphs(ctx):
    for signs in ([1, 1, 1, 1], [1, -1, 1, 1]):
        g = synth.from_edges(2, 2, [0, 1, 0, 1], [0, 0, 1, 1], signs)
        r = ctx.upload(g)
        assert r.count_base() == oracle.count(g)
        r.free()
    for seed in range(20):
        rng = np.random.default_rng(seed)
        nU, nV = int(rng.integers(2, 12)), int(rng.integers(2, 12))
        g = synth.uniform(5000 + seed, nU, nV, int(rng.integers(0, nU * nV + 1)), 0.5)
        r = ctx.upload(g)
        assert r.count_base() == oracle.count(g), seed
        r.free()
