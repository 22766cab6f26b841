"""Incremental re-count under sign flips (bb_count_flipped): after any set
of flips the counts must equal the oracle's on the flipped graph, whether
the library walked only the butterflies through the flipped edges or
recounted; small flip sets on large graphs must take the incremental walk,
and flip sets where butterflies hold several flipped edges must stay exact."""
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


def flipped(g, sign):
    return synth.SignedBipartite(g.nU, g.nV, g.rowptr, g.col, sign, g.name + "/f")


def run_sequence(ctx, g, sizes, seed, expect_incremental=None):
    r = ctx.upload(g)
    c = r.count()
    assert (c.balanced, c.total) == oracle.count(g, threads=8)
    sign = g.sign.copy()
    rng = np.random.default_rng(seed)
    modes = []
    for k in sizes:
        idx = rng.choice(g.nE, size=min(k, g.nE), replace=False)
        b, t, inc = r.count_flipped(idx)
        sign[idx] = -sign[idx]
        assert (b, t) == oracle.count(flipped(g, sign), threads=8), (g.name, k, inc)
        modes.append(inc)
    # the resident graph's signs match: a plain recount agrees
    c = r.count()
    assert (c.balanced, c.total) == oracle.count(flipped(g, sign), threads=8)
    r.free()
    if expect_incremental is not None:
        assert modes == expect_incremental, modes
    return modes


def test_small_flip_sets_are_incremental_and_exact(ctx):
    g = synth.chung_lu_scaled(43, 2_000_000)
    run_sequence(ctx, g, [1, 3, 10, 40], seed=1, expect_incremental=[True] * 4)


def test_large_flip_sets_recount(ctx):
    g = synth.chung_lu_scaled(41, 200_000)
    modes = run_sequence(ctx, g, [g.nE // 10, g.nE // 100, 2], seed=2)
    assert modes[0] is False and modes[-1] is True


def test_butterflies_with_several_flipped_edges(ctx):
    # dense graphs: most butterflies through a flipped edge hold other flipped edges
    rng = np.random.default_rng(9)
    for trial in range(6):
        m, n = int(rng.integers(4, 9)), int(rng.integers(4, 9))
        g = synth.from_dense(rng.choice([-1, 1], size=(m, n)).astype(np.int8))
        run_sequence(ctx, g, [1, 2, 3, 5, m * n // 2, 7], seed=trial)
    g = synth.vote(3, 30, 400, 0.5, 2, 0.55, 0.8)
    run_sequence(ctx, g, [5, 50, 200], seed=3)


def test_duplicates_and_cache_invalidation(ctx):
    g = synth.uniform_2k_1k()
    r = ctx.upload(g)
    r.count()
    sign = g.sign.copy()
    # an index listed twice flips back; three times flips once
    b, t, inc = r.count_flipped([5, 5, 9, 9, 9, 17])
    sign[[9, 17]] = -sign[[9, 17]]
    assert (b, t) == oracle.count(flipped(g, sign))
    # a plain flip drops the cached counts: the next call recounts, exactly
    r.flip([100])
    sign[100] = -sign[100]
    b, t, inc = r.count_flipped([200])
    sign[200] = -sign[200]
    assert inc is False and (b, t) == oracle.count(flipped(g, sign))
    # nothing to flip: the cached counts come back
    b2, t2, _ = r.count_flipped([])
    assert (b2, t2) == (b, t)
    with pytest.raises(pkg.BBError):
        r.count_flipped([g.nE])
    r.free()
