"""The one-shot device path replays the work after validation as a captured
CUDA graph when a call repeats the previous one's shape and buffers. These
tests check that replays read the buffers afresh (a changed input changes
the result, as the oracle says), that timing events still time the kernels,
that the launch counter counts replayed kernels, and that a different shape
or buffer set in between is counted directly and correctly."""
import numpy as np
import pytest

import oracle
import paper_2308_07932_gb300 as pkg
from paper_2308_07932_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    c = pkg.Context(0)
    yield c
    c.close()


def on_device(g):
    t = [torch.from_numpy(a).cuda() for a in (g.rowptr, g.col, g.sign)]
    torch.cuda.synchronize()
    return t


@pytest.mark.parametrize("timing", [False, True])
def test_repeated_calls_replay_and_read_fresh_inputs(ctx, timing):
    g = synth.chung_lu_scaled(51, 150_000)
    want = oracle.count(g)
    rp, cl, sg = on_device(g)
    ctx.set_timing(timing)
    try:
        got, used = [], []
        for _ in range(4):
            l0 = pkg.launch_count()
            c = ctx.count_tensors(g.nV, rp, cl, sg)
            used.append(pkg.launch_count() - l0)
            got.append((c.balanced, c.total))
            if timing:
                t = ctx.last_timing()
                assert t["build_ms"] > 0 and t["count_ms"] > 0
                assert sum(k["ms"] for k in t["kernels"].values()) > 0
        assert got == [want] * 4
        assert len(set(used)) == 1 and used[0] > 10  # replays count their kernels
        # change the signs in place: the replay must see the new signs
        flip = np.random.default_rng(5).choice(g.nE, size=g.nE // 50, replace=False)
        s2 = g.sign.copy()
        s2[flip] = -s2[flip]
        sg.copy_(torch.from_numpy(s2))
        torch.cuda.synchronize()
        g2 = synth.SignedBipartite(g.nU, g.nV, g.rowptr, g.col, s2, g.name + "_flipped")
        want2 = oracle.count(g2)
        for _ in range(2):
            c = ctx.count_tensors(g.nV, rp, cl, sg)
            assert (c.balanced, c.total) == want2
        assert want2[1] == want[1] and want2[0] != want[0]
    finally:
        ctx.set_timing(False)


def test_alternating_shapes_stay_correct(ctx):
    gs = [synth.chung_lu_scaled(52, 60_000), synth.uniform_2k_1k()]
    wants = [oracle.count(g) for g in gs]
    dev = [on_device(g) for g in gs]
    for i in [0, 0, 1, 0, 1, 1, 1, 0, 0]:
        rp, cl, sg = dev[i]
        c = ctx.count_tensors(gs[i].nV, rp, cl, sg)
        assert (c.balanced, c.total) == wants[i]


def test_invalid_input_after_replay_is_rejected(ctx):
    g = synth.chung_lu_scaled(53, 40_000)
    want = oracle.count(g)
    rp, cl, sg = on_device(g)
    for _ in range(3):
        c = ctx.count_tensors(g.nV, rp, cl, sg)
        assert (c.balanced, c.total) == want
    bad = sg.clone()
    bad[7] = 0  # a sign that is neither +1 nor -1
    with pytest.raises(pkg.BBError):
        ctx.count_tensors(g.nV, rp, cl, bad)
    sg2 = sg.clone()
    sg2[7] = 0
    with pytest.raises(pkg.BBError):
        ctx.count_tensors(g.nV, rp, cl, sg2)
    c = ctx.count_tensors(g.nV, rp, cl, sg)
    assert (c.balanced, c.total) == want


def test_repeated_degenerate_graphs(ctx):
    """Repeats of empty and tiny graphs (host path: the staging buffers
    repeat, so the second call captures and later calls replay)."""
    cases = [
        (synth.SignedBipartite(3, 4, np.zeros(4, np.int64), np.zeros(0, np.int32),
                               np.zeros(0, np.int8)), (0, 0)),
        (synth.SignedBipartite(0, 5, np.zeros(1, np.int64), np.zeros(0, np.int32),
                               np.zeros(0, np.int8)), (0, 0)),
        (synth.from_edges(1, 60, [0] * 60, list(range(60)), [1] * 60), (0, 0)),
        (synth.from_edges(2, 2, [0, 0, 1, 1], [0, 1, 0, 1], [1, 1, 1, -1]), (0, 1)),
        (synth.from_edges(2, 2, [0, 0, 1, 1], [0, 1, 0, 1], [1, -1, -1, 1]), (1, 1)),
    ]
    for g, want in cases:
        for _ in range(4):
            c = ctx.count(g)
            assert (c.balanced, c.total) == want, g.name
