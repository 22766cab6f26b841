"""Batched counts (many resident graphs in one captured launch sequence):
every graph's counts must equal the oracle's and bb_count's for it alone,
whatever the launch shapes, across replays and after sign flips of member
graphs."""
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


def small_mix(n, m_hi=2e5):
    """The batched mix (log-uniform edges, ratio, exponent, sign bias) with a
    smaller edge ceiling, so the oracle checks every graph quickly."""
    return synth.batch_graphs(n, m_hi=m_hi)


@pytest.fixture(scope="module")
def mix(ctx):
    hosts = small_mix(48)
    # degenerate members: no edges, a single butterfly, one dense vote graph
    # whose anchors are split over several CTAs, a graph with one dense anchor
    hosts.append(synth.from_edges(5, 7, [], [], []))
    hosts.append(synth.from_edges(2, 2, [0, 1, 0, 1], [0, 0, 1, 1], [1, -1, 1, 1]))
    hosts.append(synth.vote(11, 40, 6_000, 0.5, 2, 0.55, 0.8))
    hosts.append(synth.uniform_2k_1k())
    graphs = [ctx.upload(g) for g in hosts]
    want = [oracle.count(g, threads=4) for g in hosts]
    yield hosts, graphs, want
    for g in graphs:
        g.free()


def test_batch_matches_oracle_and_single_counts(ctx, mix):
    hosts, graphs, want = mix
    b = pkg.Batch(ctx, graphs)
    bal, tot = b.count()
    for i, g in enumerate(graphs):
        assert (int(bal[i]), int(tot[i])) == want[i], hosts[i].name
        single = g.count()
        assert (single.balanced, single.total) == want[i]
    b.free()


@pytest.mark.parametrize("chunk,conc,frac", [(1, 0, 1.0), (7, 1, 0.25), (64, 1, 0.5), (3, 0, 0.75)])
def test_batch_shapes_do_not_change_counts(ctx, mix, chunk, conc, frac):
    hosts, graphs, want = mix
    b = pkg.Batch(ctx, graphs)
    t = b.tune()
    t.warp_chunk, t.concurrent = chunk, conc
    for k in range(len(pkg.KERNELS)):
        t.grid_frac[k] = frac
    b.set_tune(t)
    got = b.tune().to_dict()
    assert got["warp_chunk"] == chunk and got["concurrent"] == conc
    for _ in range(3):  # replays of the captured graph
        bal, tot = b.count()
        assert [(int(x), int(y)) for x, y in zip(bal, tot)] == want
    b.free()


SHAPES = [
    # most anchors out of the warp class, small dense split parts
    {"warp_w_max": 64, "warp_small_w": 0, "team_w_max": 256, "split_wedges": 1024},
    # warp anchors hash every endpoint when they can
    {"warp_w_max": 16384, "warp_small_w": 16384, "team_w_max": 16384, "split_wedges": 1 << 20},
    {"warp_w_max": 2048, "warp_small_w": 96, "team_w_max": 4096, "split_wedges": 16384},
]


@pytest.mark.parametrize("staged", [0, 1])
def test_bucket_shapes_per_size_class_keep_counts(ctx, mix, staged):
    hosts, graphs, want = mix
    b = pkg.Batch(ctx, graphs)
    try:
        for rot in range(len(SHAPES)):
            t = b.tune()
            t.dense_staged = staged
            for k in range(pkg.NSIZE):   # a different shape per size class
                t.shape[k] = pkg.ClassShape.from_dict(SHAPES[(k + rot) % len(SHAPES)])
            b.set_tune(t)
            got = b.tune().to_dict()
            assert got["dense_staged"] == staged
            assert got["shape"] == [SHAPES[(k + rot) % len(SHAPES)] for k in range(pkg.NSIZE)]
            for _ in range(2):
                bal, tot = b.count()
                assert [(int(x), int(y)) for x, y in zip(bal, tot)] == want
            # a re-classified member counts right on its own too
            for i in (0, len(graphs) - 2, len(graphs) - 1):
                c = graphs[i].count()
                assert (c.balanced, c.total) == want[i]
    finally:
        b.set_tune({**b.tune().to_dict(), "dense_staged": 0,
                    "shape": [pkg.ClassShape.DEFAULT] * pkg.NSIZE})
        b.free()


def test_shape_argument_errors(ctx, mix):
    hosts, graphs, want = mix
    b = pkg.Batch(ctx, graphs)
    for bad in ({"warp_w_max": 0}, {"warp_w_max": 20000}, {"warp_w_max": 100, "warp_small_w": 200},
                {"team_w_max": 0}, {"split_wedges": 100}):
        t = b.tune()
        t.shape[1] = pkg.ClassShape.from_dict({**pkg.ClassShape.DEFAULT, **bad})
        with pytest.raises(pkg.BBError) as ei:
            b.set_tune(t)
        assert ei.value.name == "BB_ERR_INVALID_ARG"
        with pytest.raises(pkg.BBError):
            ctx.set_shape({**pkg.ClassShape.DEFAULT, **bad})
    bal, tot = b.count()   # unchanged after the rejected tunes
    assert [(int(x), int(y)) for x, y in zip(bal, tot)] == want
    b.free()


def test_single_graph_shapes(ctx):
    graphs = [synth.chung_lu_scaled(71, 300_000), synth.vote(12, 40, 6_000, 0.5, 2, 0.55, 0.8),
              synth.uniform_2k_1k()]
    want = [oracle.count(g, threads=4) for g in graphs]
    try:
        for shape in SHAPES:
            for staged in (False, True):
                ctx.set_shape(shape, staged)
                for g, w in zip(graphs, want):
                    c = ctx.count(g)
                    assert (c.balanced, c.total) == w, (g.name, shape, staged)
        ctx.set_shape(None)
        res = ctx.upload(graphs[0])
        try:
            for shape in SHAPES:
                res.set_shape(shape, True)
                c = res.count(per_vertex=True)
                assert (c.balanced, c.total) == want[0]
                assert int(c.per_vertex.sum()) == 4 * want[0][0]
                gids = np.arange(0, graphs[0].nU + graphs[0].nV, 997)
                assert np.array_equal(c.per_vertex[gids],
                                      oracle.per_vertex(graphs[0], gids=gids, threads=4))
        finally:
            res.free()
    finally:
        ctx.set_shape(None)


def test_traced_batch_count(ctx, mix):
    hosts, graphs, want = mix
    b = pkg.Batch(ctx, graphs)
    ctx.set_timing(True)
    try:
        bal, tot = b.count()
        tr = ctx.last_timing()
    finally:
        ctx.set_timing(False)
    assert [(int(x), int(y)) for x, y in zip(bal, tot)] == want
    assert tr["count_ms"] > 0
    assert sum(tr["kernels"][k]["anchors"] for k in pkg.KERNELS) > 0
    assert sum(tr["kernels"][k]["wedges"] for k in pkg.KERNELS) == sum(g.info()[3] for g in graphs)
    bal, tot = b.count()  # captured again afterwards
    assert [(int(x), int(y)) for x, y in zip(bal, tot)] == want
    b.free()


def test_batch_order_and_subsets(ctx, mix):
    hosts, graphs, want = mix
    rng = np.random.default_rng(5)
    order = rng.permutation(len(graphs))[:17]
    b = pkg.Batch(ctx, [graphs[i] for i in order])
    bal, tot = b.count()
    assert [(int(x), int(y)) for x, y in zip(bal, tot)] == [want[i] for i in order]
    b.free()
    one = pkg.Batch(ctx, [graphs[3]])
    assert tuple(int(x[0]) for x in one.count()) == want[3]
    one.free()
    # copies of one graph would share its accumulator: refused
    with pytest.raises(pkg.BBError):
        pkg.Batch(ctx, [graphs[0], graphs[0]])


def test_batch_sees_sign_flips(ctx, mix):
    hosts, graphs, want = mix
    b = pkg.Batch(ctx, graphs)
    rng = np.random.default_rng(9)
    flipped, lists = {}, {}
    for i in (0, 5, len(hosts) - 1):
        g = hosts[i]
        if g.nE == 0:
            continue
        idx = rng.choice(g.nE, size=max(1, g.nE // 100), replace=False)
        graphs[i].flip(idx)
        lists[i] = idx
        s = g.sign.copy()
        s[idx] = -s[idx]
        h = synth.SignedBipartite(g.nU, g.nV, g.rowptr, g.col, s, g.name + "/flip")
        flipped[i] = oracle.count(h, threads=4)
    bal, tot = b.count()
    for i in range(len(graphs)):
        assert (int(bal[i]), int(tot[i])) == flipped.get(i, want[i]), i
    for i, idx in lists.items():  # flip back: the other tests use the originals
        graphs[i].flip(idx)
    bal, tot = b.count()
    assert [(int(x), int(y)) for x, y in zip(bal, tot)] == want
    b.free()


def test_autotune_keeps_counts(ctx):
    hosts = small_mix(24, m_hi=5e5)
    graphs = [ctx.upload(g) for g in hosts]
    want = [oracle.count(g, threads=4) for g in hosts]
    b = pkg.Batch(ctx, graphs)
    t, ms = b.autotune(reps=2)
    assert ms > 0
    d = t.to_dict()
    assert 1 <= d["warp_chunk"] <= 1024
    assert all(0 < f <= 1 for f in d["grid_frac"].values())
    assert b.tune().to_dict() == d
    bal, tot = b.count()
    assert [(int(x), int(y)) for x, y in zip(bal, tot)] == want
    b.free()
    for g in graphs:
        g.free()


def test_batch_argument_errors(ctx, mix):
    hosts, graphs, want = mix
    with pytest.raises(pkg.BBError) as ei:
        pkg.Batch(ctx, [])
    assert ei.value.name == "BB_ERR_INVALID_ARG"
    other = pkg.Context(0)
    try:
        with pytest.raises(pkg.BBError) as ei:
            pkg.Batch(other, graphs[:2])
        assert ei.value.name == "BB_ERR_INVALID_ARG"
    finally:
        other.close()
    b = pkg.Batch(ctx, graphs[:2])
    t = pkg.BatchTune()
    t.warp_chunk = 0
    with pytest.raises(pkg.BBError):
        b.set_tune(t)
    b.free()
