"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
bit-exact, on seeded graphs from tiny to the full 2M x 500k workload.

Integer counts must match exactly. The wedge count the library reports
(the metric's unit) is checked against an independent NumPy computation of
the priority wedges of Algorithm 2 on small graphs.
"""
import json
import os

import numpy as np
import pytest

import oracle
import paper_2308_07932_gb300 as pkg
from paper_2308_07932_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EXPECTED = json.load(open(os.path.join(GOLDEN, "expected_counts.json")))


@pytest.fixture(scope="module")
def ctx():
    c = pkg.Context(0)
    yield c
    c.close()


def same(ctx, g, threads=4):
    got = ctx.count(g)
    want = oracle.count(g, threads=threads)
    assert (got.balanced, got.total) == want, (g.name, got, want)
    return got


def priority_wedges(g):
    """Wedges u - v - w with u the highest-priority vertex (Def. 4, gid = u
    or |U| + v): for every middle v and every neighbour u of v ranked above
    v, the neighbours of v ranked below u. Written with NumPy sorts."""
    u, v, _ = g.edges()
    n = g.nU + g.nV
    deg = np.concatenate([np.diff(g.rowptr), np.bincount(g.col, minlength=g.nV)])
    order = np.lexsort((np.arange(n), deg))
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    src = np.concatenate([u, g.nU + v])
    dst = np.concatenate([g.nU + v, u])
    rs, rd = rank[src], rank[dst]
    o = np.lexsort((rd, rs))
    rs, rd = rs[o], rd[o]
    start = np.searchsorted(rs, rs, side="left")
    pos = np.arange(rs.size) - start      # neighbours of middle rs ranked below rd
    up = rd > rs                           # rd outranks the middle
    return int(pos[up].sum())


# ------------------------------------------------------------ small cases
def read_fig1():
    rows = []
    for line in open(os.path.join(GOLDEN, "fig1_signed_butterflies.txt")):
        if line.startswith("#") or not line.strip():
            continue
        p = line.split()
        rows.append(([int(x) for x in p[2:6]], int(p[6]), int(p[7])))
    return rows


def test_fig1_six_butterflies(ctx):
    for signs, bal, tot in read_fig1():
        g = synth.from_edges(2, 2, [0, 1, 0, 1], [0, 0, 1, 1], signs)
        c = ctx.count(g)
        assert (c.balanced, c.total) == (bal, tot)
        assert c.wedges == 2


def test_lemma2_k2n(ctx):
    rng = np.random.default_rng(0)
    for l in range(0, 9):
        for m in range(0, 9):
            us, vs, ss = [], [], []
            for v in range(l + m):
                a = int(rng.choice([-1, 1]))
                us += [0, 1]; vs += [v, v]; ss += [a, a if v < l else -a]
            g = synth.from_edges(2, l + m, us, vs, ss)
            c = ctx.count(g)
            assert (c.balanced, c.total) == (l * (l - 1) // 2 + m * (m - 1) // 2,
                                            (l + m) * (l + m - 1) // 2)


def test_complete_bipartite(ctx):
    rng = np.random.default_rng(1)
    for a, b in [(2, 2), (5, 7), (40, 33), (300, 200)]:
        x, y = rng.choice([-1, 1], size=a), rng.choice([-1, 1], size=b)
        g = synth.from_dense(np.outer(x, y))
        c = ctx.count(g)
        want = a * (a - 1) // 2 * (b * (b - 1) // 2)
        assert (c.balanced, c.total) == (want, want)
        R = synth.from_dense(rng.choice([-1, 1], size=(a, b)))
        same(ctx, R)


def test_random_tiny_graphs(ctx):
    for seed in range(150):
        rng = np.random.default_rng(seed)
        nU, nV = int(rng.integers(1, 14)), int(rng.integers(1, 14))
        m = int(rng.integers(0, nU * nV + 1))
        g = synth.uniform(500 + seed, nU, nV, m, float(rng.uniform(0.1, 0.9)))
        c = same(ctx, g)
        assert c.wedges == priority_wedges(g)


def test_empty_and_degenerate(ctx):
    e = synth.SignedBipartite(3, 4, np.zeros(4, np.int64), np.zeros(0, np.int32),
                              np.zeros(0, np.int8))
    c = ctx.count(e)
    assert (c.balanced, c.total, c.wedges) == (0, 0, 0)
    for g in [synth.from_edges(1, 1, [0], [0], [-1]),
              synth.from_edges(1, 60, [0] * 60, list(range(60)), [1] * 60),
              synth.from_edges(60, 1, list(range(60)), [0] * 60, [-1] * 60),
              synth.from_edges(2, 2, [0, 0, 1], [0, 1, 1], [1, 1, 1])]:
        c = ctx.count(g)
        assert (c.balanced, c.total) == (0, 0)
    z = synth.SignedBipartite(0, 5, np.zeros(1, np.int64), np.zeros(0, np.int32),
                              np.zeros(0, np.int8))
    assert tuple(ctx.count(z))[:2] == (0, 0)


def test_uniform_2k_1k(ctx):
    g = synth.uniform_2k_1k()
    rec = EXPECTED["uniform_2000x1000_e20000_p0.7"]
    c = ctx.count(g)
    assert (c.balanced, c.total) == (rec["balanced"], rec["total"])
    assert c.wedges == priority_wedges(g)


def test_unsorted_rows_and_relabels(ctx):
    g = synth.chung_lu_scaled(9, 30_000)
    want = oracle.count(g)
    rng = np.random.default_rng(4)
    col, sign = g.col.copy(), g.sign.copy()
    for u in range(g.nU):  # shuffle every row
        a, b = g.rowptr[u], g.rowptr[u + 1]
        p = rng.permutation(b - a)
        col[a:b] = col[a:b][p]
        sign[a:b] = sign[a:b][p]
    g2 = synth.SignedBipartite(g.nU, g.nV, g.rowptr, col, sign)
    for h in [g2, synth.swap_sides(g), synth.permute_ids(g, 1)]:
        c = ctx.count(h)
        assert (c.balanced, c.total) == want


@pytest.mark.parametrize("seed,m,p", [(21, 20_000, 0.5), (22, 80_000, 0.8), (23, 200_000, 0.6),
                                      (24, 600_000, 0.9)])
def test_powerlaw_graphs(ctx, seed, m, p):
    g = synth.chung_lu_scaled(seed, m, p_pos=p)
    c = same(ctx, g)
    if m <= 200_000:
        assert c.wedges == priority_wedges(g)


@pytest.mark.parametrize("nU,nV,pe", [(100, 20_000, 0.4), (250, 6_000, 0.3), (40, 30_000, 0.6)])
def test_dense_vote_graphs_split_anchors(ctx, nU, nV, pe):
    # few dense anchors with many wedges each: the split-and-merge path
    g = synth.vote(nU * 7 + nV, nU, nV, pe, 2, 0.55, 0.8)
    c = same(ctx, g)
    assert c.wedges == priority_wedges(g)


def test_windowed_dense_anchor(ctx):
    # K_{60000,4}: anchors with ~60k vertices above them and 4 middles each,
    # so the dense endpoint range is walked in windows
    rng = np.random.default_rng(7)
    nU, nV = 60_000, 4
    u = np.repeat(np.arange(nU), nV)
    v = np.tile(np.arange(nV), nU)
    s = rng.choice([-1, 1], size=u.size)
    g = synth.from_edges(nU, nV, u, v, s)
    c = same(ctx, g)
    assert c.total == nU * (nU - 1) // 2 * 6


def test_high_degree_star_and_invalid_inputs(ctx):
    # a V vertex of degree 65,536 (above the 16-bit tally range) is counted:
    # a star has no butterflies
    star = synth.from_edges(65_536, 1, np.arange(65_536), np.zeros(65_536, np.int64),
                            np.ones(65_536))
    c = ctx.count(star)
    assert (c.balanced, c.total) == (0, 0) == oracle.count(star)
    base = synth.from_edges(2, 3, [0, 0, 1], [0, 1, 2], [1, -1, 1])
    bad = [
        synth.SignedBipartite(2, 3, base.rowptr, base.col, np.array([1, 0, 1], np.int8)),
        synth.SignedBipartite(2, 3, base.rowptr, np.array([0, 3, 1], np.int32), base.sign),
        synth.SignedBipartite(2, 3, np.array([0, 2, 3]), np.array([1, 1, 0], np.int32),
                              np.array([1, -1, 1], np.int8)),
        synth.SignedBipartite(2, 3, np.array([0, 3, 2]), base.col, base.sign),
    ]
    for g in bad:
        with pytest.raises(pkg.BBError) as ei:
            ctx.count(g)
        assert ei.value.name == "BB_ERR_INVALID_ARG"
    # the context stays usable after rejected inputs
    same(ctx, synth.uniform(3, 50, 50, 600, 0.5))


@pytest.mark.parametrize("length", [2, 3, 5, 17, 33, 100, 300, 600, 3000])
def test_duplicate_edge_found_in_every_row_sort(ctx, length):
    # one edge listed twice in a row of `length` entries, on the U side
    # (one U vertex's row) and on the V side (one V vertex's row): each row
    # length class is sorted by a different kernel, and each must report it
    rng = np.random.default_rng(length)
    nbrs = rng.choice(4 * length, length, replace=False)
    u_side = synth.SignedBipartite(
        1, 4 * length, np.array([0, length + 1], np.int64),
        np.concatenate([nbrs, nbrs[:1]]).astype(np.int32), np.ones(length + 1, np.int8),
        f"dup in a U row of {length}")
    rows = np.concatenate([np.arange(length), [length // 2]])
    order = np.argsort(rows, kind="stable")
    v_side = synth.SignedBipartite(
        length, 1, np.searchsorted(rows[order], np.arange(length + 1)).astype(np.int64),
        np.zeros(length + 1, np.int32), np.ones(length + 1, np.int8), f"dup in a V row of {length}")
    for g in (u_side, v_side):
        with pytest.raises(pkg.BBError) as ei:
            ctx.count(g)
        assert ei.value.name == "BB_ERR_INVALID_ARG", g.name
    same(ctx, synth.uniform(5, 40, 40, 500, 0.5))


def test_budget_is_enforced():
    with pkg.Context(0, budget_bytes=1 << 20) as small:
        with pytest.raises(pkg.BBError) as ei:
            small.count(synth.chung_lu_scaled(3, 200_000))
        assert ei.value.name == "BB_ERR_BUDGET"


def test_device_inputs_match_host_inputs(ctx):
    torch = pytest.importorskip("torch")
    g = synth.chung_lu_scaled(41, 200_000)
    rec = EXPECTED["chunglu_m200000_s41"]
    rp = torch.from_numpy(g.rowptr).cuda()
    cl = torch.from_numpy(g.col).cuda()
    sg = torch.from_numpy(g.sign).cuda()
    torch.cuda.synchronize()
    c = ctx.count_tensors(g.nV, rp, cl, sg)
    assert (c.balanced, c.total) == (rec["balanced"], rec["total"])
    h = ctx.count(g)
    assert (h.balanced, h.total, h.wedges) == (c.balanced, c.total, c.wedges)


def test_resident_graph_and_sign_flips(ctx):
    g = synth.chung_lu_scaled(43, 100_000)
    want = oracle.count(g)
    G = ctx.upload(g)
    c = G.count()
    assert (c.balanced, c.total) == want
    assert c.wedges == priority_wedges(g)
    rng = np.random.default_rng(5)
    idx = rng.choice(g.nE, size=g.nE // 100, replace=False)
    G.flip(idx)
    s2 = g.sign.copy()
    s2[idx] = -s2[idx]
    g2 = synth.SignedBipartite(g.nU, g.nV, g.rowptr, g.col, s2)
    c2 = G.count()
    assert (c2.balanced, c2.total) == oracle.count(g2)
    G.flip(idx)
    c3 = G.count()
    assert (c3.balanced, c3.total) == want
    G.free()


def test_repeat_calls_identical(ctx):
    g = synth.chung_lu_scaled(44, 300_000)
    a = ctx.count(g)
    for _ in range(3):
        b = ctx.count(g)
        assert tuple(a) == tuple(b)


# ---------------------------------------------- stored full-size workloads
def _check_stored(ctx, name, make):
    rec = EXPECTED[name]
    g = make()
    assert g.nE == rec["nE"]
    c = ctx.count(g)
    assert (c.balanced, c.total) == (rec["balanced"], rec["total"]), (name, c, rec)
    return g, c


def test_vote_500_50k(ctx):
    _check_stored(ctx, "vote_500x50000_p0.4_b2", synth.vote_500_50k)


def test_chunglu_2m_scaled(ctx):
    _check_stored(ctx, "chunglu_m2000000_s43", lambda: synth.chung_lu_scaled(43, 2_000_000))


def test_chunglu_2m_x_500k_full(ctx):
    """The bench workload at full size: exact counts, the switching
    invariance (negate all edges at a random vertex set) and all-positive
    balanced == total, evaluated on the GPU."""
    g, c = _check_stored(ctx, "chunglu_2Mx500k_e20M_a2.1_p0.8", synth.chung_lu_2m)
    rng = np.random.default_rng(11)
    u, v, s = g.edges()
    xu = rng.choice([-1, 1], size=g.nU).astype(np.int8)
    yv = rng.choice([-1, 1], size=g.nV).astype(np.int8)
    g2 = synth.SignedBipartite(g.nU, g.nV, g.rowptr, g.col, (s * xu[u] * yv[v]).astype(np.int8))
    c2 = ctx.count(g2)
    assert (c2.balanced, c2.total) == (c.balanced, c.total)
    g3 = synth.SignedBipartite(g.nU, g.nV, g.rowptr, g.col, np.ones_like(g.sign))
    c3 = ctx.count(g3)
    assert c3.balanced == c3.total == c.total


# ------------------------------------------------------- per-vertex counts
@pytest.mark.parametrize("make", [
    lambda: synth.uniform(61, 30, 25, 300, 0.6),
    lambda: synth.uniform_2k_1k(),
    lambda: synth.chung_lu_scaled(62, 60_000),
    lambda: synth.vote(63, 80, 6_000, 0.4, 2, 0.55, 0.8),
])
def test_per_vertex_matches_oracle(ctx, make):
    g = make()
    c = ctx.count(g, per_vertex=True)
    want = oracle.per_vertex(g, threads=4)
    assert np.array_equal(c.per_vertex, want)
    assert c.per_vertex[: g.nU].sum() == 2 * c.balanced
    assert c.per_vertex[g.nU:].sum() == 2 * c.balanced


@pytest.mark.parametrize("n_other", [60_000, 4_400_000])
def test_long_rows_both_row_sorts(ctx, n_other):
    # rows above 2,048 entries: sorted through a bitmap over the other
    # side's ranks when that side has at most 8 * 2^19 vertices, by the
    # per-row radix sort beyond; most of the 4.4M vertices are isolated
    rng = np.random.default_rng(n_other)
    us, vs = [], []
    for v, d in enumerate((3_000, 2_500, 40)):
        us.append(rng.choice(min(n_other, 20_000), d, replace=False) * (n_other // 20_000))
        vs.append(np.full(d, v))
    u, v = np.concatenate(us), np.concatenate(vs)
    g = synth.from_edges(n_other, 3, u, v, rng.choice([-1, 1], size=u.size), f"long rows {n_other}")
    want = oracle.count(g, threads=4)
    for h in (g, synth.swap_sides(g)):
        c = ctx.count(h)
        assert (c.balanced, c.total) == want, h.name


def test_per_vertex_tiny_and_windowed(ctx):
    for seed in range(40):
        rng = np.random.default_rng(700 + seed)
        nU, nV = int(rng.integers(1, 12)), int(rng.integers(1, 12))
        g = synth.uniform(700 + seed, nU, nV, int(rng.integers(0, nU * nV + 1)), 0.5)
        assert np.array_equal(ctx.count(g, per_vertex=True).per_vertex, oracle.per_vertex(g))
    # K_{60000,4}: dense windows over the endpoint range
    rng = np.random.default_rng(8)
    u = np.repeat(np.arange(60_000), 4)
    v = np.tile(np.arange(4), 60_000)
    g = synth.from_edges(60_000, 4, u, v, rng.choice([-1, 1], size=u.size))
    ids = np.array([0, 1, 59_999, 30_000, 60_000, 60_001, 60_003])
    pv = ctx.count(g, per_vertex=True).per_vertex
    assert np.array_equal(pv[ids], oracle.per_vertex(g, ids))


def test_per_vertex_resident_and_device(ctx):
    torch = pytest.importorskip("torch")
    g = synth.chung_lu_scaled(64, 80_000)
    want = oracle.per_vertex(g, threads=4)
    G = ctx.upload(g)
    assert np.array_equal(G.count(per_vertex=True).per_vertex, want)
    G.free()
    rp = torch.from_numpy(g.rowptr).cuda()
    cl = torch.from_numpy(g.col).cuda()
    sg = torch.from_numpy(g.sign).cuda()
    out = torch.zeros(g.nU + g.nV, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    ctx.count_tensors(g.nV, rp, cl, sg, per_vertex=out)
    assert np.array_equal(out.cpu().numpy(), want)


@pytest.mark.parametrize("name,make", [
    ("vote_500x50000_p0.4_b2", synth.vote_500_50k),
    ("chunglu_2Mx500k_e20M_a2.1_p0.8", synth.chung_lu_2m),
])
def test_per_vertex_full_size_sampled(ctx, name, make):
    rec = EXPECTED[name]
    g = make()
    c = ctx.count(g, per_vertex=True)
    assert (c.balanced, c.total) == (rec["balanced"], rec["total"])
    ids = np.array(rec["per_vertex_gids"])
    assert np.array_equal(c.per_vertex[ids], np.array(rec["per_vertex"]))
    assert c.per_vertex[: g.nU].sum() == 2 * c.balanced
    assert c.per_vertex[g.nU:].sum() == 2 * c.balanced


# Bucket shapes that move anchors between the classes: most anchors out of
# the warp class with small split dense parts, warp anchors hashing every
# endpoint, and a mix. The per-vertex and per-edge walks of every class
# (including split parts and their second launch) must give the oracle's
# values under each.
PV_SHAPES = [
    {"warp_w_max": 64, "warp_small_w": 0, "team_w_max": 256, "split_wedges": 1024},
    {"warp_w_max": 16384, "warp_small_w": 16384, "team_w_max": 16384, "split_wedges": 1 << 20},
    {"warp_w_max": 2048, "warp_small_w": 96, "team_w_max": 4096, "split_wedges": 16384},
]


@pytest.mark.parametrize("shape", range(len(PV_SHAPES)))
@pytest.mark.parametrize("make", [
    lambda: synth.chung_lu_scaled(65, 60_000),
    lambda: synth.vote(66, 60, 5_000, 0.4, 2, 0.55, 0.8),
])
def test_per_vertex_and_edge_under_bucket_shapes(ctx, make, shape):
    g = make()
    want_v = oracle.per_vertex(g, threads=4)
    want_e = oracle.per_edge(g, threads=8)
    r = ctx.upload(g)
    try:
        r.set_shape(PV_SHAPES[shape])
        for _ in range(2):  # the split parts' merged counters are released for the next call
            c = r.count(per_vertex=True)
            assert np.array_equal(c.per_vertex, want_v), g.name
            pe, b, t = r.count_edges()
            assert np.array_equal(pe, want_e), g.name
            assert (b, t) == (c.balanced, c.total)
        assert (r.count().balanced, r.count().total) == (c.balanced, c.total)
    finally:
        r.free()


# ------------------------------------------------------------- per edge
@pytest.mark.parametrize("make", [
    lambda: synth.uniform_2k_1k(),
    lambda: synth.chung_lu_scaled(41, 200_000),
    lambda: synth.vote(7, 40, 3_000, 0.4, 2, 0.55, 0.8),
    lambda: synth.from_dense(np.ones((5, 7), dtype=np.int8)),
])
def test_per_edge_matches_oracle(ctx, make):
    g = make()
    r = ctx.upload(g)
    pe, b, t = r.count_edges()
    want = oracle.per_edge(g, threads=8)
    assert np.array_equal(pe, want), g.name
    assert (b, t) == oracle.count(g, threads=4)
    assert int(pe.sum()) == 4 * b
    # after sign flips of 1 % of the edges, and back
    idx = np.random.default_rng(3).choice(g.nE, max(1, g.nE // 100), replace=False)
    r.flip(idx)
    s = g.sign.copy()
    s[idx] = -s[idx]
    h = synth.SignedBipartite(g.nU, g.nV, g.rowptr, g.col, s, g.name + "/f")
    assert np.array_equal(r.count_edges()[0], oracle.per_edge(h, threads=8))
    r.flip(idx)
    assert np.array_equal(r.count_edges()[0], want)
    r.free()


def test_per_edge_tiny_and_degenerate(ctx):
    for signs in ([1, 1, 1, 1], [1, -1, 1, 1], [-1, -1, 1, 1]):
        g = synth.from_edges(2, 2, [0, 1, 0, 1], [0, 0, 1, 1], signs)
        r = ctx.upload(g)
        assert np.array_equal(r.count_edges()[0], oracle.per_edge(g))
        r.free()
    for g in (synth.from_edges(3, 4, [], [], []), synth.from_edges(1, 5, [0] * 5, range(5), [1] * 5)):
        r = ctx.upload(g)
        pe, b, t = r.count_edges()
        assert pe.size == g.nE and not pe.any() and (b, t) == (0, 0)
        r.free()
    for seed in range(20):
        rng = np.random.default_rng(seed)
        nU, nV = int(rng.integers(2, 12)), int(rng.integers(2, 12))
        g = synth.uniform(4000 + seed, nU, nV, int(rng.integers(0, nU * nV + 1)), 0.5)
        r = ctx.upload(g)
        assert np.array_equal(r.count_edges()[0], oracle.per_edge(g)), seed
        r.free()


@pytest.mark.parametrize("name,make", [("chunglu_2Mx500k_e20M_a2.1_p0.8", "chung_lu_2m"),
                                       ("vote_500x50000_p0.4_b2", "vote_500_50k")])
def test_per_edge_full_size_sampled(ctx, name, make):
    g = getattr(synth, make)()
    r = ctx.upload(g)
    pe, b, t = r.count_edges()
    want = EXPECTED[name]
    assert (b, t) == (want["balanced"], want["total"])
    assert int(pe.sum()) == 4 * b
    # sampled edges against the oracle, including the edges of the densest rows
    rng = np.random.default_rng(11)
    deg = np.diff(g.rowptr)
    hub = int(np.argmax(deg))
    idx = np.concatenate([rng.choice(g.nE, 60, replace=False),
                          np.arange(g.rowptr[hub], g.rowptr[hub] + 5)])
    assert np.array_equal(pe[idx], oracle.per_edge(g, idx, threads=16))
    r.free()
