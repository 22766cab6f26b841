"""GPU parity of the matrix-product path: graphs whose smaller side is small
and dense are counted from X X^T and |X| |X|^T (Lemma 2 per pair of that
side) instead of by wedges. Every count is checked bit-exactly against the
CPU oracle, against the wedge kernels on the same graph, and, for the
largest case, against NumPy int64 products."""
import numpy as np
import pytest

import oracle
import paper_2308_07932_gb300 as pkg
from paper_2308_07932_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.product]


@pytest.fixture(scope="module")
def ctx():
    c = pkg.Context(0)
    c.set_timing(True)
    yield c
    c.close()


@pytest.fixture(autouse=True)
def product_on():
    prev = pkg.set_matrix_product(True)
    yield
    pkg.set_matrix_product(prev)


def dense_graph(seed, a, b, density, p_pos=0.6):
    rng = np.random.default_rng(seed)
    A = np.where(rng.random((a, b)) < density, np.where(rng.random((a, b)) < p_pos, 1, -1), 0)
    return synth.from_dense(A.astype(np.int8))


def pair_sums(A):
    """Lemma 2 over the pairs of rows of a dense {-1, 0, 1} matrix, with
    NumPy int64 products (rows = the pair side)."""
    X = A.astype(np.int64)
    D = X @ X.T
    N = np.abs(X) @ np.abs(X).T
    iu = np.triu_indices(A.shape[0], 1)
    d, n = D[iu], N[iu]
    S, Aa = (n + d) // 2, (n - d) // 2
    c2 = lambda x: x * (x - 1) // 2
    return int((c2(S) + c2(Aa)).sum()), int(c2(n).sum())


def counted_by_product(ctx):
    t = ctx.last_timing()
    return t["product_ms"] > 0 and all(k["ms"] == 0 for k in t["kernels"].values())


def check_both_paths(ctx, g, want):
    assert pkg.matrix_product_plan(g.nU, g.nV, g.nE), g.name
    c = ctx.count(g)
    assert (c.balanced, c.total) == want, (g.name, "product", c, want)
    assert counted_by_product(ctx)
    prev = pkg.set_matrix_product(False)
    try:
        assert not pkg.matrix_product_plan(g.nU, g.nV, g.nE)
        w = ctx.count(g)
        assert (w.balanced, w.total) == want, (g.name, "wedges", w, want)
        assert not counted_by_product(ctx)
        assert w.wedges == c.wedges  # the reported wedge count is the graph's either way
    finally:
        pkg.set_matrix_product(prev)
    return c


def test_vote_graphs_both_orientations(ctx):
    for seed, a, b in [(11, 64, 6000), (12, 200, 2500), (13, 37, 9001)]:
        g = synth.vote(seed, a, b, 0.4, 2, 0.55, 0.8)
        want = oracle.count(g, threads=4)
        check_both_paths(ctx, g, want)
        gs = synth.swap_sides(g)  # pair side V
        check_both_paths(ctx, gs, want)


def test_ragged_widths_and_empty_rows(ctx):
    # middle counts that are not multiples of 8 (padded matrix rows), empty
    # rows on both sides, all-positive and all-negative rows
    for seed, a, b, dens in [(21, 40, 4099, 0.6), (22, 8, 65_537, 0.3), (23, 129, 1_023, 0.9)]:
        D = synth.to_dense(dense_graph(seed, a, b, dens))
        D[a // 2, :] = 0                    # an isolated pair-side vertex
        D[:, : b // 7] = 0                  # isolated middles
        D[1, D[1] != 0] = 1                 # an all-positive row
        D[2, D[2] != 0] = -1                # an all-negative row
        g = synth.from_dense(D)
        want = oracle.count(g, threads=4)
        assert want == pair_sums(D)
        check_both_paths(ctx, g, want)


def test_complete_graphs_closed_form(ctx):
    # K_{m,n} with all signs +1: balanced = total = C(m,2) C(n,2)
    for m, n in [(2, 40_000), (3, 30_000), (16, 4_101)]:
        g = synth.from_dense(np.ones((m, n), np.int8))
        want = (m * (m - 1) // 2 * (n * (n - 1) // 2),) * 2
        check_both_paths(ctx, g, want)


def test_pair_tallies_near_the_exactness_bound(ctx):
    # 4 full rows of 2^21 - 1 middles: every pair's S + A is 2^21 - 1, the
    # largest sum the plan admits
    b = (1 << 21) - 1
    rng = np.random.default_rng(31)
    D = np.where(rng.random((4, b)) < 0.5, 1, -1).astype(np.int8)
    g = synth.from_dense(D)
    assert pkg.matrix_product_plan(g.nU, g.nV, g.nE)
    want = pair_sums(D)
    c = ctx.count(g)
    assert (c.balanced, c.total) == want
    assert counted_by_product(ctx)


def test_device_inputs_replay_and_resident_graphs(ctx):
    torch = pytest.importorskip("torch")
    g = synth.vote(41, 96, 12_000, 0.4, 2, 0.55, 0.8)
    want = oracle.count(g, threads=4)
    dev = torch.device("cuda", 0)
    rp, cl, sg = (torch.from_numpy(x).to(dev) for x in (g.rowptr, g.col, g.sign))
    # the second and third calls replay a captured step
    for _ in range(3):
        c = ctx.count_device(g.nU, g.nV, g.nE, rp.data_ptr(), cl.data_ptr(), sg.data_ptr())
        assert (c.balanced, c.total) == want
        assert counted_by_product(ctx)
    prev = pkg.set_matrix_product(False)
    try:  # a changed mode is captured afresh
        for _ in range(2):
            c = ctx.count_device(g.nU, g.nV, g.nE, rp.data_ptr(), cl.data_ptr(), sg.data_ptr())
            assert (c.balanced, c.total) == want
            assert not counted_by_product(ctx)
    finally:
        pkg.set_matrix_product(prev)
    c = ctx.count_device(g.nU, g.nV, g.nE, rp.data_ptr(), cl.data_ptr(), sg.data_ptr())
    assert (c.balanced, c.total) == want and counted_by_product(ctx)
    G = ctx.upload(g)
    try:
        c = G.count()
        assert (c.balanced, c.total) == want and counted_by_product(ctx)
        # per-vertex counts take the wedge kernels on the same resident graph
        pv = G.count(per_vertex=True)
        assert (pv.balanced, pv.total) == want
        assert not counted_by_product(ctx)
        np.testing.assert_array_equal(pv.per_vertex, oracle.per_vertex(g, threads=4))
    finally:
        G.free()


def test_allocation_free_call_keeps_the_wedge_kernels():
    torch = pytest.importorskip("torch")
    import ctypes
    g = synth.vote(51, 40, 4_000, 0.5, 2, 0.55, 0.8)
    assert pkg.matrix_product_plan(g.nU, g.nV, g.nE)
    want = oracle.count(g, threads=4)
    dev = torch.device("cuda", 0)
    rp, cl, sg = (torch.from_numpy(x).to(dev) for x in (g.rowptr, g.col, g.sign))
    csr = pkg._Csr(g.nU, g.nV, g.nE, rp.data_ptr(), cl.data_ptr())
    b, t, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    st = pkg.lib().bb_count_csr_device_noalloc(ctypes.byref(csr), ctypes.c_void_p(sg.data_ptr()),
                                               None, ctypes.byref(b), ctypes.byref(t),
                                               ctypes.byref(w))
    assert st == 0
    assert (b.value, t.value) == want


def test_duplicate_edge_is_reported_on_the_product_path(ctx):
    g = synth.vote(61, 48, 5_000, 0.4, 2, 0.55, 0.8)
    u, v, s = g.edges()
    for k in (0, len(u) // 2, len(u) - 1):  # first, middle and last edge listed twice
        d = synth.from_edges(g.nU, g.nV, np.append(u, u[k]), np.append(v, v[k]),
                             np.append(s, -s[k]), "dup")
        assert pkg.matrix_product_plan(d.nU, d.nV, d.nE)
        with pytest.raises(pkg.BBError) as ei:
            ctx.count(d)
        assert ei.value.name == "BB_ERR_INVALID_ARG"
        assert "twice" in str(ei.value)
    c = ctx.count(g)  # the context is usable afterwards
    assert (c.balanced, c.total) == oracle.count(g, threads=4)


def test_flips_on_a_product_graph_recount_exactly(ctx):
    # a resident graph counted by the products: flips recount (no walk) and
    # the counts follow the oracle on the flipped graph
    g = synth.vote(71, 64, 6_000, 0.4, 2, 0.55, 0.8)
    G = ctx.upload(g)
    try:
        c = G.count()
        assert (c.balanced, c.total) == oracle.count(g, threads=4) and counted_by_product(ctx)
        sign = g.sign.copy()
        rng = np.random.default_rng(72)
        for k in (10, 1000):
            idx = rng.choice(g.nE, size=k, replace=False)
            b, t, inc = G.count_flipped(idx)
            sign[idx] = -sign[idx]
            fl = synth.SignedBipartite(g.nU, g.nV, g.rowptr, g.col, sign, g.name + "/f")
            assert (b, t) == oracle.count(fl, threads=4)
            assert not inc
    finally:
        G.free()
