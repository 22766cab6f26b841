"""Vertices of degree above 65,535 (wide anchors): their per-pair tallies
need 32-bit fields. Checked against Lemma 2's closed forms on complete
bipartite graphs and against the oracle on power-law graphs with hubs, for
counts, per-vertex and per-edge outputs, on both sides."""
from math import comb

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


def k2n(n, l):
    """K_{2,n}: u0 all positive, u1 positive on the first l middles and
    negative on the rest, so l middles are symmetric (Def. 5) and n - l
    asymmetric (Def. 6)."""
    u = np.concatenate([np.zeros(n, np.int64), np.ones(n, np.int64)])
    v = np.concatenate([np.arange(n), np.arange(n)])
    s = np.concatenate([np.ones(n), np.where(np.arange(n) < l, 1, -1)])
    return synth.from_edges(2, n, u, v, s, f"K2,{n}/l={l}")


def lemma2(n, l):
    """(balanced, total) of k2n by Lemma 2: one pair with l symmetric and
    n - l asymmetric wedges."""
    return comb(l, 2) + comb(n - l, 2), comb(n, 2)


@pytest.mark.parametrize("n,l", [(65_535, 65_535), (65_535, 30_000), (65_535, 0),
                                 (70_000, 70_000), (70_000, 40_000), (131_072, 65_536)])
def test_k2n_lemma2_at_and_above_16_bits(ctx, n, l):
    # n = 65,535: every tally of the one pair reaches the 16-bit maximum
    # (no carry into the other field); above it the pair is a wide anchor
    g = k2n(n, l)
    want = lemma2(n, l)
    for h in (g, synth.swap_sides(g)):
        c = ctx.count(h)
        assert (c.balanced, c.total) == want, (h.name, c, want)


def test_k2n_per_vertex_and_per_edge_wide(ctx):
    n, l = 70_000, 40_000
    g = k2n(n, l)
    b, _ = lemma2(n, l)
    sym = np.arange(n) < l
    # a middle of type t lies in cnt_t - 1 balanced butterflies (both
    # middles of a balanced butterfly share a type), each u in all of them
    want_v = np.where(sym, l - 1, n - l - 1)
    res = ctx.upload(g)
    try:
        c = res.count(per_vertex=True)
        assert (c.balanced, c.per_vertex[0], c.per_vertex[1]) == (b, b, b)
        assert np.array_equal(c.per_vertex[2:], want_v)
        pe, bb, _ = res.count_edges()
        assert bb == b
        u, v, _ = g.edges()
        assert np.array_equal(pe, want_v[v])
    finally:
        res.free()


def hub_graph(seed, hub_deg=(100_000, 110_000)):
    """A power-law graph (Chung-Lu recipe, 20k x 150k) plus two U hubs of
    the given degrees on uniform random V vertices: the lower hub is a wide
    anchor whose endpoint is the higher one, and both are endpoints of the
    other U anchors."""
    base = synth.chung_lu(seed, 20_000, 150_000, 420_000, 2.1, 2.1, 50_000.0, 0.8)
    u, v, s = base.edges()
    rng = np.random.default_rng(seed)
    hu, hv, hs = [u], [v], [s]
    for k, d in enumerate(hub_deg):
        nbr = rng.choice(base.nV, d, replace=False)
        hu.append(np.full(d, base.nU + k))
        hv.append(nbr)
        hs.append(np.where(rng.random(d) < 0.7, 1, -1))
    return synth.from_edges(base.nU + len(hub_deg), base.nV, np.concatenate(hu),
                            np.concatenate(hv), np.concatenate(hs), f"hubs{seed}")


@pytest.mark.parametrize("swap", [False, True])
def test_power_law_with_wide_hubs(ctx, swap):
    g = hub_graph(61)
    if swap:
        g = synth.swap_sides(g)
    deg = np.concatenate([np.diff(g.rowptr), np.bincount(g.col, minlength=g.nV)])
    assert (deg > 65_535).sum() == 2
    want = oracle.count(g, threads=8)
    c = ctx.count(g)
    assert (c.balanced, c.total) == want
    res = ctx.upload(g)
    try:
        r = res.count(per_vertex=True)
        assert (r.balanced, r.total) == want
        assert int(r.per_vertex.sum()) == 4 * want[0]
        hubs = np.nonzero(deg > 65_535)[0]
        rng = np.random.default_rng(5)
        gids = np.unique(np.concatenate([hubs, rng.choice(g.nU + g.nV, 40, replace=False)]))
        exp = oracle.per_vertex(g, gids=gids, threads=8)
        assert np.array_equal(r.per_vertex[gids], exp)
        pe, bb, _ = res.count_edges()
        assert bb == want[0] and int(pe.sum()) == 4 * want[0]
        eids = np.unique(rng.choice(g.nE, 60, replace=False))
        assert np.array_equal(pe[eids], oracle.per_edge(g, edges=eids, threads=8))
    finally:
        res.free()


def test_wide_members_in_a_batch(ctx):
    # the batched dense kernel walks wide jobs itself
    hosts = [k2n(70_000, 40_000), synth.swap_sides(k2n(131_072, 65_536)), hub_graph(62),
             synth.uniform_2k_1k()]
    want = [lemma2(70_000, 40_000), lemma2(131_072, 65_536), oracle.count(hosts[2], threads=8),
            oracle.count(hosts[3])]
    graphs = [ctx.upload(g) for g in hosts]
    try:
        b = pkg.Batch(ctx, graphs)
        for _ in range(2):
            bal, tot = b.count()
            assert [(int(x), int(y)) for x, y in zip(bal, tot)] == want
        b.free()
    finally:
        for g in graphs:
            g.free()
