"""Pins for the CPU oracle: facts fixed by the paper and by mathematics,
independent of the oracle's own code.

  * Fig. 1 / Def. 2: the six signed butterflies (golden fixture);
  * Lemma 2: a pair with l symmetric and m asymmetric wedges holds
    C(l,2)+C(m,2) balanced butterflies out of C(l+m,2);
  * complete graphs K_{m,n}: C(m,2)C(n,2) butterflies, all balanced when the
    signs factor as x_u * y_v (switching-equivalent to all positive);
  * brute force over all vertex 4-tuples, written here in Python;
  * the dense closed form from two float64 matrix products (a library GEMM);
  * invariants: vertex switching, sign flips (total), side swap, relabelling,
    per-vertex sums equal twice the balanced count;
  * planted mistakes in the oracle (compile-time variants) each break a pin.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2308_07932_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------- test helpers
def brute_force(g):
    """Defs. 1-2 written out: every (u1<u2, v1<v2) with all four edges is a
    butterfly; it is balanced when the product of its four signs is +1."""
    sign = {}
    u, v, s = g.edges()
    for a, b, c in zip(u.tolist(), v.tolist(), s.tolist()):
        sign[(a, b)] = c
    bal = tot = 0
    pv = [0] * (g.nU + g.nV)
    for u1, u2 in itertools.combinations(range(g.nU), 2):
        for v1, v2 in itertools.combinations(range(g.nV), 2):
            e = [(u1, v1), (u1, v2), (u2, v1), (u2, v2)]
            if all(x in sign for x in e):
                tot += 1
                if sign[e[0]] * sign[e[1]] * sign[e[2]] * sign[e[3]] == 1:
                    bal += 1
                    for x in (u1, u2):
                        pv[x] += 1
                    for y in (v1, v2):
                        pv[g.nU + y] += 1
    return bal, tot, np.array(pv, dtype=np.int64)


def dense_closed_form(g):
    """With the signed biadjacency A, M = A A^T and C = |A||A|^T: for a pair
    u1 < u2, P + N = C and P - N = M, hence total = sum C(C,2) and
    balanced = sum (C^2 + M^2 - 2C)/4. float64 products are exact here
    (integer entries far below 2^53)."""
    A = synth.to_dense(g).astype(np.float64)
    M = A @ A.T
    C = np.abs(A) @ np.abs(A).T
    iu = np.triu_indices(g.nU, 1)
    Mi = M[iu].astype(np.int64)
    Ci = C[iu].astype(np.int64)
    total = int((Ci * (Ci - 1) // 2).sum())
    balanced = int(((Ci * Ci + Mi * Mi - 2 * Ci) // 4).sum())
    return balanced, total


def read_fig1():
    rows = []
    with open(os.path.join(GOLDEN, "fig1_signed_butterflies.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows.append((p[0], p[1], [int(x) for x in p[2:6]], int(p[6]), int(p[7])))
    return rows


def fig1_graph(signs):
    # U = {u_i=0, u_j=1}, V = {v_i=0, v_j=1}; signs are s(v_i,u_i) s(v_i,u_j) s(v_j,u_i) s(v_j,u_j)
    return synth.from_edges(2, 2, [0, 1, 0, 1], [0, 0, 1, 1], signs)


def k2n(l, m, seed=0):
    """K_{2,l+m}: l middles with equal signs to both U vertices (symmetric
    wedges), m with opposite signs (asymmetric wedges)."""
    rng = np.random.default_rng(seed)
    us, vs, ss = [], [], []
    for v in range(l + m):
        a = int(rng.choice([-1, 1]))
        b = a if v < l else -a
        us += [0, 1]
        vs += [v, v]
        ss += [a, b]
    return synth.from_edges(2, l + m, us, vs, ss)


def c2(n):
    return n * (n - 1) // 2


# ------------------------------------------------------- the pins (reused)
def pin_fig1(count):
    for panel, caption, signs, bal, tot in read_fig1():
        assert count(fig1_graph(signs)) == (bal, tot), panel


def pin_lemma2(count):
    for l in range(0, 7):
        for m in range(0, 7):
            g = k2n(l, m, seed=10 * l + m)
            assert count(g) == (c2(l) + c2(m), c2(l + m)), (l, m)


def pin_complete(count):
    rng = np.random.default_rng(5)
    for mU, nV in [(2, 2), (3, 5), (7, 4), (9, 9)]:
        x = rng.choice([-1, 1], size=mU)
        y = rng.choice([-1, 1], size=nV)
        g = synth.from_dense(np.outer(x, y))
        want = c2(mU) * c2(nV)
        assert count(g) == (want, want), (mU, nV)
        R = rng.choice([-1, 1], size=(mU, nV))
        assert count(synth.from_dense(R))[1] == want


def pin_brute(count, seeds=range(40)):
    for seed in seeds:
        rng = np.random.default_rng(seed)
        nU, nV = int(rng.integers(2, 9)), int(rng.integers(2, 9))
        m = int(rng.integers(0, nU * nV + 1))
        g = synth.uniform(1000 + seed, nU, nV, m, float(rng.uniform(0.2, 0.8)))
        b, t, _ = brute_force(g)
        assert count(g) == (b, t), seed


PINS = [pin_fig1, pin_lemma2, pin_complete, pin_brute]


def oracle_count_fn(mutant=0, side=-1):
    return lambda g: oracle.count(g, side=side, mutant=mutant)


# ------------------------------------------------------------------ tests
@pytest.mark.parametrize("side", [-1, 0, 1])
def test_fig1_six_butterflies(side):
    pin_fig1(oracle_count_fn(side=side))
    for panel, caption, signs, bal, tot in read_fig1():
        g = fig1_graph(signs)
        assert oracle.bb_base(g) == (bal, tot)
        assert brute_force(g)[:2] == (bal, tot)
        assert list(oracle.per_vertex(g)) == [bal] * 4


def test_fig1_caption_matches_signs():
    # the caption lists the signs; balance = even number of '-' (Def. 2)
    for panel, caption, signs, bal, tot in read_fig1():
        assert sorted(caption) == sorted("+" if s > 0 else "-" for s in signs)
        assert bal == (1 if caption.count("-") % 2 == 0 else 0)


@pytest.mark.parametrize("side", [-1, 0, 1])
def test_lemma2_closed_form(side):
    pin_lemma2(oracle_count_fn(side=side))


def test_lemma2_per_vertex():
    for l, m in [(0, 0), (1, 0), (3, 0), (0, 4), (2, 3), (5, 6)]:
        g = k2n(l, m, seed=l * 7 + m)
        pv = oracle.per_vertex(g)
        bal = c2(l) + c2(m)
        assert pv[0] == bal and pv[1] == bal
        want_v = [max(l - 1, 0)] * l + [max(m - 1, 0)] * m
        assert list(pv[2:]) == want_v


def test_complete_bipartite():
    pin_complete(oracle_count_fn())
    g = synth.from_dense(np.ones((6, 8), dtype=np.int8))
    want = c2(6) * c2(8)
    assert oracle.count(g) == (want, want)
    assert oracle.bb_base(g) == (want, want)


def test_brute_force_tiny_graphs():
    pin_brute(oracle_count_fn(), seeds=range(120))


def test_brute_force_per_vertex():
    for seed in range(60):
        rng = np.random.default_rng(seed)
        nU, nV = int(rng.integers(2, 10)), int(rng.integers(2, 10))
        g = synth.uniform(2000 + seed, nU, nV, int(rng.integers(0, nU * nV + 1)), 0.6)
        b, t, pv = brute_force(g)
        assert np.array_equal(oracle.per_vertex(g), pv), seed
        cb, ct, cpv = oracle.brute(g, with_per_vertex=True)
        assert (cb, ct) == (b, t) and np.array_equal(cpv, pv)


def test_bb_base_agrees():
    graphs = [synth.uniform(s, 60, 40, 900, 0.6) for s in range(5)]
    graphs += [synth.chung_lu_scaled(7, 20_000), synth.uniform_2k_1k()]
    for g in graphs:
        assert oracle.bb_base(g) == oracle.count(g), g.name


def test_both_sides_agree():
    for g in [synth.uniform(3, 300, 100, 5000, 0.7), synth.chung_lu_scaled(11, 50_000),
              synth.vote(3, 40, 400, 0.4, 2, 0.55, 0.8)]:
        assert oracle.count(g, side=0) == oracle.count(g, side=1), g.name


def test_dense_closed_form_uniform_2k_1k():
    g = synth.uniform_2k_1k()
    assert oracle.count(g) == dense_closed_form(g)


def test_dense_closed_form_vote_and_powerlaw():
    for g in [synth.vote(9, 200, 5000, 0.4, 2, 0.55, 0.8), synth.chung_lu_scaled(3, 30_000)]:
        assert oracle.count(g, threads=4) == dense_closed_form(g), g.name


@pytest.mark.slow
def test_dense_closed_form_vote_500_50k():
    g = synth.vote_500_50k()
    assert oracle.count(g, threads=oracle.default_threads()) == dense_closed_form(g)


def test_switching_and_flip_invariance():
    g = synth.uniform(21, 400, 150, 6000, 0.65)
    b0, t0 = oracle.count(g)
    rng = np.random.default_rng(0)
    u, v, s = g.edges()
    # vertex switching: negate every edge at a random set of vertices
    xu = rng.choice([-1, 1], size=g.nU)
    yv = rng.choice([-1, 1], size=g.nV)
    g2 = synth.from_edges(g.nU, g.nV, u, v, s * xu[u] * yv[v])
    assert oracle.count(g2) == (b0, t0)
    # flipping arbitrary edge signs keeps the total
    flip = rng.random(s.size) < 0.3
    g3 = synth.from_edges(g.nU, g.nV, u, v, np.where(flip, -s, s))
    assert oracle.count(g3)[1] == t0
    # all positive: every butterfly is balanced
    g4 = synth.from_edges(g.nU, g.nV, u, v, np.ones_like(s))
    assert oracle.count(g4) == (t0, t0)


def test_swap_and_relabel_invariance():
    g = synth.chung_lu_scaled(5, 40_000)
    want = oracle.count(g)
    assert oracle.count(synth.swap_sides(g)) == want
    for seed in range(3):
        assert oracle.count(synth.permute_ids(g, seed)) == want


def test_per_vertex_sums_and_relabel():
    g = synth.uniform(8, 300, 120, 4000, 0.7)
    bal, _ = oracle.count(g)
    pv = oracle.per_vertex(g)
    assert pv[: g.nU].sum() == 2 * bal
    assert pv[g.nU:].sum() == 2 * bal
    # relabelling moves the per-vertex counts with the vertices
    rng = np.random.default_rng(3)
    pu, pvv = rng.permutation(g.nU), rng.permutation(g.nV)
    u, v, s = g.edges()
    g2 = synth.from_edges(g.nU, g.nV, pu[u], pvv[v], s)
    pv2 = oracle.per_vertex(g2)
    assert np.array_equal(pv2[pu], pv[: g.nU])
    assert np.array_equal(pv2[g.nU + pvv], pv[g.nU:])
    # a listed subset gives the same values as the full vector
    ids = np.array([0, 5, g.nU + 3, g.nU + g.nV - 1])
    assert np.array_equal(oracle.per_vertex(g, ids), pv[ids])


def test_sample_count_covers_full():
    g = synth.chung_lu_scaled(13, 30_000)
    b, t = oracle.count(g, side=1)
    sb, st, steps, full = oracle.sample_count(g, np.arange(g.nV), side=1, threads=3)
    assert (sb, st) == (b, t) and steps == full
    half = np.arange(0, g.nV, 2)
    rest = np.arange(1, g.nV, 2)
    b1, t1, s1, _ = oracle.sample_count(g, half, side=1)
    b2, t2, s2, _ = oracle.sample_count(g, rest, side=1)
    assert (b1 + b2, t1 + t2, s1 + s2) == (b, t, full)


def test_thread_count_does_not_change_result():
    g = synth.chung_lu_scaled(17, 60_000)
    assert oracle.count(g, threads=1) == oracle.count(g, threads=5)


def test_iid_signs_statistics():
    # each butterfly is balanced with probability (1 + (2p-1)^4) / 2 under
    # independent signs; loose check on a graph with ~1e6 butterflies
    p = 0.7
    g = synth.uniform(31, 400, 200, 12_000, p)
    b, t = oracle.count(g)
    q = (1 + (2 * p - 1) ** 4) / 2
    assert t > 10_000
    assert abs(b - q * t) < 0.05 * t


def test_invalid_graphs_rejected():
    base = synth.from_edges(2, 2, [0, 0, 1], [0, 1, 1], [1, -1, 1])
    bad_sign = synth.SignedBipartite(2, 2, base.rowptr, base.col, np.array([1, 0, 1], np.int8))
    dup = synth.SignedBipartite(2, 2, np.array([0, 2, 3]), np.array([1, 1, 0], np.int32),
                                np.array([1, 1, 1], np.int8))
    oob = synth.SignedBipartite(2, 2, base.rowptr, np.array([0, 2, 1], np.int32), base.sign)
    for g in (bad_sign, dup, oob):
        with pytest.raises(ValueError):
            oracle.count(g)


def test_empty_and_degenerate():
    e = synth.SignedBipartite(3, 4, np.zeros(4, np.int64), np.zeros(0, np.int32),
                              np.zeros(0, np.int8))
    assert oracle.count(e) == (0, 0)
    assert list(oracle.per_vertex(e)) == [0] * 7
    star = synth.from_edges(1, 50, [0] * 50, list(range(50)), [1] * 50)
    assert oracle.count(star) == (0, 0)
    path = synth.from_edges(2, 2, [0, 0, 1], [0, 1, 1], [1, 1, 1])
    assert oracle.count(path) == (0, 0)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5])
def test_planted_mistakes_are_caught(mutant):
    """Each compile-time variant plants one plausible mistake in the oracle
    (1 drops the C(N,2) term, 2 ignores one sign, 3 admits s2 == s1,
    4 is off by one, 5 counts total as balanced); some pin must fail."""
    count = oracle_count_fn(mutant=mutant)
    failed = []
    for pin in PINS:
        try:
            pin(count)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"mutant {mutant} passed every pin"


# ---------------------------------------------------------- per-edge pins
def brute_per_edge(g):
    """Defs. 1-2 written out per edge: every balanced (u1<u2, v1<v2) adds one
    to each of its four edges. Returned in input CSR edge order."""
    u, v, s = g.edges()
    sign = {(a, b): c for a, b, c in zip(u.tolist(), v.tolist(), s.tolist())}
    pe = {k: 0 for k in sign}
    for u1, u2 in itertools.combinations(range(g.nU), 2):
        for v1, v2 in itertools.combinations(range(g.nV), 2):
            e = [(u1, v1), (u1, v2), (u2, v1), (u2, v2)]
            if all(x in sign for x in e) and sign[e[0]] * sign[e[1]] * sign[e[2]] * sign[e[3]] == 1:
                for x in e:
                    pe[x] += 1
    return np.array([pe[(a, b)] for a, b in zip(u.tolist(), v.tolist())], dtype=np.int64)


def pin_per_edge_fig1(per_edge):
    for panel, caption, signs, bal, tot in read_fig1():
        assert list(per_edge(fig1_graph(signs))) == [bal] * 4, panel


def pin_per_edge_complete(per_edge):
    for mU, nV in [(2, 3), (4, 4), (5, 7)]:
        g = synth.from_dense(np.ones((mU, nV), dtype=np.int8))
        assert set(per_edge(g).tolist()) == {(mU - 1) * (nV - 1)}, (mU, nV)


def pin_per_edge_brute(per_edge, seeds=range(30)):
    for seed in seeds:
        rng = np.random.default_rng(seed)
        nU, nV = int(rng.integers(2, 9)), int(rng.integers(2, 9))
        g = synth.uniform(3000 + seed, nU, nV, int(rng.integers(0, nU * nV + 1)), 0.55)
        assert np.array_equal(per_edge(g), brute_per_edge(g)), seed


def pin_per_edge_sum(per_edge):
    for g in (synth.uniform(7, 60, 40, 900, 0.6), synth.chung_lu_scaled(13, 20_000)):
        assert int(per_edge(g).sum()) == 4 * oracle.count(g)[0], g.name


PE_PINS = [pin_per_edge_fig1, pin_per_edge_complete, pin_per_edge_brute, pin_per_edge_sum]


def test_per_edge_pins():
    for pin in PE_PINS:
        pin(lambda g: oracle.per_edge(g, threads=2))


def test_per_edge_lemma2_and_switching():
    # K_{2,n} with l symmetric and m asymmetric middles: an edge at a middle of
    # type t lies in (count of t) - 1 balanced butterflies
    for l, m in [(0, 0), (2, 0), (3, 4), (5, 1)]:
        g = k2n(l, m, seed=l * 5 + m)
        pe = oracle.per_edge(g)
        u, v, _ = g.edges()
        pv = oracle.per_vertex(g)
        for k in range(g.nE):
            assert pe[k] == pv[g.nU + v[k]], (l, m, k)
    # negating every edge at one vertex leaves every per-edge count unchanged
    g = synth.chung_lu_scaled(21, 30_000)
    u, v, s = g.edges()
    s2 = np.where(u == 3, -s, s).astype(np.int8)
    h = synth.SignedBipartite(g.nU, g.nV, g.rowptr, g.col, s2, g.name + "/sw")
    assert np.array_equal(oracle.per_edge(g, threads=4), oracle.per_edge(h, threads=4))
    # a listed subset gives the same values as the full run
    idx = np.random.default_rng(1).choice(g.nE, 50, replace=False)
    assert np.array_equal(oracle.per_edge(g, idx), oracle.per_edge(g, threads=4)[idx])


@pytest.mark.parametrize("mutant", [6, 7])
def test_planted_per_edge_mistakes_are_caught(mutant):
    """6 admits u2 == u1 (the edge's own row as the second U vertex), 7
    ignores the fourth sign; some per-edge pin must fail."""
    failed = []
    for pin in PE_PINS:
        try:
            pin(lambda g: oracle.per_edge(g, mutant=mutant))
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"mutant {mutant} passed every per-edge pin"


def test_generator_fingerprints():
    """The generators are deterministic: their graphs match stored digests,
    so stored oracle values refer to the same inputs on every machine."""
    import hashlib
    import json
    with open(os.path.join(GOLDEN, "expected_counts.json")) as f:
        exp = json.load(f)
    for name in ["uniform_2000x1000_e20000_p0.7", "chunglu_m200000_s41"]:
        rec = exp[name]
        g = {"uniform_2000x1000_e20000_p0.7": synth.uniform_2k_1k,
             "chunglu_m200000_s41": lambda: synth.chung_lu_scaled(41, 200_000)}[name]()
        h = hashlib.sha256()
        for a in (g.rowptr, g.col, g.sign):
            h.update(np.ascontiguousarray(a).tobytes())
        assert h.hexdigest() == rec["sha256"], name
        assert oracle.count(g, threads=4) == (rec["balanced"], rec["total"])
