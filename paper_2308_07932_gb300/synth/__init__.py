"""Seeded synthetic signed bipartite graphs (inputs only).

This module makes graphs; it holds none of the counting arithmetic. The CPU
oracle tests and the CUDA path both read graphs made here, so a graph is fully
determined by its recipe and seed on every machine (the C generator avoids
libm transcendental functions and FMA contraction; see ``bbsynth.c``).

The named workloads stand in for the paper's datasets (Section "Datasets",
Table 1), which are not available: uniform (small real signed sets), Chung-Lu
power-law (rating-like graphs), and vote-like (senate/house-like dense
graphs with correlated signs).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bbsynth.c")
_LIB = os.path.join(_HERE, "libbbsynth.so")
_lib = None


class _Graph(ctypes.Structure):
    _fields_ = [
        ("nU", ctypes.c_int64),
        ("nV", ctypes.c_int64),
        ("nE", ctypes.c_int64),
        ("rowptr", ctypes.POINTER(ctypes.c_int64)),
        ("col", ctypes.POINTER(ctypes.c_int32)),
        ("sign", ctypes.POINTER(ctypes.c_int8)),
    ]


def build(force: bool = False) -> str:
    """Compile the generator library in place (gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        G = ctypes.POINTER(_Graph)
        lib.synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_int64, ctypes.c_double, G]
        lib.synth_chung_lu.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, G]
        lib.synth_vote.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_double, ctypes.c_int64, ctypes.c_double,
                                   ctypes.c_double, G]
        for f in (lib.synth_uniform, lib.synth_chung_lu, lib.synth_vote):
            f.restype = ctypes.c_int
        lib.synth_free.argtypes = [G]
        lib.synth_free.restype = None
        lib.synth_log_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                          ctypes.c_double]
        lib.synth_log_uniform.restype = ctypes.c_double
        lib.synth_uniform_real.argtypes = lib.synth_log_uniform.argtypes
        lib.synth_uniform_real.restype = ctypes.c_double
        lib.synth_uniform_ints.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                           ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        lib.synth_uniform_ints.restype = None
        lib.synth_exponential.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                          ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
        lib.synth_exponential.restype = None
        _lib = lib
    return _lib


@dataclass
class SignedBipartite:
    """U-side CSR of a signed bipartite graph.

    rowptr: int64[nU+1]; col: int32[nE] (V ids, strictly increasing per row);
    sign: int8[nE] in {+1, -1}.
    """

    nU: int
    nV: int
    rowptr: np.ndarray
    col: np.ndarray
    sign: np.ndarray
    name: str = ""

    @property
    def nE(self) -> int:
        return int(self.col.shape[0])

    def edges(self):
        """(u, v, sign) arrays of all edges in CSR order."""
        u = np.repeat(np.arange(self.nU, dtype=np.int64), np.diff(self.rowptr))
        return u, self.col.astype(np.int64), self.sign.astype(np.int64)


def _take(g: _Graph, rc: int, name: str) -> SignedBipartite:
    lib = _load()
    if rc != 0:
        lib.synth_free(ctypes.byref(g))
        raise ValueError(f"generator {name} failed with code {rc}")
    nU, nV, nE = g.nU, g.nV, g.nE
    rowptr = np.ctypeslib.as_array(g.rowptr, shape=(nU + 1,)).copy()
    col = np.ctypeslib.as_array(g.col, shape=(max(nE, 1),))[:nE].copy()
    sign = np.ctypeslib.as_array(g.sign, shape=(max(nE, 1),))[:nE].copy()
    lib.synth_free(ctypes.byref(g))
    return SignedBipartite(int(nU), int(nV), rowptr, col, sign, name)


def uniform(seed: int, nU: int, nV: int, m: int, p_pos: float) -> SignedBipartite:
    """m distinct edges drawn uniformly without replacement; sign +1 w.p. p_pos."""
    g = _Graph()
    rc = _load().synth_uniform(seed, nU, nV, m, p_pos, ctypes.byref(g))
    return _take(g, rc, f"uniform(seed={seed},{nU}x{nV},m={m},p={p_pos})")


def chung_lu(seed: int, nU: int, nV: int, m_draw: int, alpha_u: float, alpha_v: float,
             cap_deg: float, p_pos: float) -> SignedBipartite:
    """Chung-Lu power-law graph: m_draw pairs drawn by expected degree, deduplicated."""
    g = _Graph()
    rc = _load().synth_chung_lu(seed, nU, nV, m_draw, alpha_u, alpha_v, cap_deg, p_pos,
                                ctypes.byref(g))
    return _take(g, rc, f"chung_lu(seed={seed},{nU}x{nV},draw={m_draw},a={alpha_u}/{alpha_v},p={p_pos})")


def vote(seed: int, nU: int, nV: int, p_edge: float, n_blocks: int, p_stance: float,
         agree: float) -> SignedBipartite:
    """Dense vote-like graph with per-(v, U-block) stances."""
    g = _Graph()
    rc = _load().synth_vote(seed, nU, nV, p_edge, n_blocks, p_stance, agree, ctypes.byref(g))
    return _take(g, rc, f"vote(seed={seed},{nU}x{nV},p={p_edge},blocks={n_blocks})")


def log_uniform(seed: int, stream: int, lo: float, hi: float) -> float:
    return float(_load().synth_log_uniform(seed, stream, lo, hi))


def uniform_real(seed: int, stream: int, lo: float, hi: float) -> float:
    return float(_load().synth_uniform_real(seed, stream, lo, hi))


def uniform_ints(seed: int, stream: int, n: int, bound: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int64)
    _load().synth_uniform_ints(seed, stream, n, bound,
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return out


def exponential_gaps(seed: int, stream: int, n: int, rate: float) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().synth_exponential(seed, stream, n, rate,
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


# ------------------------------------------------------------------ workloads
# Uniform small signed graph (stands in for Bonanza/Senate-scale real sets).
def uniform_2k_1k(seed: int = 1) -> SignedBipartite:
    g = uniform(seed, 2000, 1000, 20000, 0.7)
    g.name = "uniform_2000x1000_e20000_p0.7"
    return g


# Chung-Lu rating-like graph: |U|=2M, |V|=500k, ~20M distinct edges after
# dedup of 21.6M draws, Pareto(2.1) expected degrees capped at 50,000, p(+)=0.8.
CHUNG_LU_2M_DRAW = 21_600_000


def chung_lu_2m(seed: int = 2) -> SignedBipartite:
    g = chung_lu(seed, 2_000_000, 500_000, CHUNG_LU_2M_DRAW, 2.1, 2.1, 50_000.0, 0.8)
    g.name = "chunglu_2Mx500k_e20M_a2.1_p0.8"
    return g


# Vote-like dense graph: |U|=500, |V|=50,000, edge prob 0.4 (~10M edges),
# 2 U-blocks, stance +1 w.p. 0.55, in-block agreement 0.8.
def vote_500_50k(seed: int = 3) -> SignedBipartite:
    g = vote(seed, 500, 50_000, 0.4, 2, 0.55, 0.8)
    g.name = "vote_500x50000_p0.4_b2"
    return g


def chung_lu_scaled(seed: int, m: int, ratio_uv: float = 4.0, alpha: float = 2.1,
                    p_pos: float = 0.8, cap: float = 50_000.0) -> SignedBipartite:
    """Chung-Lu graph with the 2M-x-500k graph's shape at another size:
    |U| = m/10, |V| = |U|/ratio_uv, m*1.08 draws."""
    nU = max(2, int(round(m / 10)))
    nV = max(2, int(round(nU / ratio_uv)))
    return chung_lu(seed, nU, nV, int(round(m * 1.08)), alpha, alpha, cap, p_pos)


# Batched mix: graph i has seed base+i; |E| log-uniform in [1e3, 2e6];
# |U|:|V| log-uniform in [1, 10]; exponent uniform in [2.1, 2.8];
# p(+) uniform in [0.5, 0.9]; |U|+|V| = |E|/8; expected degrees capped at
# min(50,000, other side size).
@dataclass
class MixParams:
    seed: int
    m: int
    nU: int
    nV: int
    alpha: float
    p_pos: float


def batch_params(i: int, base_seed: int = 4, m_lo: float = 1e3, m_hi: float = 2e6) -> MixParams:
    s = base_seed + i
    m = int(round(log_uniform(s, 101, m_lo, m_hi)))
    r = log_uniform(s, 102, 1.0, 10.0)
    alpha = uniform_real(s, 103, 2.1, 2.8)
    p = uniform_real(s, 104, 0.5, 0.9)
    n = max(4, m // 8)
    nU = max(2, int(round(n * r / (1.0 + r))))
    nV = max(2, n - nU)
    return MixParams(s, m, nU, nV, alpha, p)


def batch_graph(i: int, base_seed: int = 4, m_lo: float = 1e3, m_hi: float = 2e6) -> SignedBipartite:
    q = batch_params(i, base_seed, m_lo, m_hi)
    g = chung_lu(q.seed, q.nU, q.nV, q.m, q.alpha, q.alpha, 50_000.0, q.p_pos)
    g.name = f"mix[{i}]"
    return g


def batch_graphs(count: int, base_seed: int = 4, m_lo: float = 1e3, m_hi: float = 2e6,
                 threads: int | None = None) -> list[SignedBipartite]:
    """Generate graphs 0..count-1 of the batched mix in parallel host threads."""
    threads = threads or min(32, os.cpu_count() or 4)
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda i: batch_graph(i, base_seed, m_lo, m_hi), range(count)))


# Serving pool: |E| log-uniform in [1e4, 5e7], drawn as the 2M-x-500k graph
# (exponent 2.1, p(+)=0.8, |U| = |E|/10, |V| = |U|/4).
def serving_params(i: int, base_seed: int = 5, m_lo: float = 1e4, m_hi: float = 5e7) -> int:
    return int(round(log_uniform(base_seed * 1_000_003 + i, 201, m_lo, m_hi)))


def serving_graph(i: int, base_seed: int = 5, m_lo: float = 1e4, m_hi: float = 5e7) -> SignedBipartite:
    m = serving_params(i, base_seed, m_lo, m_hi)
    g = chung_lu_scaled(base_seed * 1_000_003 + i, m)
    g.name = f"serve[{i}]"
    return g


def permute_ids(g: SignedBipartite, seed: int) -> SignedBipartite:
    """Relabel U and V ids by seeded random permutations (same graph up to
    isomorphism). Uses numpy's PCG64 for the permutation; no counting."""
    rng = np.random.default_rng(seed)
    pu = rng.permutation(g.nU)
    pv = rng.permutation(g.nV)
    u, v, s = g.edges()
    return from_edges(g.nU, g.nV, pu[u], pv[v], s, g.name + f"/perm{seed}")


def swap_sides(g: SignedBipartite) -> SignedBipartite:
    """The same graph with U and V exchanged."""
    u, v, s = g.edges()
    return from_edges(g.nV, g.nU, v, u, s, g.name + "/swap")


def from_edges(nU: int, nV: int, u, v, s, name: str = "") -> SignedBipartite:
    """Build the U-side CSR (rows sorted by v) from edge arrays."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    s = np.asarray(s, dtype=np.int8)
    order = np.lexsort((v, u))
    u, v, s = u[order], v[order], s[order]
    rowptr = np.zeros(nU + 1, dtype=np.int64)
    np.add.at(rowptr, u + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int64)
    return SignedBipartite(nU, nV, rowptr, v.astype(np.int32), s.astype(np.int8), name)


def from_dense(A) -> SignedBipartite:
    """Graph from a dense nU x nV matrix with entries in {-1, 0, +1}."""
    A = np.asarray(A)
    u, v = np.nonzero(A)
    return from_edges(A.shape[0], A.shape[1], u, v, A[u, v])


def to_dense(g: SignedBipartite) -> np.ndarray:
    A = np.zeros((g.nU, g.nV), dtype=np.int8)
    u, v, s = g.edges()
    A[u, v] = s
    return A
