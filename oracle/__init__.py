"""CPU oracle for balanced butterfly counting.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package. It
shares no code with the CUDA path and never imports it.

Every function here computes a quantity the paper defines:
  * ``count``       - balanced and total butterflies (Defs. 1-2), by plain
                      pair enumeration without degree priority;
  * ``per_vertex``  - balanced butterflies containing each vertex
                      (Algorithm 3, vBBFC, read with w != x);
  * ``per_edge``    - balanced butterflies containing each edge (the
                      edge-level extension, eBBFC), from the definition;
  * ``bb_base``     - the same counts by Algorithm 1 (BB-Base), an
                      independent enumeration used as a cross-check;
  * ``brute``       - Defs. 1-2 by brute force over all vertex 4-tuples.

Pins (see tests/test_oracle_*.py): Fig. 1's six butterflies, Lemma 2 on
K_{2,n}, K_{m,n} closed forms, switching / relabelling invariants, brute
force on tiny graphs, BB-Base agreement and the dense closed form.
``sample_count`` (the timed CPU baseline) is pinned through ``count``:
with every start listed it returns the same sums.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bb_oracle.c")
_libs: dict[int, ctypes.CDLL] = {}

I64P = ctypes.POINTER(ctypes.c_int64)
I32P = ctypes.POINTER(ctypes.c_int32)
I8P = ctypes.POINTER(ctypes.c_int8)

_ERR = {-1: "invalid graph", -2: "out of memory", -3: "count exceeds int64"}


def lib_path(mutant: int = 0) -> str:
    name = "libbboracle.so" if mutant == 0 else f"libbboracle_m{mutant}.so"
    if mutant == 0:
        return os.path.join(_HERE, name)
    return os.path.join(_HERE, "_build", name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, pthreads). ``mutant`` > 0 builds a
    planted-mistake variant used only by the pin-strength tests."""
    out = lib_path(mutant)
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               f"-DORACLE_MUTANT={mutant}", "-o", tmp, _SRC])
        os.replace(tmp, out)
    return out


def _lib(mutant: int = 0) -> ctypes.CDLL:
    if mutant not in _libs:
        L = ctypes.CDLL(build(mutant))
        L.oracle_count.argtypes = [ctypes.c_int64, ctypes.c_int64, I64P, I32P, I8P,
                                   ctypes.c_int, ctypes.c_int, I64P, I64P]
        L.oracle_count_sample.argtypes = [ctypes.c_int64, ctypes.c_int64, I64P, I32P, I8P,
                                          ctypes.c_int, I64P, ctypes.c_int64, ctypes.c_int,
                                          I64P, I64P, I64P, I64P]
        L.oracle_per_vertex.argtypes = [ctypes.c_int64, ctypes.c_int64, I64P, I32P, I8P,
                                        I64P, ctypes.c_int64, ctypes.c_int, I64P]
        L.oracle_per_edge.argtypes = [ctypes.c_int64, ctypes.c_int64, I64P, I32P, I8P,
                                      I64P, ctypes.c_int64, ctypes.c_int, I64P]
        L.oracle_bb_base.argtypes = [ctypes.c_int64, ctypes.c_int64, I64P, I32P, I8P, I64P, I64P]
        L.oracle_brute.argtypes = [ctypes.c_int64, ctypes.c_int64, I64P, I32P, I8P, I64P, I64P,
                                   I64P]
        for f in (L.oracle_count, L.oracle_count_sample, L.oracle_per_vertex, L.oracle_per_edge,
                  L.oracle_bb_base, L.oracle_brute):
            f.restype = ctypes.c_int
        _libs[mutant] = L
    return _libs[mutant]


def _arrays(g):
    rowptr = np.ascontiguousarray(g.rowptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    sign = np.ascontiguousarray(g.sign, dtype=np.int8)
    if col.size == 0:  # ctypes wants a real buffer
        col = np.zeros(1, np.int32)
        sign = np.ones(1, np.int8)
    return rowptr, col, sign, (rowptr.ctypes.data_as(I64P), col.ctypes.data_as(I32P),
                               sign.ctypes.data_as(I8P))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what}: {_ERR.get(rc, rc)}")


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def count(g, side: int = -1, threads: int = 1, mutant: int = 0) -> tuple[int, int]:
    """(balanced, total) butterflies of graph ``g`` (Defs. 1-2).

    side: 0 puts the endpoint pairs on U, 1 on V, -1 picks the cheaper side.
    """
    _, _, _, (rp, c, s) = keep = _arrays(g)
    b, t = ctypes.c_int64(), ctypes.c_int64()
    rc = _lib(mutant).oracle_count(g.nU, g.nV, rp, c, s, side, threads, ctypes.byref(b),
                                   ctypes.byref(t))
    del keep
    _check(rc, "count")
    return int(b.value), int(t.value)


def sample_count(g, starts, side: int, threads: int = 1):
    """Contribution of the endpoint pairs {s1, s2 > s1} for the listed s1 on
    ``side``; returns (balanced, total, steps walked, steps of the full count)."""
    _, _, _, (rp, c, s) = keep = _arrays(g)
    st = np.ascontiguousarray(starts, dtype=np.int64)
    out = [ctypes.c_int64() for _ in range(4)]
    rc = _lib().oracle_count_sample(g.nU, g.nV, rp, c, s, side, st.ctypes.data_as(I64P),
                                    st.size, threads, *[ctypes.byref(o) for o in out])
    del keep
    _check(rc, "sample_count")
    return tuple(int(o.value) for o in out)


def per_vertex(g, gids=None, threads: int = 1) -> np.ndarray:
    """Balanced butterflies containing each vertex (Algorithm 3, w != x).

    gids: None for every vertex (U ids 0..nU-1 then V ids nU..nU+nV-1), or a
    list of such ids. Returns int64 counts in the same order.
    """
    _, _, _, (rp, c, s) = keep = _arrays(g)
    if gids is None:
        n = g.nU + g.nV
        out = np.zeros(n, np.int64)
        rc = _lib().oracle_per_vertex(g.nU, g.nV, rp, c, s, None, 0, threads,
                                      out.ctypes.data_as(I64P))
    else:
        ids = np.ascontiguousarray(gids, dtype=np.int64)
        out = np.zeros(ids.size, np.int64)
        rc = _lib().oracle_per_vertex(g.nU, g.nV, rp, c, s, ids.ctypes.data_as(I64P), ids.size,
                                      threads, out.ctypes.data_as(I64P))
    del keep
    _check(rc, "per_vertex")
    return out


def per_edge(g, edges=None, threads: int = 1, mutant: int = 0) -> np.ndarray:
    """Balanced butterflies containing each edge (the paper's edge-level
    extension, eBBFC), from the definition: every butterfly through the edge
    enumerated by its other two vertices and tested with Def. 2.

    edges: None for every edge in input CSR order, or a list of positions in
    the input CSR. Returns int64 counts in the same order.
    """
    _, _, _, (rp, c, s) = keep = _arrays(g)
    if edges is None:
        out = np.zeros(g.nE, np.int64)
        rc = _lib(mutant).oracle_per_edge(g.nU, g.nV, rp, c, s, None, 0, threads,
                                          out.ctypes.data_as(I64P))
    else:
        ids = np.ascontiguousarray(edges, dtype=np.int64)
        out = np.zeros(ids.size, np.int64)
        rc = _lib(mutant).oracle_per_edge(g.nU, g.nV, rp, c, s, ids.ctypes.data_as(I64P),
                                          ids.size, threads, out.ctypes.data_as(I64P))
    del keep
    _check(rc, "per_edge")
    return out


def bb_base(g) -> tuple[int, int]:
    """(balanced, total) by Algorithm 1 (BB-Base): priority wedges grouped in
    H(w), every pair tested for balance explicitly."""
    _, _, _, (rp, c, s) = keep = _arrays(g)
    b, t = ctypes.c_int64(), ctypes.c_int64()
    rc = _lib().oracle_bb_base(g.nU, g.nV, rp, c, s, ctypes.byref(b), ctypes.byref(t))
    del keep
    _check(rc, "bb_base")
    return int(b.value), int(t.value)


def brute(g, with_per_vertex: bool = False):
    """Defs. 1-2 over all vertex 4-tuples (|U|, |V| <= 4096; use tiny graphs)."""
    _, _, _, (rp, c, s) = keep = _arrays(g)
    b, t = ctypes.c_int64(), ctypes.c_int64()
    pv = np.zeros(g.nU + g.nV, np.int64) if with_per_vertex else None
    rc = _lib().oracle_brute(g.nU, g.nV, rp, c, s, ctypes.byref(b), ctypes.byref(t),
                             pv.ctypes.data_as(I64P) if pv is not None else None)
    del keep
    _check(rc, "brute")
    return (int(b.value), int(t.value), pv) if with_per_vertex else (int(b.value), int(t.value))
