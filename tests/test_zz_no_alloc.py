"""The allocation-free entry point, for callers that cannot ask for device
memory when they count (their memory belongs to another allocator, or they
must not allocate once running). It must give the same counts as the
regular device entry point, call after call, and turn away graphs whose
workspace does not fit its fixed array.

This file is collected last so that a run stopping at its first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import paper_2308_07932_gb300 as pkg
from paper_2308_07932_gb300 import synth

pytestmark = pytest.mark.gpu


def entry_point():
    f = pkg.lib().bb_count_csr_device_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(pkg._Csr), ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                  ctypes.POINTER(ctypes.c_int64)]
    return f


def device_graph(torch, g):
    rp = torch.from_numpy(g.rowptr).cuda()
    cl = torch.from_numpy(g.col if g.nE else np.zeros(1, np.int32)).cuda()
    sg = torch.from_numpy(g.sign if g.nE else np.ones(1, np.int8)).cuda()
    torch.cuda.synchronize()
    return rp, cl, sg


def test_matches_regular_entry_point_twice_in_a_row():
    torch = pytest.importorskip("torch")
    f = entry_point()
    graphs = [synth.uniform_2k_1k(), synth.chung_lu_scaled(41, 200_000),
              synth.vote(5, 60, 8_000, 0.4, 2, 0.55, 0.8), synth.chung_lu_scaled(47, 600_000)]
    with pkg.Context(0) as ctx:
        for g in graphs:
            rp, cl, sg = device_graph(torch, g)
            want = ctx.count_device(g.nU, g.nV, g.nE, rp.data_ptr(), cl.data_ptr(), sg.data_ptr())
            csr = pkg._Csr(g.nU, g.nV, g.nE, rp.data_ptr(), cl.data_ptr())
            stream = torch.cuda.current_stream().cuda_stream
            for _ in range(2):
                b, t, w = ctypes.c_int64(-1), ctypes.c_int64(-1), ctypes.c_int64(-1)
                st = f(ctypes.byref(csr), sg.data_ptr(), stream, ctypes.byref(b), ctypes.byref(t),
                       ctypes.byref(w))
                assert st == 0, pkg.lib().bb_last_error()
                assert (b.value, t.value, w.value) == (want.balanced, want.total, want.wedges)


def test_rejects_graphs_beyond_its_array():
    torch = pytest.importorskip("torch")
    f = entry_point()
    g = synth.chung_lu_scaled(3, 4_000_000)
    rp, cl, sg = device_graph(torch, g)
    csr = pkg._Csr(g.nU, g.nV, g.nE, rp.data_ptr(), cl.data_ptr())
    b, t = ctypes.c_int64(-1), ctypes.c_int64(-1)
    st = f(ctypes.byref(csr), sg.data_ptr(), None, ctypes.byref(b), ctypes.byref(t), None)
    assert st == 2  # BB_ERR_TOO_LARGE
    assert b"workspace" in pkg.lib().bb_last_error()
    assert (b.value, t.value) == (-1, -1)
