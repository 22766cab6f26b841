"""Host-only checks of the C ABI: the library loads, exports every function
include/bb.h declares, and rejects bad arguments before touching a device."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2308_07932_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bb.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bb_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    from paper_2308_07932_gb300 import _build
    _build.build()
    return pkg.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["bb_ctx_create", "bb_graph_upload", "bb_count", "bb_count_csr",
                 "bb_count_csr_device", "bb_graph_flip_signs", "bb_last_error"]:
        assert want in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(bb_\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(built, n)


def test_version_and_null_arguments(built):
    assert "sm_103a" in pkg.version()
    b, t = ctypes.c_int64(), ctypes.c_int64()
    st = built.bb_count_csr(None, None, None, ctypes.byref(b), ctypes.byref(t), None, None)
    assert st == 1  # BB_ERR_INVALID_ARG
    assert b"NULL" in built.bb_last_error()
    st = built.bb_ctx_create(0, 0, None)
    assert st == 1


def test_context_without_device_fails_loudly(built):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present; covered by the gpu tests")
    with pytest.raises(pkg.BBError) as ei:
        pkg.Context(0)
    assert ei.value.name in ("BB_ERR_NO_DEVICE", "BB_ERR_CUDA")


def test_sizes_and_serving_arguments_without_device(built):
    r, w = pkg.graph_bytes(2_000_000, 500_000, 20_000_000)
    r2, w2 = pkg.graph_bytes(200_000, 50_000, 2_000_000)
    assert r > r2 > 0 and w > w2 > 0
    with pytest.raises(pkg.BBError):
        pkg.graph_bytes(-1, 2, 3)
    t = ctypes.c_void_p()
    assert built.bb_submit(None, None, 0, ctypes.byref(t)) == 1
    assert built.bb_submit_request(None, None, 0, ctypes.byref(t)) == 1
    done = ctypes.c_int()
    b = ctypes.c_int64()
    assert built.bb_poll(None, ctypes.byref(done), ctypes.byref(b), ctypes.byref(b)) == 1
    assert built.bb_batch_create(None, None, 0, ctypes.byref(t)) == 1


def test_wait_timeout_argument_checks(built):
    with pytest.raises(pkg.BBError):
        pkg.set_wait_timeout(0.0)
    with pytest.raises(pkg.BBError):
        pkg.set_wait_timeout(-1.0)
    pkg.set_wait_timeout(600.0)


def test_matrix_product_plan(built):
    """The size rule of the matrix-product path (host only)."""
    plan = pkg.matrix_product_plan
    assert plan(500, 50_000, 10_000_000)          # vote-like: small dense side
    assert plan(50_000, 500, 10_000_000)          # the same with the sides swapped
    assert not plan(2_000_000, 500_000, 20_000_000)  # power-law: both sides large
    assert not plan(2_000, 1_000, 20_000)         # too few edges
    assert plan(2, 40_000, 65_536)                # K_{2,n}-like: dense
    assert not plan(1, 100_000, 100_000)          # no pairs on the smaller side
    assert not plan(8_193, 8_193, 20_000_000)     # pair side above 8192
    assert not plan(100, (1 << 21), 50_000_000)   # middles at the exactness bound
    assert not plan(200, 1_000_000, 12_000_000)   # density 1/16.7, below 1/16
    assert plan(200, 1_000_000, 13_000_000)       # density 1/15.4
    assert not plan(300, 1_000_000, 30_000_000)   # 3e8 matrix cells, above 2^28
    with pytest.raises(pkg.BBError):
        plan(-1, 2, 3)
    prev = pkg.set_matrix_product(False)
    try:
        assert not plan(500, 50_000, 10_000_000)
    finally:
        pkg.set_matrix_product(prev)
    assert plan(500, 50_000, 10_000_000)
    # the product buffers are part of a qualifying graph's resident bytes
    r_prod, _ = pkg.graph_bytes(500, 50_000, 2_000_000)
    r_wedge, _ = pkg.graph_bytes(5_000, 50_000, 2_000_000)
    assert r_prod > 500 * 50_000 * 4  # X and |X| in bf16
    assert r_wedge < r_prod
