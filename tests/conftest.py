import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")
    config.addinivalue_line("markers",
                            "product: runs with the matrix-product path allowed (off otherwise)")


@pytest.fixture(autouse=True)
def _wedge_kernels_unless_product(request):
    """GPU tests exercise the wedge kernels: the matrix-product path, which
    counts qualifying dense graphs without them, is switched off around each
    GPU test not marked `product`."""
    if request.node.get_closest_marker("gpu") is None or request.node.get_closest_marker("product"):
        yield
        return
    import paper_2308_07932_gb300 as pkg
    prev = pkg.set_matrix_product(False)
    try:
        yield
    finally:
        pkg.set_matrix_product(prev)
