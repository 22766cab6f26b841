"""Failure handling without faulting the GPU: a blocking call whose device
work outlasts the wait limit returns BB_ERR_TIMEOUT (the limit is made
tiny; the work itself is ordinary and finishes), the context and the
serving engine stay usable afterwards, and results are right again once
the limit is restored."""
import pytest

import oracle
import paper_2308_07932_gb300 as pkg
from paper_2308_07932_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    g = synth.chung_lu_scaled(43, 2_000_000)
    return g, oracle.count(g, threads=8)


def restore():
    import torch
    pkg.set_wait_timeout(600.0)
    torch.cuda.synchronize()   # the timed-out work drains on its own


def test_blocking_count_times_out_then_recovers(big):
    g, want = big
    with pkg.Context(0) as ctx:
        try:
            pkg.set_wait_timeout(1e-4)
            with pytest.raises(pkg.BBError) as ei:
                ctx.count(g)
            assert ei.value.name == "BB_ERR_TIMEOUT"
        finally:
            restore()
        c = ctx.count(g)
        assert (c.balanced, c.total) == want


def test_served_request_times_out_then_recovers(big):
    g, want = big
    with pkg.Context(0) as ctx:
        ctx.serve(slots=2, arena_bytes=2 << 30)
        try:
            pkg.set_wait_timeout(1e-4)
            with pytest.raises(pkg.BBError) as ei:
                ctx.submit_request(7, g).wait()
            assert ei.value.name == "BB_ERR_TIMEOUT"
        finally:
            restore()
        # the timed-out graph was dropped; a new upload of the key counts right
        o = ctx.submit_request(7, g).wait()
        assert (o.balanced, o.total) == want
        st = ctx.serve_stats()
        assert st["failed"] == 1 and st["completed"] == 1
