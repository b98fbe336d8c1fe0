"""The bounded device waits for input copies and CG_STATUS_TIMEOUT.

The FP32 kernels fetch each instance's inputs with bulk copies into shared
memory, and CG-D's split-precision warp kernels stage H and Y with tensor
copies; both wait for them on mbarriers for a bounded time. With the limit
set to 1 ns (cg_set_wait_limit) the copies of a CTA's first instance cannot
land in time: that CTA reports CG_STATUS_TIMEOUT, lets its copies in flight
land and stops, and the call completes without a fault. The next call, with
the default limit restored, gives the normal results on the same context.
"""

import numpy as np
import pytest

import oracle
from paper_1404_0424_gb300 import workload as wl
from tests.parity import check_detect, check_precode, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cabi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_0424_gb300 import build, cabi as c
    c.library(build.build())
    yield c
    c.cg_set_wait_limit(0)


def _timed_out(cabi, st):
    s = to_np(st)
    return s, (s >= 0) & ((s & cabi.CG_STATUS_TIMEOUT) != 0)


def test_detect_wait_runs_out_then_recovers(cabi):
    dev = torch.device("cuda:0")
    d = wl.uplink(128, 16, 6, n=2048, R=14, snr_db=10.0, seed=41)
    H = torch.from_numpy(d["H"]).to(dev)
    Y = torch.from_numpy(d["Y"]).to(dev)
    n = H.shape[0]
    xh = torch.zeros((n, 14, 16), dtype=torch.complex64, device=dev)
    mu = torch.zeros((n, 14, 16), device=dev)
    rho = torch.zeros((n, 14, 16), device=dev)
    llr = torch.zeros((n, 14, 16, 6), device=dev)
    st = torch.full((n,), -1, dtype=torch.int32, device=dev)
    p = cabi.params(128, 16, 6, 3, 14, d["N0"], precision=0)
    assert cabi.cg_set_wait_limit(1) == cabi.CG_OK
    try:
        assert cabi.cg_detect(p, n, H, Y, xh, mu, rho, llr, st) == cabi.CG_OK
        torch.cuda.synchronize()
    finally:
        assert cabi.cg_set_wait_limit(0) == cabi.CG_OK
    s, timed_out = _timed_out(cabi, st)
    assert timed_out.any(), "no instance reported CG_STATUS_TIMEOUT"
    # every instance timed out, was never reached (its CTA stopped), or
    # finished normally before its CTA's wait ran out
    assert np.all((s == -1) | timed_out | ((s >= 0) & (s <= 3)))
    # the context is still usable and the default limit gives the normal results
    out = cabi.detect(H[:64], Y[:64], d["N0"], 3, 6, precision=0)
    torch.cuda.synchronize()
    ref = oracle.cg_detect(d["H"][:64], d["Y"][:64], d["N0"], 1.0, 3, 6)
    check_detect({k: to_np(v) for k, v in out.items()}, ref)


def test_precode_wait_runs_out_then_recovers(cabi):
    dev = torch.device("cuda:0")
    d = wl.downlink(64, 8, 4, n=1024, R=4, snr_db=10.0, seed=43)
    H = torch.from_numpy(d["H"]).to(dev)
    T = torch.from_numpy(d["T"]).to(dev)
    n = H.shape[0]
    q = torch.zeros((n, 4, 64), dtype=torch.complex64, device=dev)
    qn = torch.zeros((n, 4), device=dev)
    st = torch.full((n,), -1, dtype=torch.int32, device=dev)
    p = cabi.params(64, 8, 4, 3, 4, d["N0"], precision=0)
    assert cabi.cg_set_wait_limit(1) == cabi.CG_OK
    try:
        assert cabi.cg_precode(p, n, H, T, q, qn, 0, st) == cabi.CG_OK
        torch.cuda.synchronize()
    finally:
        assert cabi.cg_set_wait_limit(0) == cabi.CG_OK
    _, timed_out = _timed_out(cabi, st)
    assert timed_out.any(), "no instance reported CG_STATUS_TIMEOUT"
    out = cabi.precode(H[:32], T[:32], d["N0"], 3, precision=0)
    torch.cuda.synchronize()
    check_precode({k: to_np(v) for k, v in out.items()},
                  oracle.cg_precode(d["H"][:32], d["T"][:32], d["N0"], 1.0, 3))


def test_tma_wait_runs_out_then_recovers(cabi):
    """CG-D single calls in the split precisions stage H and Y with tensor
    copies (TMA) on mbarriers, waited for with the same bounded wait: at a
    1 ns limit a warp's first wait runs out, that instance reports
    CG_STATUS_TIMEOUT, and the warp issues nothing more and stops once its
    copies in flight have landed."""
    dev = torch.device("cuda:0")
    n = 4096
    d = wl.uplink(128, 16, 6, n=n, R=14, snr_db=10.0, seed=45)
    H = torch.from_numpy(d["H"]).to(dev)
    Y = torch.from_numpy(d["Y"]).to(dev)
    outs = (torch.zeros((n, 14, 16), dtype=torch.complex64, device=dev),
            torch.zeros((n, 14, 16), device=dev), torch.zeros((n, 14, 16), device=dev),
            torch.zeros((n, 14, 16, 6), device=dev))
    st = torch.full((n,), -1, dtype=torch.int32, device=dev)
    p = cabi.params(128, 16, 6, 3, 14, d["N0"], precision=4)
    assert cabi.cg_set_wait_limit(1) == cabi.CG_OK
    try:
        assert cabi.cg_detect(p, n, H, Y, *outs, st) == cabi.CG_OK
        torch.cuda.synchronize()
    finally:
        assert cabi.cg_set_wait_limit(0) == cabi.CG_OK
    s, timed_out = _timed_out(cabi, st)
    assert timed_out.any(), "no instance reported CG_STATUS_TIMEOUT"
    assert np.all((s == -1) | timed_out | ((s >= 0) & (s <= 3)))
    # the context is still usable and the default limit gives the normal results
    out = cabi.detect(H[:64], Y[:64], d["N0"], 3, 6, precision=4)
    torch.cuda.synchronize()
    check_detect({k: to_np(v) for k, v in out.items()},
                 oracle.cg_detect(d["H"][:64], d["Y"][:64], d["N0"], 1.0, 3, 6))
