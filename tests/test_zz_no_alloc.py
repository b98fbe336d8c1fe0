"""cg_batch_run_static: batched problems for callers that may not allocate.

A slot-deadline receiver loop, or code confined to a device-memory budget
owned by another allocator, cannot call cudaMalloc; this entry point runs
the batched kernels with their work tables in a static device array. The
test checks its results against the existing single-shape entry points
(cg_detect / cg_precode), within the parity tolerances, on two calls in a
row. The file sorts last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

from paper_1404_0424_gb300 import workload as wl
from tests.parity import TOL_LLR, TOL_SINR, TOL_X

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cabi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_0424_gb300 import build, cabi as c
    c.library(build.build())
    return c


def _close(a, b, tol, axis=-1):
    a = a.detach().cpu().numpy().astype(np.complex128)
    b = b.detach().cpu().numpy().astype(np.complex128)
    nb = np.linalg.norm(b, axis=axis)
    d = np.linalg.norm(a - b, axis=axis)
    return bool(np.all(d <= tol * nb + 1e-30))


def _problems(dev, seed=17):
    """Detection and precoding problems of several shapes; every third
    detection problem uses the exact tracker (Eq. 10), so exact and
    approximate problems share padded user counts 8, 16 and 32."""
    rng = np.random.default_rng(seed)
    shapes = [(64, 8), (128, 16), (128, 32), (33, 5), (100, 12), (96, 32)]
    probs = []
    for k in range(36):
        B, U = shapes[k % len(shapes)]
        R = int(rng.integers(1, 15))
        q = int(rng.choice([4, 6, 8]))
        K = max(1, min(U // 4, 8))
        n = int(rng.integers(1, 4))
        op = k % 2
        exact = int(op == 0 and k % 3 == 0)
        if op == 0:
            d = wl.uplink(B, U, q, n=n, R=R, snr_db=12.0, seed=seed * 100 + k)
            inp = torch.from_numpy(d["Y"]).to(dev)
        else:
            d = wl.downlink(B, U, q, n=n, R=R, snr_db=12.0, seed=seed * 100 + k)
            inp = torch.from_numpy(d["T"]).to(dev)
        probs.append(dict(op=op, B=B, U=U, R=R, q=q, K=K, n=n, N0=d["N0"], exact=exact,
                          H=torch.from_numpy(d["H"]).to(dev), inp=inp))
    return probs


def _outputs(p, dev):
    n, R, U, B, q = p["n"], p["R"], p["U"], p["B"], p["q"]
    if p["op"] == 0:
        return {"xhat": torch.full((n, R, U), np.nan, dtype=torch.complex64, device=dev),
                "mu": torch.full((n, R, U), np.nan, device=dev),
                "rho": torch.full((n, R, U), np.nan, device=dev),
                "llr": torch.full((n, R, U, q), np.nan, device=dev),
                "status": torch.full((n,), -1, dtype=torch.int32, device=dev)}
    return {"q": torch.full((n, R, B), np.nan, dtype=torch.complex64, device=dev),
            "qnorm": torch.full((n, R), np.nan, device=dev),
            "status": torch.full((n,), -1, dtype=torch.int32, device=dev)}


def _descs(cabi, probs, outs):
    descs = []
    for p, o in zip(probs, outs):
        if p["op"] == 0:
            descs.append(cabi.desc(0, p["B"], p["U"], p["R"], p["K"], p["N0"], p["H"],
                                   p["inp"], o["xhat"], qam_bits=p["q"], sinr_mode=p["exact"],
                                   mu=o["mu"], rho=o["rho"], aux=o["llr"], status=o["status"]))
        else:
            descs.append(cabi.desc(1, p["B"], p["U"], p["R"], p["K"], p["N0"], p["H"],
                                   p["inp"], o["q"], aux=o["qnorm"], status=o["status"]))
    return descs


@pytest.mark.parametrize("precision", [4, 3, 2])
def test_static_batch_matches_single_calls_twice(cabi, precision):
    """Calls in a row against cg_detect / cg_precode of the same precision
    (FP16X3, BF16X3 and one-pass FP16), with exact-tracker and approximate
    problems mixed. The first call may load the batch kernels' device code
    (CUDA loads modules lazily, which takes device memory); the two calls
    after it must leave the device's free memory exactly as it was."""
    dev = torch.device("cuda:0")
    probs = _problems(dev)
    refs = []
    for p in probs:
        if p["op"] == 0:
            refs.append(cabi.detect(p["H"], p["inp"], p["N0"], p["K"], p["q"],
                                    sinr_mode=p["exact"], precision=precision))
        else:
            refs.append(cabi.precode(p["H"], p["inp"], p["N0"], p["K"], precision=precision))
    outs = [[_outputs(p, dev) for p in probs] for _ in range(3)]
    descs = [_descs(cabi, probs, o) for o in outs]
    torch.cuda.synchronize()
    free_before = None
    for call in range(3):
        rc = cabi.cg_batch_run_static(descs[call], precision)
        assert rc == 0, cabi.cg_strerror(rc)
        torch.cuda.synchronize()
        if call == 0:
            free_before = torch.cuda.mem_get_info(dev)[0]
        else:
            assert torch.cuda.mem_get_info(dev)[0] == free_before, "device memory was allocated"
        for p, o, r in zip(probs, outs[call], refs):
            assert torch.equal(o["status"], r["status"])
            if p["op"] == 0:
                assert _close(o["xhat"], r["xhat"], TOL_X), f"call {call}: x_hat"
                for k in ("mu", "rho"):
                    a, b = o[k].cpu().numpy(), r[k].cpu().numpy()
                    assert np.all(np.abs(a - b) <= TOL_SINR * np.abs(b)), f"call {call}: {k}"
                a, b = o["llr"].cpu().numpy(), r["llr"].cpu().numpy()
                bound = TOL_LLR * np.abs(b).max(axis=(1, 2, 3), keepdims=True)
                assert np.all(np.abs(a - b) <= bound), f"call {call}: llr"
            else:
                assert _close(o["q"], r["q"], TOL_X), f"call {call}: q"
                a, b = o["qnorm"].cpu().numpy(), r["qnorm"].cpu().numpy()
                assert np.all(np.abs(a - b) <= TOL_X * np.abs(b)), f"call {call}: qnorm"


def test_static_batch_skips_empty_problems(cabi):
    """A descriptor with no instances is validated and sizes no bin."""
    dev = torch.device("cuda:0")
    probs = _problems(dev)[:4]
    outs = [_outputs(p, dev) for p in probs]
    descs = _descs(cabi, probs, outs)
    H = torch.zeros((1, 256, 32), dtype=torch.complex64, device=dev)
    Y = torch.zeros((1, 16, 256), dtype=torch.complex64, device=dev)
    x = torch.zeros((1, 16, 32), dtype=torch.complex64, device=dev)
    descs.append(cabi.desc(0, 256, 32, 16, 32, 1.0, H, Y, x, qam_bits=8, sinr_mode=1, n_inst=0))
    assert cabi.cg_batch_run_static(descs, 4) == 0
    torch.cuda.synchronize()
    for p, o in zip(probs, outs):
        key = "xhat" if p["op"] == 0 else "q"
        assert torch.isfinite(torch.view_as_real(o[key])).all()


def test_static_batch_rejects_oversized_requests(cabi):
    dev = torch.device("cuda:0")
    H = torch.zeros((1, 8, 4), dtype=torch.complex64, device=dev)
    Y = torch.zeros((1, 1, 8), dtype=torch.complex64, device=dev)
    x = torch.zeros((1, 1, 4), dtype=torch.complex64, device=dev)
    one = cabi.desc(0, 8, 4, 1, 1, 1.0, H, Y, x, qam_bits=2)
    too_many = [one] * (cabi.CG_STATIC_MAX_PROBLEMS + 1)
    assert cabi.cg_batch_run_static(too_many, 4) == cabi.CG_ETOOBIG
    big = cabi.desc(0, 8, 4, 1, 1, 1.0, H, Y, x, qam_bits=2,
                    n_inst=cabi.CG_STATIC_MAX_INSTANCES + 1)
    assert cabi.cg_batch_run_static([big], 4) == cabi.CG_ETOOBIG
