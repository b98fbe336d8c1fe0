"""Element-by-element comparison of the CUDA path with the FP64 oracle.

Tolerances (FP32 kernels against the FP64 oracle run with the same K):
  x_hat   ||dx||_2 / ||x_ref||_2 <= 1e-4 per (instance, right-hand side)
  mu, rho |d| <= 1e-4 |ref| elementwise
  LLR     |d| <= 1e-3 max|LLR_ref| over each instance
  hard bits (LLR > 0) identical wherever |LLR_ref| exceeds that bound
  status  identical
  q       ||dq||_2 / ||q_ref||_2 <= 1e-4 per (instance, right-hand side)
"""

import numpy as np

TOL_X = 1e-4
TOL_SINR = 1e-4
TOL_LLR = 1e-3


def to_np(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


def check_detect(gpu: dict, ref: dict, tol_x=TOL_X, tol_sinr=TOL_SINR, tol_llr=TOL_LLR,
                 check_status=True):
    x = to_np(gpu["xhat"]).astype(np.complex128)
    xr = ref["x_hat"]
    nr = np.linalg.norm(xr, axis=-1)
    dx = np.linalg.norm(x - xr, axis=-1)
    zero = nr == 0
    assert np.all(dx[zero] == 0), "x_hat must be exactly zero where the oracle's is"
    if np.any(~zero):
        ex = (dx[~zero] / nr[~zero]).max()
        assert ex <= tol_x, f"x_hat relative error {ex:.3e} > {tol_x}"
    for key in ("mu", "rho"):
        g = to_np(gpu[key]).astype(np.float64)
        r = ref[key]
        bad = np.abs(g - r) > tol_sinr * np.abs(r) + 1e-30
        assert not bad.any(), (f"{key}: {bad.sum()} entries off, worst rel "
                               f"{(np.abs(g - r) / np.maximum(np.abs(r), 1e-30)).max():.3e}")
    llr = to_np(gpu["llr"]).astype(np.float64)
    lr = ref["llr"]
    axes = tuple(range(1, lr.ndim))
    bound = tol_llr * np.abs(lr).max(axis=axes, keepdims=True)
    bad = np.abs(llr - lr) > bound
    assert not bad.any(), (f"LLR: {bad.sum()} entries beyond {tol_llr}*max|LLR|, worst "
                           f"{(np.abs(llr - lr) / np.maximum(bound, 1e-30)).max():.3f} x bound")
    decided = np.abs(lr) > bound
    assert np.array_equal((llr > 0)[decided], (lr > 0)[decided]), "hard decisions differ"
    if check_status:
        st = to_np(gpu["status"])
        assert np.array_equal(st, ref["status"]), f"status {st} vs {ref['status']}"


def check_precode(gpu: dict, ref: dict, normalize=False, tol=TOL_X):
    q = to_np(gpu["q"]).astype(np.complex128)
    qr = ref["s"] if normalize else ref["q"]
    nr = np.linalg.norm(qr, axis=-1)
    dq = np.linalg.norm(q - qr, axis=-1)
    nz = nr > 0
    assert np.all(dq[~nz] == 0)
    if np.any(nz):
        e = (dq[nz] / nr[nz]).max()
        assert e <= tol, f"q relative error {e:.3e} > {tol}"
    qn = to_np(gpu["qnorm"]).astype(np.float64)
    rn = ref["qnorm"]
    assert np.all(np.abs(qn - rn) <= tol * np.abs(rn) + 1e-30), "qnorm mismatch"
    assert np.array_equal(to_np(gpu["status"]), ref["status"])
