"""Thin ctypes binding of libcgmimo (include/cgmimo.h).

The functions cg_detect, cg_precode, cg_detect_host, cg_precode_host,
cg_neumann_detect, cg_neumann_precode, cg_release_workspace, cg_strerror and
cg_version have the names and argument order of the C ABI. detect(),
precode(), neumann_detect() and neumann_precode() are conveniences that allocate the
outputs as torch tensors and marshal pointers; every step of the computation
runs in the CUDA library. There is no fallback: if the library is missing
the first call raises.
"""

from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
HEADER = os.path.join(_ROOT, "include", "cgmimo.h")
LIB_PATH = os.path.join(_PKG, "_build", "libcgmimo.so")


def _header_constants(path: str = HEADER) -> dict:
    consts = {}
    with open(path) as f:
        for m in re.finditer(r"^#define\s+(CG_\w+)\s+\(?(-?\d+)\)?", f.read(), re.M):
            consts[m.group(1)] = int(m.group(2))
    return consts


C = _header_constants()
globals().update(C)


class CgParams(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int32), ("U", ctypes.c_int32), ("qam_bits", ctypes.c_int32),
                ("K", ctypes.c_int32), ("R", ctypes.c_int32), ("N0", ctypes.c_float),
                ("Es", ctypes.c_float), ("sinr_mode", ctypes.c_int32),
                ("amul_mode", ctypes.c_int32), ("precision", ctypes.c_int32)]


class CgDesc(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("B", ctypes.c_int32), ("U", ctypes.c_int32),
                ("R", ctypes.c_int32), ("K", ctypes.c_int32), ("qam_bits", ctypes.c_int32),
                ("sinr_mode", ctypes.c_int32), ("normalize", ctypes.c_int32),
                ("N0", ctypes.c_float), ("Es", ctypes.c_float), ("n_inst", ctypes.c_int64),
                ("H", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("mu", ctypes.c_void_p), ("rho", ctypes.c_void_p), ("aux", ctypes.c_void_p),
                ("status", ctypes.c_void_p)]


class CgServeCfg(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("max_B", ctypes.c_int32),
                ("max_R", ctypes.c_int32), ("ctas_per_class", ctypes.c_int32),
                ("idle_timeout_ms", ctypes.c_int32)]


class CgReqStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("submit_ns", ctypes.c_int64), ("complete_ns", ctypes.c_int64),
                ("device_first_ns", ctypes.c_int64), ("device_done_ns", ctypes.c_int64)]


class CgError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {cg_strerror(code)} ({code})")
        self.code = code


_lib = None
_VP = ctypes.c_void_p
_FP = ctypes.POINTER(ctypes.c_float)
_IP = ctypes.POINTER(ctypes.c_int32)

_SIGS = {
    "cg_detect": [ctypes.POINTER(CgParams), ctypes.c_int64, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                  _VP],
    "cg_precode": [ctypes.POINTER(CgParams), ctypes.c_int64, _VP, _VP, _VP, _VP, ctypes.c_int32,
                   _VP, _VP],
    "cg_detect_host": [ctypes.POINTER(CgParams), ctypes.c_int64, _VP, _VP, _VP, _VP, _VP, _VP,
                       _VP, _VP],
    "cg_precode_host": [ctypes.POINTER(CgParams), ctypes.c_int64, _VP, _VP, _VP, _VP,
                        ctypes.c_int32, _VP, _VP],
    "cg_neumann_detect": [ctypes.POINTER(CgParams), ctypes.c_int64, _VP, _VP, _VP, _VP, _VP],
    "cg_neumann_precode": [ctypes.POINTER(CgParams), ctypes.c_int64, _VP, _VP, _VP, _VP,
                           ctypes.c_int32, _VP, _VP],
    "cg_release_workspace": [],
    "cg_plan_create": [ctypes.POINTER(CgDesc), ctypes.c_int64, ctypes.c_int32, _VP,
                       ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64)],
    "cg_plan_run": [_VP, _VP],
    "cg_plan_info": [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
    "cg_plan_destroy": [_VP],
    "cg_batch_run_static": [ctypes.POINTER(CgDesc), ctypes.c_int64, ctypes.c_int32, _VP],
    "cg_serve_create": [ctypes.POINTER(CgServeCfg), ctypes.POINTER(ctypes.c_void_p)],
    "cg_serve_submit": [_VP, ctypes.POINTER(CgDesc), ctypes.POINTER(ctypes.c_uint64)],
    "cg_serve_poll": [_VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                      ctypes.POINTER(CgReqStats)],
    "cg_serve_destroy": [_VP],
    "cg_set_wait_limit": [ctypes.c_int64],
    "cg_plan_schedule": [_VP, _VP],
    "cg_tune_cache_load": [ctypes.c_char_p],
    "cg_tune_cache_save": [ctypes.c_char_p],
    "cg_tune_cache_size": [],
    "cg_strerror": [ctypes.c_int],
    "cg_version": [],
}


def library(path: str | None = None) -> ctypes.CDLL:
    """Loads libcgmimo.so once (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise OSError(f"libcgmimo.so not found at {p}; run paper_1404_0424_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, args in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name == "cg_strerror" else ctypes.c_int
        _lib = lib
    return _lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):          # numpy array (host)
        return t.ctypes.data
    return int(t)


def _stream(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # noqa: BLE001
            return None
        return None
    return getattr(stream, "cuda_stream", stream)


def params(B, U, qam_bits, K, R, N0, Es=1.0, sinr_mode=0, amul_mode=0, precision=0) -> CgParams:
    return CgParams(int(B), int(U), int(qam_bits), int(K), int(R), float(N0), float(Es),
                    int(sinr_mode), int(amul_mode), int(precision))


# ---------------------------------------------------------------------------
# C ABI, same names
# ---------------------------------------------------------------------------

def cg_strerror(code: int) -> str:
    return library().cg_strerror(int(code)).decode()


def cg_set_wait_limit(timeout_ns: int) -> int:
    return library().cg_set_wait_limit(int(timeout_ns))


def cg_version() -> int:
    return library().cg_version()


def cg_release_workspace() -> int:
    return library().cg_release_workspace()


def cg_detect(p: CgParams, n_inst, H, Y, xhat=None, mu=None, rho=None, llr=None, status=None,
              stream=None) -> int:
    return library().cg_detect(ctypes.byref(p), int(n_inst), _ptr(H), _ptr(Y), _ptr(xhat),
                               _ptr(mu), _ptr(rho), _ptr(llr), _ptr(status), _stream(stream))


def cg_precode(p: CgParams, n_inst, H, T, q, qnorm=None, normalize=0, status=None,
               stream=None) -> int:
    return library().cg_precode(ctypes.byref(p), int(n_inst), _ptr(H), _ptr(T), _ptr(q),
                                _ptr(qnorm), int(normalize), _ptr(status), _stream(stream))


def cg_neumann_detect(p: CgParams, n_inst, H, Y, xhat, status=None, stream=None) -> int:
    return library().cg_neumann_detect(ctypes.byref(p), int(n_inst), _ptr(H), _ptr(Y),
                                       _ptr(xhat), _ptr(status), _stream(stream))


def cg_neumann_precode(p: CgParams, n_inst, H, T, q, qnorm=None, normalize=0, status=None,
                       stream=None) -> int:
    return library().cg_neumann_precode(ctypes.byref(p), int(n_inst), _ptr(H), _ptr(T), _ptr(q),
                                        _ptr(qnorm), int(normalize), _ptr(status),
                                        _stream(stream))


def cg_detect_host(p: CgParams, n_inst, H, Y, xhat=None, mu=None, rho=None, llr=None,
                   status=None, stream=None) -> int:
    return library().cg_detect_host(ctypes.byref(p), int(n_inst), _ptr(H), _ptr(Y), _ptr(xhat),
                                    _ptr(mu), _ptr(rho), _ptr(llr), _ptr(status),
                                    _stream(stream))


def cg_precode_host(p: CgParams, n_inst, H, T, q, qnorm=None, normalize=0, status=None,
                    stream=None) -> int:
    return library().cg_precode_host(ctypes.byref(p), int(n_inst), _ptr(H), _ptr(T), _ptr(q),
                                     _ptr(qnorm), int(normalize), _ptr(status), _stream(stream))


def cg_plan_create(descs, precision=-1, stream=None):
    """descs: sequence of CgDesc. Returns (rc, plan handle or None, bad_index)."""
    arr = (CgDesc * max(len(descs), 1))(*descs)
    plan = ctypes.c_void_p()
    bad = ctypes.c_int64(-1)
    rc = library().cg_plan_create(arr, len(descs), int(precision), _stream(stream),
                                  ctypes.byref(plan), ctypes.byref(bad))
    return rc, (plan.value if rc == 0 else None), bad.value


def cg_plan_run(plan, stream=None) -> int:
    return library().cg_plan_run(plan, _stream(stream))


def cg_plan_info(plan):
    prec = ctypes.c_int32()
    nb = ctypes.c_int32()
    rc = library().cg_plan_info(plan, ctypes.byref(prec), ctypes.byref(nb))
    return rc, prec.value, nb.value


class CgSchedule(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("order", ctypes.c_int32),
                ("concurrent", ctypes.c_int32), ("grid_pct", ctypes.c_int32),
                ("source", ctypes.c_int32), ("ms", ctypes.c_float)]


def cg_plan_schedule(plan):
    """Returns (rc, dict of the plan's schedule)."""
    s = CgSchedule()
    rc = library().cg_plan_schedule(plan, ctypes.byref(s))
    return rc, {f: getattr(s, f) for f, _ in CgSchedule._fields_}


def cg_tune_cache_load(path: str) -> int:
    return library().cg_tune_cache_load(os.fsencode(path))


def cg_tune_cache_save(path: str) -> int:
    return library().cg_tune_cache_save(os.fsencode(path))


def cg_tune_cache_size() -> int:
    return library().cg_tune_cache_size()


def cg_plan_destroy(plan) -> int:
    return library().cg_plan_destroy(plan)


def cg_batch_run_static(descs, precision=4, stream=None) -> int:
    """Batched problems through the allocation-free entry point (see cgmimo.h)."""
    arr = (CgDesc * max(len(descs), 1))(*descs)
    return library().cg_batch_run_static(arr, len(descs), int(precision), _stream(stream))


def cg_serve_create(capacity=256, precision=4, hbm_budget_bytes=40 << 30, max_B=256, max_R=16,
                    ctas_per_class=0, idle_timeout_ms=500):
    """Returns (rc, server handle or None)."""
    cfg = CgServeCfg(int(capacity), int(precision), int(hbm_budget_bytes), int(max_B),
                     int(max_R), int(ctas_per_class), int(idle_timeout_ms))
    srv = ctypes.c_void_p()
    rc = library().cg_serve_create(ctypes.byref(cfg), ctypes.byref(srv))
    return rc, (srv.value if rc == 0 else None)


def cg_serve_submit(server, req: CgDesc):
    """Returns (rc, ticket)."""
    t = ctypes.c_uint64()
    rc = library().cg_serve_submit(server, ctypes.byref(req), ctypes.byref(t))
    return rc, t.value


def cg_serve_poll(server, ticket):
    """Returns (rc, done, CgReqStats)."""
    done = ctypes.c_int32()
    st = CgReqStats()
    rc = library().cg_serve_poll(server, int(ticket), ctypes.byref(done), ctypes.byref(st))
    return rc, done.value, st


def cg_serve_destroy(server) -> int:
    return library().cg_serve_destroy(server)


def desc(op, B, U, R, K, N0, H, inp, out, qam_bits=2, Es=1.0, sinr_mode=0, normalize=0,
         mu=None, rho=None, aux=None, status=None, n_inst=None) -> CgDesc:
    """A CgDesc over tensors (n_inst defaults to H.shape[0])."""
    n = int(H.shape[0]) if n_inst is None else int(n_inst)
    return CgDesc(int(op), int(B), int(U), int(R), int(K), int(qam_bits), int(sinr_mode),
                  int(normalize), float(N0), float(Es), n, _ptr(H), _ptr(inp), _ptr(out),
                  _ptr(mu), _ptr(rho), _ptr(aux), _ptr(status))


# ---------------------------------------------------------------------------
# Conveniences over torch tensors (allocation and pointer marshalling only)
# ---------------------------------------------------------------------------

def _check(rc: int, where: str):
    if rc != 0:
        raise CgError(rc, where)


def detect(H, Y, N0, K, qam_bits, Es=1.0, sinr_mode=0, amul_mode=0, precision=0,
           outputs=("xhat", "mu", "rho", "llr", "status"), stream=None) -> dict:
    """CG-D on device tensors H[n, B, U], Y[n, R, B] (complex64, contiguous)."""
    import torch
    n, B, U = H.shape
    R = Y.shape[1]
    assert Y.shape == (n, R, B) and H.is_contiguous() and Y.is_contiguous()
    assert H.dtype == torch.complex64 and Y.dtype == torch.complex64
    dev = H.device
    out = {}
    if "xhat" in outputs:
        out["xhat"] = torch.empty((n, R, U), dtype=torch.complex64, device=dev)
    if "mu" in outputs:
        out["mu"] = torch.empty((n, R, U), dtype=torch.float32, device=dev)
    if "rho" in outputs:
        out["rho"] = torch.empty((n, R, U), dtype=torch.float32, device=dev)
    if "llr" in outputs:
        out["llr"] = torch.empty((n, R, U, qam_bits), dtype=torch.float32, device=dev)
    if "status" in outputs:
        out["status"] = torch.empty((n,), dtype=torch.int32, device=dev)
    p = params(B, U, qam_bits, K, R, N0, Es, sinr_mode, amul_mode, precision)
    _check(cg_detect(p, n, H, Y, out.get("xhat"), out.get("mu"), out.get("rho"), out.get("llr"),
                     out.get("status"), stream), "cg_detect")
    return out


def precode(H, T, N0, K, Es=1.0, normalize=False, amul_mode=0, precision=0, stream=None) -> dict:
    """CG-P on device tensors H[n, B, U], T[n, R, U] (complex64, contiguous)."""
    import torch
    n, B, U = H.shape
    R = T.shape[1]
    assert T.shape == (n, R, U) and H.is_contiguous() and T.is_contiguous()
    dev = H.device
    out = {"q": torch.empty((n, R, B), dtype=torch.complex64, device=dev),
           "qnorm": torch.empty((n, R), dtype=torch.float32, device=dev),
           "status": torch.empty((n,), dtype=torch.int32, device=dev)}
    p = params(B, U, 2, K, R, N0, Es, 0, amul_mode, precision)
    _check(cg_precode(p, n, H, T, out["q"], out["qnorm"], int(bool(normalize)), out["status"],
                      stream), "cg_precode")
    return out


def neumann_detect(H, Y, N0, K, Es=1.0, precision=4, stream=None) -> dict:
    """Neumann-series x_hat (Sec. III-F) on device tensors H[n, B, U], Y[n, R, B]."""
    import torch
    n, B, U = H.shape
    R = Y.shape[1]
    assert Y.shape == (n, R, B) and H.is_contiguous() and Y.is_contiguous()
    dev = H.device
    out = {"xhat": torch.empty((n, R, U), dtype=torch.complex64, device=dev),
           "status": torch.empty((n,), dtype=torch.int32, device=dev)}
    p = params(B, U, 2, K, R, N0, Es, 0, 0, precision)
    _check(cg_neumann_detect(p, n, H, Y, out["xhat"], out["status"], stream), "cg_neumann_detect")
    return out


def neumann_precode(H, T, N0, K, Es=1.0, normalize=False, precision=4, stream=None) -> dict:
    """Neumann-series precoding q = H v (Sec. III-F) on device tensors H[n, B, U], T[n, R, U]."""
    import torch
    n, B, U = H.shape
    R = T.shape[1]
    assert T.shape == (n, R, U) and H.is_contiguous() and T.is_contiguous()
    dev = H.device
    out = {"q": torch.empty((n, R, B), dtype=torch.complex64, device=dev),
           "qnorm": torch.empty((n, R), dtype=torch.float32, device=dev),
           "status": torch.empty((n,), dtype=torch.int32, device=dev)}
    p = params(B, U, 2, K, R, N0, Es, 0, 0, precision)
    _check(cg_neumann_precode(p, n, H, T, out["q"], out["qnorm"], int(bool(normalize)),
                              out["status"], stream), "cg_neumann_precode")
    return out
