"""The C-ABI library builds, loads, exports every declared symbol and rejects
invalid arguments on the host (no GPU needed: validation precedes CUDA)."""

import ctypes
import os
import re

import pytest

from paper_1404_0424_gb300 import build, cabi

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared_functions():
    names = set()
    for fn in os.listdir(INCLUDE):
        if fn.endswith(".h"):
            src = open(os.path.join(INCLUDE, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(cg_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return cabi.library(build.build())


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "cg_detect" in names and "cg_precode" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
        assert isinstance(getattr(lib, n), ctypes._CFuncPtr)


def test_binding_names_match_the_abi():
    for n in declared_functions():
        assert callable(getattr(cabi, n, None)), f"binding lacks {n}"


def test_version_and_strerror(lib):
    assert cabi.cg_version() >= 100
    assert cabi.cg_strerror(cabi.CG_EINVAL).startswith("CG_EINVAL")
    assert "unknown" in cabi.cg_strerror(12345)


GOOD = dict(B=32, U=4, qam_bits=4, K=3, R=1, N0=0.4)


@pytest.mark.parametrize("bad", [
    dict(U=0), dict(U=33), dict(B=3), dict(B=257), dict(R=0), dict(R=17), dict(K=0),
    dict(K=5), dict(qam_bits=3), dict(qam_bits=10), dict(N0=0.0), dict(N0=float("nan")),
    dict(N0=-1.0), dict(N0=float("inf"))])
def test_detect_rejects_invalid_parameters(lib, bad):
    kw = {**GOOD, **bad}
    p = cabi.params(kw["B"], kw["U"], kw["qam_bits"], kw["K"], kw["R"], kw["N0"])
    assert cabi.cg_detect(p, 4, 16, 16) == cabi.CG_EINVAL
    assert cabi.cg_detect_host(p, 4, 16, 16) == cabi.CG_EINVAL


def test_detect_rejects_bad_modes_pointers_and_counts(lib):
    p = cabi.params(32, 4, 4, 3, 1, 0.4, Es=1.0, sinr_mode=2)
    assert cabi.cg_detect(p, 1, 16, 16) == cabi.CG_EINVAL
    p = cabi.params(32, 4, 4, 3, 1, 0.4, amul_mode=7)
    assert cabi.cg_detect(p, 1, 16, 16) == cabi.CG_EINVAL
    p = cabi.params(32, 4, 4, 3, 1, 0.4, precision=9)
    assert cabi.cg_detect(p, 1, 16, 16) == cabi.CG_EINVAL
    # the exact tracker needs the Gram: no implicit product with it
    p = cabi.params(32, 4, 4, 3, 1, 0.4, sinr_mode=1, amul_mode=2)
    assert cabi.cg_detect(p, 1, 16, 16) == cabi.CG_ENOTSUP
    p = cabi.params(32, 4, 4, 3, 1, 0.4, Es=0.0)
    assert cabi.cg_detect(p, 1, 16, 16) == cabi.CG_EINVAL
    p = cabi.params(**GOOD)
    assert cabi.cg_detect(p, -1, 16, 16) == cabi.CG_EINVAL
    assert cabi.cg_detect(p, 1, None, 16) == cabi.CG_EINVAL
    assert cabi.cg_detect(p, 1, 16, 12) == cabi.CG_EINVAL       # Y not 8-byte aligned
    assert cabi.cg_detect(p, 1, 16, 16, 20) == cabi.CG_EINVAL   # xhat not 8-byte aligned
    assert cabi.cg_detect(p, 1, 16, 16, None, None, None, 12) == cabi.CG_EINVAL  # llr
    assert lib.cg_detect(None, 1, 16, 16, None, None, None, None, None, None) == cabi.CG_EINVAL
    assert cabi.cg_detect(p, 0, None, None) == cabi.CG_OK         # empty batch


def test_precode_rejects_invalid_arguments(lib):
    p = cabi.params(**GOOD)
    assert cabi.cg_precode(p, 1, 16, 16, None) == cabi.CG_EINVAL  # q required
    assert cabi.cg_precode(p, 1, 16, 16, 16, 2) == cabi.CG_EINVAL  # qnorm misaligned
    p = cabi.params(32, 4, 4, 5, 1, 0.4)
    assert cabi.cg_precode(p, 1, 16, 16, 16) == cabi.CG_EINVAL
    assert cabi.cg_precode_host(p, 1, 16, 16, 16) == cabi.CG_EINVAL
    assert cabi.cg_precode(cabi.params(**GOOD), 0, None, None, None) == cabi.CG_OK


def test_plan_rejects_invalid_descriptors_on_the_host(lib):
    good = cabi.CgDesc(0, 32, 4, 1, 3, 4, 0, 0, 0.5, 1.0, 1, 16, 16, 16, None, None, None, None)
    bad_k = cabi.CgDesc(0, 32, 4, 1, 5, 4, 0, 0, 0.5, 1.0, 1, 16, 16, 16, None, None, None, None)
    bad_op = cabi.CgDesc(7, 32, 4, 1, 3, 4, 0, 0, 0.5, 1.0, 1, 16, 16, 16, None, None, None, None)
    no_q = cabi.CgDesc(1, 32, 4, 1, 3, 4, 0, 0, 0.5, 1.0, 1, 16, 16, None, None, None, None, None)
    neg_n = cabi.CgDesc(0, 32, 4, 1, 3, 4, 0, 0, 0.5, 1.0, -2, 16, 16, 16, None, None, None, None)
    for descs, idx in (([good, bad_k], 1), ([bad_op], 0), ([good, good, no_q], 2), ([neg_n], 0)):
        rc, plan, bad = cabi.cg_plan_create(descs, 4)
        assert rc == cabi.CG_EINVAL and plan is None and bad == idx
    assert cabi.cg_plan_create([good], 0)[0] == cabi.CG_ENOTSUP     # FP32 plans: no
    assert cabi.cg_plan_create([good], 9)[0] == cabi.CG_EINVAL
    assert lib.cg_plan_run(None, None) == cabi.CG_EINVAL
    assert lib.cg_plan_destroy(None) == cabi.CG_EINVAL


def test_serve_rejects_invalid_configuration_on_the_host(lib):
    for bad in (dict(capacity=0), dict(capacity=(1 << 14) + 1), dict(precision=0),
                dict(precision=7), dict(hbm_budget_bytes=0),
                dict(max_B=0), dict(max_B=257), dict(max_R=17), dict(ctas_per_class=-1),
                dict(idle_timeout_ms=0), dict(idle_timeout_ms=120000)):
        rc, srv = cabi.cg_serve_create(**bad)
        assert rc == cabi.CG_EINVAL and srv is None, bad
    good = cabi.CgDesc(0, 32, 4, 1, 3, 4, 0, 0, 0.5, 1.0, 1, 16, 16, 16, None, None, None, None)
    assert cabi.cg_serve_submit(None, good)[0] == cabi.CG_EINVAL
    assert cabi.cg_serve_poll(None, 0)[0] == cabi.CG_EINVAL
    assert lib.cg_serve_destroy(None) == cabi.CG_EINVAL


def test_cgls_and_neumann_reject_on_the_host(lib):
    # CGLS needs no Gram, so it does not combine with the exact tracker
    p = cabi.params(32, 4, 4, 3, 1, 0.4, sinr_mode=1, amul_mode=cabi.CG_AMUL_CGLS)
    assert cabi.cg_detect(p, 1, 16, 16) == cabi.CG_ENOTSUP
    p = cabi.params(32, 4, 4, 3, 1, 0.4, amul_mode=cabi.CG_AMUL_CGLS + 1)
    assert cabi.cg_detect(p, 1, 16, 16) == cabi.CG_EINVAL
    # Neumann series: 1 <= K <= CG_NEUMANN_K_MAX terms, a tensor-core precision,
    # x_hat (detection) or q (precoding) required
    for K, prec, want in [(0, 4, cabi.CG_EINVAL), (cabi.CG_NEUMANN_K_MAX + 1, 4, cabi.CG_EINVAL),
                          (3, cabi.CG_PREC_FP32, cabi.CG_ENOTSUP), (3, 9, cabi.CG_EINVAL)]:
        p = cabi.params(32, 4, 4, K, 1, 0.4, precision=prec)
        assert cabi.cg_neumann_detect(p, 1, 16, 16, 16) == want, (K, prec)
        assert cabi.cg_neumann_precode(p, 1, 16, 16, 16) == want, (K, prec)
    p = cabi.params(32, 4, 4, 3, 1, 0.4, precision=4)
    assert cabi.cg_neumann_detect(p, 1, 16, 16, None) == cabi.CG_EINVAL
    assert cabi.cg_neumann_detect(p, 1, 16, 12, 16) == cabi.CG_EINVAL   # Y not 8-byte aligned
    assert cabi.cg_neumann_detect(p, -1, 16, 16, 16) == cabi.CG_EINVAL
    assert cabi.cg_neumann_precode(p, 1, 16, 16, None) == cabi.CG_EINVAL
    assert cabi.cg_neumann_precode(p, 1, None, 16, 16) == cabi.CG_EINVAL
    assert lib.cg_neumann_detect(None, 1, None, None, None, None, None) == cabi.CG_EINVAL
    assert lib.cg_neumann_precode(None, 1, None, None, None, None, 0, None, None) == \
        cabi.CG_EINVAL


def test_wait_limit_range(lib):
    assert cabi.cg_set_wait_limit(-1) == cabi.CG_EINVAL
    assert cabi.cg_set_wait_limit(61 * 10**9) == cabi.CG_EINVAL
    assert cabi.cg_set_wait_limit(0) == cabi.CG_OK      # back to the 2 s default
