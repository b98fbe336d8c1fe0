"""Serving (cg_serve_*): continuous batching of uneven requests.

Each request's result is the same alone and in the mix; results match the
single-shape calls; admission (ring slots, HBM budget), idle exit with
relaunch on demand, latency stamps and shutdown with work in flight. Every
wait in these tests is bounded on the host.
"""

import time

import numpy as np
import pytest

from paper_1404_0424_gb300 import workload as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cabi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_0424_gb300 import build, cabi as c
    c.library(build.build())
    return c


def wait_done(cabi, srv, tickets, timeout=30.0):
    stats = {}
    t0 = time.monotonic()
    pending = set(tickets)
    while pending:
        for t in list(pending):
            rc, done, st = cabi.cg_serve_poll(srv, t)
            assert rc == 0, cabi.cg_strerror(rc)
            if done:
                stats[t] = st
                pending.discard(t)
        assert time.monotonic() - t0 < timeout, f"requests {pending} not done in {timeout}s"
        time.sleep(0.0002)
    return stats


SHAPES = [(64, 8), (128, 16), (256, 32), (128, 32), (33, 5), (100, 12)]


def make_requests(dev, n_req=18, seed=4):
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n_req):
        B, U = SHAPES[k % len(SHAPES)]
        R = int(rng.integers(1, 15))
        q = int(rng.choice([4, 6, 8]))
        K = max(1, min(U // 4, 8))
        n = int(rng.integers(12, 200))
        op = k % 2
        snr = float(rng.uniform(5, 25))
        if op == 0:
            d = wl.uplink_torch(B, U, q, n=n, R=R, snr_db=snr, seed=seed * 100 + k, device=dev)
            inp = d["Y"]
        else:
            d = wl.downlink_torch(B, U, q, n=n, R=R, snr_db=snr, seed=seed * 100 + k, device=dev)
            inp = d["T"]
        reqs.append(dict(op=op, B=B, U=U, R=R, q=q, K=K, n=n, N0=d["N0"], H=d["H"], inp=inp))
    return reqs


def fresh_outputs(r, dev):
    n, R, U, B, q = r["n"], r["R"], r["U"], r["B"], r["q"]
    if r["op"] == 0:
        return {"xhat": torch.full((n, R, U), np.nan, dtype=torch.complex64, device=dev),
                "mu": torch.full((n, R, U), np.nan, device=dev),
                "rho": torch.full((n, R, U), np.nan, device=dev),
                "llr": torch.full((n, R, U, q), np.nan, device=dev),
                "status": torch.full((n,), -1, dtype=torch.int32, device=dev)}
    return {"q": torch.full((n, R, B), np.nan, dtype=torch.complex64, device=dev),
            "qnorm": torch.full((n, R), np.nan, device=dev),
            "status": torch.full((n,), -1, dtype=torch.int32, device=dev)}


def as_desc(cabi, r, o):
    if r["op"] == 0:
        return cabi.desc(0, r["B"], r["U"], r["R"], r["K"], r["N0"], r["H"], r["inp"], o["xhat"],
                         qam_bits=r["q"], mu=o["mu"], rho=o["rho"], aux=o["llr"],
                         status=o["status"])
    return cabi.desc(1, r["B"], r["U"], r["R"], r["K"], r["N0"], r["H"], r["inp"], o["q"],
                     aux=o["qnorm"], status=o["status"])


def submit(cabi, srv, d, timeout=20.0):
    # the request's buffers must be ready when it is submitted: the serving
    # kernels run on their own streams and do not wait for torch's stream
    torch.cuda.current_stream().synchronize()
    t0 = time.monotonic()
    while True:
        rc, t = cabi.cg_serve_submit(srv, d)
        if rc == 0:
            return t
        assert rc == cabi.CG_EAGAIN, cabi.cg_strerror(rc)
        assert time.monotonic() - t0 < timeout, "submit kept returning CG_EAGAIN"
        time.sleep(0.0005)


def test_same_result_alone_and_in_the_mix(cabi):
    dev = torch.device("cuda:0")
    reqs = make_requests(dev)
    rc, srv = cabi.cg_serve_create(capacity=64, precision=4, idle_timeout_ms=300)
    assert rc == 0, cabi.cg_strerror(rc)
    try:
        alone = []
        for r in reqs:                       # one at a time
            o = fresh_outputs(r, dev)
            st = wait_done(cabi, srv, [submit(cabi, srv, as_desc(cabi, r, o))])
            assert all(s.status == 0 for s in st.values())
            alone.append(o)
        mixed = [fresh_outputs(r, dev) for r in reqs]
        tickets = [submit(cabi, srv, as_desc(cabi, r, o)) for r, o in zip(reqs, mixed)]
        stats = wait_done(cabi, srv, tickets)
        for r, a, m in zip(reqs, alone, mixed):
            for k in a:
                assert torch.equal(a[k], m[k]), f"{k} of request {r['op'], r['B'], r['U']} differs"
        for t in tickets:
            st = stats[t]
            assert st.status == 0
            assert 0 < st.submit_ns <= st.complete_ns
            assert 0 < st.device_first_ns <= st.device_done_ns
    finally:
        assert cabi.cg_serve_destroy(srv) == 0
    # and the served results equal the single-shape calls of the same precision
    for r, m in zip(reqs, mixed):
        if r["op"] == 0:
            ref = cabi.detect(r["H"], r["inp"], r["N0"], r["K"], r["q"], precision=4)
        else:
            ref = cabi.precode(r["H"], r["inp"], r["N0"], r["K"], precision=4)
        torch.cuda.synchronize()
        for k in m:
            assert torch.equal(m[k], ref[k]), f"served {k} differs from the single call"


def test_exact_tracker_requests(cabi):
    # exact-tracker detection (Eq. 10) at every padded user count runs on the warp
    # serving kernel with the single calls' body: bitwise equal to the single call,
    # and at 32 users also checked against the FP64 oracle
    import oracle
    from tests.parity import check_detect, to_np
    dev = torch.device("cuda:0")
    reqs = []
    for k, (B, U) in enumerate([(64, 8), (128, 16), (100, 12), (128, 32)]):
        R, q, K = 5, 4, min(U, 4)
        d = wl.uplink_torch(B, U, q, n=40, R=R, snr_db=8.0, seed=700 + k, device=dev)
        reqs.append(dict(op=0, B=B, U=U, R=R, q=q, K=K, n=40, N0=d["N0"], H=d["H"], inp=d["Y"]))
    rc, srv = cabi.cg_serve_create(capacity=16, precision=4, idle_timeout_ms=300)
    assert rc == 0, cabi.cg_strerror(rc)
    outs = [fresh_outputs(r, dev) for r in reqs]
    try:
        tickets = []
        for r, o in zip(reqs, outs):
            dsc = cabi.desc(0, r["B"], r["U"], r["R"], r["K"], r["N0"], r["H"], r["inp"],
                            o["xhat"], qam_bits=r["q"], sinr_mode=1, mu=o["mu"], rho=o["rho"],
                            aux=o["llr"], status=o["status"])
            tickets.append(submit(cabi, srv, dsc))
        wait_done(cabi, srv, tickets)
    finally:
        assert cabi.cg_serve_destroy(srv) == 0
    for r, o in zip(reqs, outs):
        ref = cabi.detect(r["H"], r["inp"], r["N0"], r["K"], r["q"], sinr_mode=1, precision=4)
        torch.cuda.synchronize()
        for k in o:
            assert torch.equal(o[k], ref[k]), f"served exact {k} differs at U={r['U']}"
        if r["U"] > 16:
            ref = oracle.cg_detect(r["H"].cpu().numpy(), r["inp"].cpu().numpy(), r["N0"], 1.0,
                                   r["K"], r["q"], "exact")
            check_detect({k: to_np(v) for k, v in o.items()}, ref)


def test_admission_by_slots_and_budget(cabi):
    dev = torch.device("cuda:0")
    r = make_requests(dev, n_req=1, seed=9)[0]
    r["n"] = 4000
    big = wl.uplink_torch(r["B"], r["U"], r["q"], n=4000, R=r["R"], snr_db=10.0, seed=1,
                          device=dev)
    r.update(H=big["H"], inp=big["Y"], op=0, N0=big["N0"])
    foot = 4000 * ((r["B"] * r["U"] + r["R"] * r["B"]) * 8 +
                   r["R"] * r["U"] * (16 + 4 * r["q"]) + 4)
    # budget for one request: a second one waits for the first to finish
    rc, srv = cabi.cg_serve_create(capacity=8, precision=4, hbm_budget_bytes=int(foot * 1.5),
                                   idle_timeout_ms=300)
    assert rc == 0
    try:
        o1, o2 = fresh_outputs(r, dev), fresh_outputs(r, dev)
        torch.cuda.current_stream().synchronize()
        rc, t1 = cabi.cg_serve_submit(srv, as_desc(cabi, r, o1))
        assert rc == 0
        rc, _ = cabi.cg_serve_submit(srv, as_desc(cabi, r, o2))
        assert rc in (cabi.CG_EAGAIN, 0)
        if rc == cabi.CG_EAGAIN:
            wait_done(cabi, srv, [t1])
            rc, t2 = cabi.cg_serve_submit(srv, as_desc(cabi, r, o2))
            assert rc == 0
            wait_done(cabi, srv, [t2])
        too_big = as_desc(cabi, r, o1)
        too_big.n_inst = 8000
        assert cabi.cg_serve_submit(srv, too_big)[0] == cabi.CG_ETOOBIG
    finally:
        assert cabi.cg_serve_destroy(srv) == 0
    # one ring slot: the second submit is refused until the first completes
    rc, srv = cabi.cg_serve_create(capacity=1, precision=4, idle_timeout_ms=300)
    try:
        o1, o2 = fresh_outputs(r, dev), fresh_outputs(r, dev)
        torch.cuda.current_stream().synchronize()
        rc, t1 = cabi.cg_serve_submit(srv, as_desc(cabi, r, o1))
        assert rc == 0
        rc2, _ = cabi.cg_serve_submit(srv, as_desc(cabi, r, o2))
        st = wait_done(cabi, srv, [t1])
        assert st[t1].status == 0
        if rc2 == cabi.CG_EAGAIN:
            rc2, t2 = cabi.cg_serve_submit(srv, as_desc(cabi, r, o2))
            assert rc2 == 0
            wait_done(cabi, srv, [t2])
        assert torch.equal(o1["xhat"], o2["xhat"])
    finally:
        assert cabi.cg_serve_destroy(srv) == 0


def test_idle_exit_relaunch_and_shutdown_in_flight(cabi):
    dev = torch.device("cuda:0")
    reqs = make_requests(dev, n_req=4, seed=12)
    rc, srv = cabi.cg_serve_create(capacity=16, precision=3, idle_timeout_ms=20)
    assert rc == 0
    try:
        outs = [fresh_outputs(r, dev) for r in reqs]
        wait_done(cabi, srv, [submit(cabi, srv, as_desc(cabi, reqs[0], outs[0]))])
        time.sleep(0.3)                 # every class kernel has idled out
        t = submit(cabi, srv, as_desc(cabi, reqs[1], outs[1]))   # relaunch on demand
        wait_done(cabi, srv, [t])
        for r, o in zip(reqs[2:], outs[2:]):
            submit(cabi, srv, as_desc(cabi, r, o))
    finally:
        assert cabi.cg_serve_destroy(srv) == 0   # stops with work possibly in flight
    torch.cuda.synchronize()


def test_slots_are_reused_only_after_poll_and_results_hold_under_reuse(cabi):
    """Many more requests than ring slots, of every class: a finished request
    keeps its slot until polled (submit says CG_EAGAIN meanwhile), a poll
    never fails for a ticket still in flight, and every result equals the
    single-shape call although each slot is reused many times."""
    dev = torch.device("cuda:0")
    reqs = make_requests(dev, n_req=60, seed=21)
    for r in reqs:                          # keep each request small: frequent reuse
        r["n"] = min(r["n"], 40)
        r["H"] = r["H"][:r["n"]].contiguous()
        r["inp"] = r["inp"][:r["n"]].contiguous()
    outs = [fresh_outputs(r, dev) for r in reqs]
    torch.cuda.current_stream().synchronize()
    rc, srv = cabi.cg_serve_create(capacity=4, precision=4, idle_timeout_ms=300)
    assert rc == 0, cabi.cg_strerror(rc)
    try:
        # fill every slot, let the requests finish unpolled: no slot frees up
        first = [submit(cabi, srv, as_desc(cabi, r, o)) for r, o in zip(reqs[:4], outs[:4])]
        torch.cuda.synchronize()   # returns once the class kernels have idled out
        assert all(bool((outs[k]["status"] == 0).all()) for k in range(4))
        assert cabi.cg_serve_submit(srv, as_desc(cabi, reqs[4], outs[4]))[0] == cabi.CG_EAGAIN
        wait_done(cabi, srv, first)
        # a reaped ticket reports done again while its slot is not reused
        rc, done, _ = cabi.cg_serve_poll(srv, first[0])
        assert rc == 0 and done == 1
        # the rest, polled lazily as in a load generator
        pending, k = {}, 4
        t0 = time.monotonic()
        while k < len(reqs) or pending:
            while k < len(reqs):
                rc, t = cabi.cg_serve_submit(srv, as_desc(cabi, reqs[k], outs[k]))
                if rc == cabi.CG_EAGAIN:
                    break
                assert rc == 0, cabi.cg_strerror(rc)
                pending[t] = k
                k += 1
            for t in list(pending):
                rc, done, st = cabi.cg_serve_poll(srv, t)
                assert rc == 0, f"poll of in-flight ticket {t}: {cabi.cg_strerror(rc)}"
                if done:
                    assert st.status == 0
                    del pending[t]
            assert time.monotonic() - t0 < 60, "requests did not finish"
    finally:
        assert cabi.cg_serve_destroy(srv) == 0
    for r, m in zip(reqs, outs):
        if r["op"] == 0:
            ref = cabi.detect(r["H"], r["inp"], r["N0"], r["K"], r["q"], precision=4)
        else:
            ref = cabi.precode(r["H"], r["inp"], r["N0"], r["K"], precision=4)
        torch.cuda.synchronize()
        for key in m:
            assert torch.equal(m[key], ref[key]), f"served {key} differs from the single call"
