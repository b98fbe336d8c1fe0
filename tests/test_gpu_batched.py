"""Batched uneven problems (cg_plan_*): each problem's result inside a mixed
batch equals the single-shape call bit for bit, and a sample matches the
FP64 oracle."""

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
    return c


SHAPES = [(64, 8), (128, 16), (128, 32), (256, 32), (100, 12), (33, 5), (48, 3), (72, 24)]


def make_batch(n_prob, seed, dev, exact_every=5):
    rng = np.random.default_rng(seed)
    probs = []
    for k in range(n_prob):
        B, U = SHAPES[rng.integers(len(SHAPES))]
        q = int(rng.choice([4, 6, 8]))
        R = int(rng.integers(1, 15))
        K = int(max(1, min(U // 4, 8)))
        snr = float(rng.uniform(5, 25))
        n = int(rng.integers(1, 4))
        op = int(rng.integers(2))
        exact = int(op == 0 and k % exact_every == 0)
        if op == 0:
            d = wl.uplink(B, U, q, n=n, R=R, snr_db=snr, seed=seed * 1000 + k)
            t = {"H": torch.from_numpy(d["H"]).to(dev), "Y": torch.from_numpy(d["Y"]).to(dev),
                 "xhat": torch.full((n, R, U), np.nan, dtype=torch.complex64, device=dev),
                 "mu": torch.full((n, R, U), np.nan, device=dev),
                 "rho": torch.full((n, R, U), np.nan, device=dev),
                 "llr": torch.full((n, R, U, q), np.nan, device=dev),
                 "status": torch.full((n,), -1, dtype=torch.int32, device=dev)}
        else:
            d = wl.downlink(B, U, q, n=n, R=R, snr_db=snr, seed=seed * 1000 + k)
            t = {"H": torch.from_numpy(d["H"]).to(dev), "T": torch.from_numpy(d["T"]).to(dev),
                 "q": torch.full((n, R, B), np.nan, dtype=torch.complex64, device=dev),
                 "qnorm": torch.full((n, R), np.nan, device=dev),
                 "status": torch.full((n,), -1, dtype=torch.int32, device=dev)}
        probs.append({"op": op, "B": B, "U": U, "R": R, "K": K, "q": q, "n": n, "exact": exact,
                      "normalize": int(op == 1 and k % 3 == 0), "d": d, "t": t})
    return probs


def descs(cabi, probs):
    out = []
    for p in probs:
        t = p["t"]
        if p["op"] == 0:
            out.append(cabi.desc(0, p["B"], p["U"], p["R"], p["K"], p["d"]["N0"], t["H"], t["Y"],
                                 t["xhat"], qam_bits=p["q"], sinr_mode=p["exact"], mu=t["mu"],
                                 rho=t["rho"], aux=t["llr"], status=t["status"]))
        else:
            out.append(cabi.desc(1, p["B"], p["U"], p["R"], p["K"], p["d"]["N0"], t["H"], t["T"],
                                 t["q"], normalize=p["normalize"], aux=t["qnorm"],
                                 status=t["status"]))
    return out


def single(cabi, p, precision):
    t = p["t"]
    if p["op"] == 0:
        return cabi.detect(t["H"], t["Y"], p["d"]["N0"], p["K"], p["q"], sinr_mode=p["exact"],
                           precision=precision)
    return cabi.precode(t["H"], t["T"], p["d"]["N0"], p["K"], normalize=bool(p["normalize"]),
                        precision=precision)


@pytest.mark.parametrize("precision", [4, 3])
def test_batch_equals_single_calls_bitwise(cabi, precision):
    dev = torch.device("cuda:0")
    probs = make_batch(40, seed=11 + precision, dev=dev)
    rc, plan, bad = cabi.cg_plan_create(descs(cabi, probs), precision)
    assert rc == 0, (cabi.cg_strerror(rc), bad)
    try:
        rc, prec, nbins = cabi.cg_plan_info(plan)
        assert rc == 0 and prec == precision and nbins >= 4
        assert cabi.cg_plan_run(plan) == 0
        torch.cuda.synchronize()
        first = [{k: v.clone() for k, v in p["t"].items()} for p in probs]
        assert cabi.cg_plan_run(plan) == 0   # replay: same outputs
        torch.cuda.synchronize()
        for p, f in zip(probs, first):
            ref = single(cabi, p, precision)
            torch.cuda.synchronize()
            keys = ("xhat", "mu", "rho", "llr", "status") if p["op"] == 0 else ("q", "qnorm",
                                                                               "status")
            for k in keys:
                assert torch.equal(p["t"][k], f[k]), f"replay differs in {k}"
                assert torch.equal(p["t"][k], ref[k]), (f"{k} differs from the single call for "
                                                        f"{p['op'], p['B'], p['U'], p['R']}")
    finally:
        cabi.cg_plan_destroy(plan)


def test_batch_matches_oracle(cabi):
    dev = torch.device("cuda:0")
    probs = make_batch(24, seed=5, dev=dev)
    rc, plan, bad = cabi.cg_plan_create(descs(cabi, probs), 4)
    assert rc == 0, (cabi.cg_strerror(rc), bad)
    try:
        assert cabi.cg_plan_run(plan) == 0
        torch.cuda.synchronize()
    finally:
        cabi.cg_plan_destroy(plan)
    for p in probs:
        d = p["d"]
        t = p["t"]
        if p["op"] == 0:
            r = oracle.cg_detect(d["H"], d["Y"], d["N0"], 1.0, p["K"], p["q"],
                                 "exact" if p["exact"] else "approx")
            check_detect({k: to_np(t[k]) for k in ("xhat", "mu", "rho", "llr", "status")}, r)
        else:
            r = oracle.cg_precode(d["H"], d["T"], d["N0"], 1.0, p["K"])
            check_precode({k: to_np(t[k]) for k in ("q", "qnorm", "status")}, r,
                          normalize=bool(p["normalize"]))


def test_auto_precision_and_config_batch(cabi):
    # 4096 problems drawn like the uneven-batch workload; AUTO picks a split mode
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(3)
    shapes = [(64, 8), (128, 16), (128, 32), (256, 32)]
    probs = []
    n = 4096
    keep = []
    for k in range(n):
        B, U = shapes[rng.integers(4)]
        R = int(rng.integers(1, 15))
        q = int(rng.choice([4, 6, 8]))
        probs.append((B, U, R, q, float(rng.uniform(5, 25))))
    ds = []
    for k, (B, U, R, q, snr) in enumerate(probs):
        H = torch.randn((1, B, U), dtype=torch.complex64, device=dev)
        Y = torch.randn((1, R, B), dtype=torch.complex64, device=dev)
        out = {"xhat": torch.empty((1, R, U), dtype=torch.complex64, device=dev),
               "mu": torch.empty((1, R, U), device=dev), "rho": torch.empty((1, R, U), device=dev),
               "llr": torch.empty((1, R, U, q), device=dev),
               "status": torch.empty((1,), dtype=torch.int32, device=dev)}
        keep.append((H, Y, out))
        ds.append(cabi.desc(0, B, U, R, max(1, min(U // 4, 8)), wl.snr_to_n0(snr, U), H, Y,
                            out["xhat"], qam_bits=q, mu=out["mu"], rho=out["rho"],
                            aux=out["llr"], status=out["status"]))
    rc, plan, bad = cabi.cg_plan_create(ds, -1)
    assert rc == 0, (cabi.cg_strerror(rc), bad)
    try:
        rc, prec, nb = cabi.cg_plan_info(plan)
        assert prec in (3, 4) and nb == 3   # (128,32) and (256,32) share the UT=32 bin
        assert cabi.cg_plan_run(plan) == 0
        torch.cuda.synchronize()
        assert all(int(o["status"][0]) == 0 for _, _, o in keep)
        for idx in (0, 17, 999, 4095):
            H, Y, o = keep[idx]
            B, U, R, q, snr = probs[idx]
            r = oracle.cg_detect(H.cpu().numpy(), Y.cpu().numpy(), wl.snr_to_n0(snr, U), 1.0,
                                 max(1, min(U // 4, 8)), q)
            check_detect({k: to_np(v) for k, v in o.items()}, r)
    finally:
        cabi.cg_plan_destroy(plan)


def test_autotuner_times_then_caches_schedules(cabi, tmp_path):
    """CG_PREC_AUTO times the schedule candidates on the batch (source
    TIMED); a second plan of the same shape class takes the schedule from the
    cache (CACHED); the cache file round-trips through save and load; a fixed
    precision gets the default schedule (FIXED). Every schedule gives the
    single calls' results."""
    dev = torch.device("cuda:0")
    probs = make_batch(48, seed=21, dev=dev, exact_every=7)
    ds = descs(cabi, probs)
    rc, plan, bad = cabi.cg_plan_create(ds, -1)
    assert rc == 0, (cabi.cg_strerror(rc), bad)
    try:
        rc, s1 = cabi.cg_plan_schedule(plan)
        assert rc == 0 and s1["source"] == cabi.CG_TUNE_TIMED and s1["ms"] > 0
        assert s1["precision"] in (3, 4) and s1["order"] in (0, 1) and 1 <= s1["grid_pct"] <= 100
        assert cabi.cg_plan_run(plan) == 0
        torch.cuda.synchronize()
        for p in probs:
            ref = single(cabi, p, s1["precision"])
            torch.cuda.synchronize()
            keys = ("xhat", "mu", "rho", "llr", "status") if p["op"] == 0 else ("q", "qnorm",
                                                                               "status")
            for k in keys:
                assert torch.equal(p["t"][k], ref[k]), f"{k} differs from the single call"
    finally:
        cabi.cg_plan_destroy(plan)
    rc, plan2, _ = cabi.cg_plan_create(ds, -1)
    assert rc == 0
    try:
        rc, s2 = cabi.cg_plan_schedule(plan2)
        assert s2["source"] == cabi.CG_TUNE_CACHED
        assert all(s2[f] == s1[f] for f in ("precision", "order", "concurrent", "grid_pct"))
    finally:
        cabi.cg_plan_destroy(plan2)
    path = tmp_path / "tune.json"
    n = cabi.cg_tune_cache_save(str(path))
    assert n >= 1 and cabi.cg_tune_cache_load(str(path)) == n
    rc, plan3, _ = cabi.cg_plan_create(ds, 4)
    assert rc == 0
    try:
        rc, s3 = cabi.cg_plan_schedule(plan3)
        assert s3["source"] == cabi.CG_TUNE_FIXED and s3["precision"] == 4
    finally:
        cabi.cg_plan_destroy(plan3)


def test_cached_schedule_decides(cabi, tmp_path):
    """An entry of the schedule cache, edited and loaded back, is the schedule
    the next plan of that shape class runs (source CACHED), and its results
    still equal the single calls."""
    import json
    dev = torch.device("cuda:0")
    probs = make_batch(24, seed=31, dev=dev, exact_every=11)
    ds = descs(cabi, probs)
    rc, plan, _ = cabi.cg_plan_create(ds, -1)
    assert rc == 0
    _, s1 = cabi.cg_plan_schedule(plan)
    cabi.cg_plan_destroy(plan)
    path = tmp_path / "tune.json"
    assert cabi.cg_tune_cache_save(str(path)) >= 1
    entries = json.loads(path.read_text())
    # the entry timed just now: the one whose fields equal the plan's schedule
    mine = [e for e in entries if all(e[f] == s1[f] for f in
                                      ("precision", "order", "concurrent", "grid_pct"))]
    assert mine
    want = {"precision": 3 if s1["precision"] == 4 else 4, "order": 1 - s1["order"],
            "concurrent": 1 - s1["concurrent"], "grid_pct": 50}
    for e in mine:
        e.update(want)
    path.write_text("[\n" + ",\n".join(json.dumps(e) for e in mine) + "\n]\n")
    assert cabi.cg_tune_cache_load(str(path)) == len(mine)
    rc, plan2, _ = cabi.cg_plan_create(ds, -1)
    assert rc == 0
    try:
        _, s2 = cabi.cg_plan_schedule(plan2)
        assert s2["source"] == cabi.CG_TUNE_CACHED
        assert all(s2[f] == want[f] for f in want), (s2, want)
        assert cabi.cg_plan_run(plan2) == 0
        torch.cuda.synchronize()
        for p in probs:
            ref = single(cabi, p, s2["precision"])
            torch.cuda.synchronize()
            keys = ("xhat", "mu", "rho", "llr", "status") if p["op"] == 0 else ("q", "qnorm",
                                                                               "status")
            for k in keys:
                assert torch.equal(p["t"][k], ref[k]), f"{k} differs from the single call"
    finally:
        cabi.cg_plan_destroy(plan2)


_CHILD = r"""
import sys, torch
sys.path.insert(0, {root!r})
from tests.test_gpu_batched import make_batch, descs
from paper_1404_0424_gb300 import build, cabi
cabi.library(build.build())
probs = make_batch(20, seed=41, dev=torch.device("cuda:0"), exact_every=13)
rc, plan, _ = cabi.cg_plan_create(descs(cabi, probs), -1)
assert rc == 0
_, s = cabi.cg_plan_schedule(plan)
cabi.cg_plan_destroy(plan)
print(s["source"], s["precision"], s["order"], s["concurrent"], s["grid_pct"])
"""


def test_schedule_cache_file_across_processes(cabi, tmp_path):
    """With CGMIMO_TUNE_CACHE naming a file, a schedule timed in one process
    is taken from the file by the next process (source CACHED)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CGMIMO_TUNE_CACHE=str(tmp_path / "cache.json"))
    code = _CHILD.format(root=root)
    outs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=600, cwd=root)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(r.stdout.split())
    assert int(outs[0][0]) == cabi.CG_TUNE_TIMED
    assert int(outs[1][0]) == cabi.CG_TUNE_CACHED
    assert outs[0][1:] == outs[1][1:]
    assert (tmp_path / "cache.json").exists()
