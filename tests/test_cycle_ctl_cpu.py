"""Algorithm 1's outer-loop decisions as the solver takes them (ctl_plan, ctl_params, ctl_mid,
ctl_collect in csrc/solver_impl.cuh, the same functions the device runs in its one-thread
kernels), driven on the host by tests/ctl_harness.cu and checked against the reading of
Algorithm 1: r_0 = r^high / s_l, the inner stop rho <= max(delta^2, (tol ||eta|| / s_l)^2),
beta_0 = s_l / (s_{l-1} rho_k) for a continued direction, a fresh start p_0 = r_0 when the
true residual leaves the recurrence's prediction (s_l > 2 s_{l-1} sqrt(rho_k)), stagnation
after five cycles without a 0.1% improvement, and the cycle and iteration caps.  Needs nvcc
(no GPU)."""
import math
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

LQ_OK, LQ_NOT_CONVERGED, LQ_ERR_NONFINITE, LQ_ERR_BREAKDOWN = 0, 1, -6, -7


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def ctl_out(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("ctl") / "ctl_harness")
    cmd = [nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a", "-O1",
           os.path.join(HERE, "ctl_harness.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    recs = {}
    for line in out.stdout.splitlines():
        tag, *rest = line.split()
        if len(rest) == 1:
            recs[tag] = int(rest[0])
        else:
            recs[tag] = {k: float(v) for k, v in (kv.split("=") for kv in rest)}
    return recs


def _status_code(name):
    import re
    text = open(os.path.join(ROOT, "include", "lq.h")).read()
    return int(re.search(r"\b" + name + r"\s*=\s*(-?\d+)", text).group(1))


def test_status_codes_match_the_header():
    assert _status_code("LQ_OK") == LQ_OK and _status_code("LQ_NOT_CONVERGED") == LQ_NOT_CONVERGED
    assert _status_code("LQ_ERR_NONFINITE") == LQ_ERR_NONFINITE
    assert _status_code("LQ_ERR_BREAKDOWN") == LQ_ERR_BREAKDOWN


def test_first_cycle_parameters(ctl_out):
    c = ctl_out["conv0"]
    assert ctl_out["plan0"] == 1
    assert c["act"] == 1 and c["cont"] == 0 and c["first"] == 1
    assert c["is"] == 1.0 / 2.0
    tol_rel = 1e-10 * 2.0 / 2.0
    assert c["stop_rho"] == max(1e-2 ** 2, tol_rel ** 2)
    assert c["k_max"] == 1000


def test_converging_cycles_continue_the_direction(ctl_out):
    s_prev, s = 2.0, 2.0
    for k in range(1, 7):
        s_prev, s = s, s * 1e-2
        c = ctl_out[f"conv{k}"]
        assert c["cycles"] == k and c["total"] == 30 * k and c["l"] == k
        assert c["s"] == s and c["best"] == s and c["stagnant"] == 0
        if k < 6:
            # the recurrence predicted s exactly (s = s_prev * sqrt(rho_k)): continue
            assert ctl_out[f"plan{k}"] == 1
            assert c["first"] == 0 and c["cont"] == 1
            assert math.isclose(c["b0"], s / (s_prev * 1e-4), rel_tol=1e-15)
            assert math.isclose(c["is"], 1.0 / s, rel_tol=1e-15)
            want = max(1e-4, (1e-10 * 2.0 / s) ** 2)
            assert math.isclose(c["stop_rho"], want, rel_tol=1e-15)
        else:
            # s = 2e-12 <= tol ||eta|| = 2e-10: converged, nothing to run
            assert ctl_out[f"plan{k}"] == 0
            assert c["done"] == 1 and c["status"] == LQ_OK and c["act"] == 0 and c["cont"] == 0


def test_drift_restarts_afresh(ctl_out):
    c = ctl_out["drift"]
    # s_new = 0.1 > 2 * 1.0 * sqrt(1e-4) = 0.02: the next cycle starts from p_0 = r_0
    assert c["first"] == 1 and c["cont"] == 0 and c["b0"] == 0.0 and c["act"] == 1


def test_stagnation_stops_after_five_cycles(ctl_out):
    plans = [ctl_out[f"stag{k}"] for k in range(1, 7)]
    assert plans == [1, 1, 1, 1, 0, 0]
    c = ctl_out["stag"]
    assert c["status"] == LQ_NOT_CONVERGED and c["done"] == 1 and c["stagnant"] >= 5


def test_cycle_and_iteration_caps(ctl_out):
    # two cycles allowed: after the second one the solve stops unconverged
    assert ctl_out["plan_maxcyc"] == 0
    assert ctl_out["maxcyc"]["status"] == LQ_NOT_CONVERGED and ctl_out["maxcyc"]["l"] == 2
    # a total cap of 50 iterations: the next cycle may take what is left of it
    assert ctl_out["iters0"]["k_max"] == 50
    assert ctl_out["iters1"]["total"] == 45 and ctl_out["iters1"]["k_max"] == 5
    assert ctl_out["plan_iters2"] == 0
    assert ctl_out["iters2"]["status"] == LQ_NOT_CONVERGED and ctl_out["iters2"]["done"] == 1


def test_breakdown_and_nonfinite(ctl_out):
    b = ctl_out["brk"]
    assert ctl_out["plan_brk"] == 0
    assert b["status"] == LQ_ERR_BREAKDOWN and b["done"] == 1 and b["xact"] == 0
    assert b["total"] == 7 and b["cycles"] == 0
    n = ctl_out["nan"]
    assert ctl_out["plan_nan"] == 0
    assert n["status"] == LQ_ERR_NONFINITE and n["done"] == 1
