"""The large-volume workload at full size: 64^3 x 128 (33.5 M sites), Haar links, four
right-hand sides in one batched solve, m_q = 0.02, FP32 inner loop on 12-real links,
FP32-pair outer loop, tolerance 1e-10.

Checks: the solver's own FP64-class residual; the whole-lattice residual recomputed with
the FP64 LEX apply kernels (checked against the oracle elsewhere); and, at sampled sites, the
residual eta - D^dag D x recomputed by the oracle from the host copies of U, eta and x.
Host memory stays near 40 GB: the right-hand sides are drawn, uploaded and checked one at
a time."""
import gc

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

DIMS = (64, 64, 64, 128)
M_Q = 0.02
NRHS = 4
TOL = 1e-10


def _neighbourhood(dims, sites):
    """The sites and their eight nearest neighbours (periodic), lexicographic."""
    L = np.array(dims, dtype=np.int64)
    S = np.array([1, L[0], L[0] * L[1], L[0] * L[1] * L[2]], dtype=np.int64)
    c = np.stack([(sites // S[mu]) % L[mu] for mu in range(4)], axis=1)
    out = [sites]
    for mu in range(4):
        for step in (1, -1):
            cc = c.copy()
            cc[:, mu] = (cc[:, mu] + step) % L[mu]
            out.append(cc @ S)
    return np.unique(np.concatenate(out))


def _normal_op_at(dims, m, U, x, sites):
    """(D^dag D x)(n) at the given sites: D x on the sites and their neighbours, then D^dag."""
    nb = _neighbourhood(dims, sites)
    y = np.zeros_like(x)
    y[nb] = oracle.dslash_sites(dims, m, U, x, nb, dagger=False)
    out = oracle.dslash_sites(dims, m, U, y, sites, dagger=True)
    del y
    return out


def _host_available_gb():
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 1e6
    return 0.0


def test_cg_large_volume_64x64x64x128_four_rhs(lqlib):
    import torch
    torch.cuda.empty_cache()
    # the workload needs ~255 GB of device memory and ~40 GB of host memory
    if torch.cuda.mem_get_info()[0] < 262e9:
        pytest.skip(f"needs 262 GB free device memory, {torch.cuda.mem_get_info()[0] / 1e9:.0f} GB free")
    if _host_available_gb() < 64:
        pytest.skip(f"needs 64 GB of available host memory, {_host_available_gb():.0f} GB available")
    V = int(np.prod(DIMS))
    sb = lqlib.field_bytes(DIMS, "spinor", "f64")
    U = synth.gauge_field(DIMS, seed=70, kind="haar")
    U_d = torch.from_numpy(U.view(np.uint8).reshape(-1)).cuda()
    eta_d = torch.empty(NRHS * sb, dtype=torch.uint8, device="cuda")
    sites = np.sort(synth.make_rng(71).choice(V, size=256, replace=False))
    eta_at = []
    for r in range(NRHS):
        e = synth.gaussian_spinor(DIMS, seed=72 + r)
        eta_d[r * sb:(r + 1) * sb].copy_(torch.from_numpy(e.view(np.uint8).reshape(-1)))
        eta_at.append(e[sites].copy())
        del e
    gc.collect()

    x_d, infos, st = lqlib.cg_solve_multi(DIMS, M_Q, NRHS, U_d, eta_d, mode="mixed_f32", tol=TOL)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    assert st == 0
    for i in infos:
        assert i["status"] == 0 and i["true_rel_resid"] <= TOL and i["iters"] > 0

    for r in range(NRHS):
        xr = x_d[r * sb:(r + 1) * sb]
        er = eta_d[r * sb:(r + 1) * sb]
        # whole lattice: r = eta - D^dag D x with the FP64 LEX apply kernels
        t = lqlib.dslash_apply(DIMS, M_Q, U_d, xr)
        q = lqlib.dslash_adjoint(DIMS, M_Q, U_d, t)
        ev = er.view(torch.float64)
        res = torch.linalg.vector_norm(ev - q.view(torch.float64)) / torch.linalg.vector_norm(ev)
        del t, q
        assert float(res) <= TOL * 1.001
        # sampled sites: the oracle from the host copies
        x = xr.cpu().numpy().view(np.complex128).reshape(V, 4, 3)
        got = _normal_op_at(DIMS, M_Q, U, x, sites)
        loc = np.linalg.norm((eta_at[r] - got).ravel()) / np.linalg.norm(eta_at[r].ravel())
        assert loc <= 3 * TOL, loc
        del x
        gc.collect()
