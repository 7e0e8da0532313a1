"""Uneven lattices solved together (lq_cg_solve_lattices): every solve against the oracle,
graph replay against one-by-one launches, the batch against per-lattice solves, the
block-size tuner and its cache, and the full-size uneven workload."""
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import formats as F
from fieldio import to_dev, to_host

pytestmark = pytest.mark.gpu

RESID_SLACK = 1.001


def _problems(specs, seed, kind="near_identity", eps=0.5, x0=None):
    """specs: (dims, nrhs, m_q) per lattice -> (host fields, problem dicts for the binding)."""
    host, probs = [], []
    for i, (dims, nrhs, m) in enumerate(specs):
        U = synth.gauge_field(dims, seed=seed + 100 * i, kind=kind, eps=eps)
        etas = [synth.gaussian_spinor(dims, seed=seed + 100 * i + 1 + r) for r in range(nrhs)]
        host.append((dims, m, U, etas))
        p = {"dims": dims, "m_q": m, "nrhs": nrhs, "U": to_dev(F.encode_gauge(U, dims)),
             "eta": to_dev(F.encode_spinor_multi(etas, dims, "f64", "lex"))}
        if x0 is not None and x0[i] is not None:
            p["x"] = to_dev(F.encode_spinor_multi(x0[i], dims, "f64", "lex"))
        probs.append(p)
    return host, probs


def _true_resid(dims, m, U, eta, x):
    r = eta - oracle.normal_op(dims, m, U, x)
    return np.linalg.norm(r.ravel()) / np.linalg.norm(eta.ravel())


def _solutions(host, xs):
    return [F.decode_spinor_multi(to_host(x), h[0], len(h[3]), "f64", "lex") for h, x in zip(host, xs)]


SMALL = [((4, 4, 4, 4), 2, 0.1), ((6, 4, 2, 4), 4, 0.2), ((2, 4, 4, 6), 1, 0.05)]


@pytest.mark.parametrize("mode", ["mixed_f32", "mixed_f16", "f64x", "f64"])
def test_lattices_against_oracle(lqlib, mode):
    host, probs = _problems(SMALL, seed=900)
    xs, infos, st = lqlib.cg_solve_lattices(probs, mode=mode, tol=1e-10)
    assert st == 0
    for (dims, m, U, etas), sol, inf in zip(host, _solutions(host, xs), infos):
        for r in range(len(etas)):
            assert inf[r]["status"] == 0 and inf[r]["true_rel_resid"] <= 1e-10
            assert inf[r]["block"] == 128
            assert _true_resid(dims, m, U, etas[r], sol[r]) <= 1e-10 * RESID_SLACK


@pytest.mark.parametrize("mode", ["mixed_f32", "mixed_f16"])
@pytest.mark.parametrize("own_cycles", [False, True])
def test_lattices_graph_replay_equals_direct_launches(lqlib, mode, own_cycles):
    """The device-driven solve (by default one graph for the whole batch, its rounds of cycles
    and their decisions on the device; with own_cycles a conditional graph that returns when
    one lattice's inner loop has stopped; the lattices have different masses, so their cycles
    end at different iterations) runs exactly the kernels a direct launch sequence issues."""
    host, probs = _problems(SMALL, seed=910)
    xa, ia, sa = lqlib.cg_solve_lattices(probs, mode=mode, tol=1e-10, graph=True, own_cycles=own_cycles)
    xb, ib, sb = lqlib.cg_solve_lattices(probs, mode=mode, tol=1e-10, graph=False, own_cycles=own_cycles)
    assert sa == sb == 0
    for a, b in zip(xa, xb):
        assert np.array_equal(to_host(a), to_host(b))
    for la, lb in zip(ia, ib):
        assert [r["iters"] for r in la] == [r["iters"] for r in lb]


@pytest.mark.parametrize("graph", [True, False])
def test_lattices_agree_with_separate_solves(lqlib, graph):
    """Every lattice of a batch runs its own kernels with the grids of a solve of that lattice
    alone (128 threads per block, the single solves' size), so the batch gives each lattice
    the bits, iterations and cycles of its own multi-right-hand-side solve."""
    host, probs = _problems(SMALL, seed=920)
    xs, infos, st = lqlib.cg_solve_lattices(probs, mode="mixed_f32", tol=1e-10, block=128, graph=graph)
    assert st == 0
    for (dims, m, U, etas), p, x, inf in zip(host, probs, xs, infos):
        x1, i1, s1 = lqlib.cg_solve_multi(dims, m, len(etas), p["U"], p["eta"], mode="mixed_f32", tol=1e-10)
        assert s1 == 0
        assert np.array_equal(to_host(x), to_host(x1))
        assert [r["iters"] for r in inf] == [r["iters"] for r in i1]
        assert [r["cycles"] for r in inf] == [r["cycles"] for r in i1]


def test_lattices_uneven_progress(lqlib):
    """A lattice whose right-hand sides are zero, one that starts at its solution, and one
    that runs; each keeps its own outcome while the others go on."""
    specs = [((4, 4, 2, 4), 2, 0.1), ((4, 4, 4, 4), 1, 0.1), ((6, 4, 4, 2), 4, 0.1)]
    host, _ = _problems(specs, seed=930)
    zeros = [np.zeros_like(e) for e in host[0][3]]
    xsol, _, _ = oracle.cg(host[1][0], 0.1, host[1][2], host[1][3][0], tol=1e-13)
    host[0] = (host[0][0], host[0][1], host[0][2], zeros)
    _, probs = _problems(specs, seed=930, x0=[None, [xsol], None])
    probs[0]["eta"] = to_dev(F.encode_spinor_multi(zeros, specs[0][0], "f64", "lex"))
    xs, infos, st = lqlib.cg_solve_lattices(probs, mode="mixed_f32", tol=1e-10)
    assert st == 0
    sols = _solutions(host, xs)
    assert all(np.all(s == 0) for s in sols[0]) and all(i["status"] == 0 for i in infos[0])
    assert infos[1][0]["iters"] == 0
    assert all(i["iters"] > 0 for i in infos[2])
    dims, m, U, etas = host[2]
    for r in range(4):
        assert _true_resid(dims, m, U, etas[r], sols[2][r]) <= 1e-10 * RESID_SLACK
    # an iteration cap stops the running lattice
    xs, infos, st = lqlib.cg_solve_lattices(probs[2:], mode="mixed_f32", tol=1e-10, max_iter=3)
    assert st == 1 and all(i["status"] == 1 for i in infos[0])


def test_lattices_autotune_and_cache(lqlib, tmp_path):
    path = tmp_path / "tune.jsonl"
    os.environ["LQ_TUNE_CACHE"] = str(path)
    try:
        host, probs = _problems(SMALL, seed=940)
        xs, infos, st = lqlib.cg_solve_lattices(probs, mode="mixed_f16", tol=1e-10, autotune=True)
        assert st == 0
        block = infos[0][0]["block"]
        assert block in (64, 128, 256) and all(i["block"] == block for li in infos for i in li)
        lines = path.read_text().splitlines()
        assert len(lines) == 1 and lines[0].startswith('{"block": %d, "key": {' % block)
        assert '"lattices":[[4,4,4,4,2],[6,4,2,4,4],[2,4,4,6,1]]' in lines[0]
        # the second call finds the key and does not tune again
        xs2, infos2, st2 = lqlib.cg_solve_lattices(probs, mode="mixed_f16", tol=1e-10, autotune=True)
        assert st2 == 0 and infos2[0][0]["block"] == block
        assert len(path.read_text().splitlines()) == 1
        for (dims, m, U, etas), sol in zip(host, _solutions(host, xs2)):
            for r in range(len(etas)):
                assert _true_resid(dims, m, U, etas[r], sol[r]) <= 1e-10 * RESID_SLACK
    finally:
        del os.environ["LQ_TUNE_CACHE"]


@pytest.mark.parametrize("mode", ["mixed_f32", "f64x"])
@pytest.mark.parametrize("block", [64, 128, 256])
def test_lattices_every_block_size(lqlib, mode, block):
    """Each block size the tuner may pick, forced by flag, solves correctly and is reported."""
    host, probs = _problems(SMALL, seed=950)
    xs, infos, st = lqlib.cg_solve_lattices(probs, mode=mode, tol=1e-10, block=block)
    assert st == 0
    assert all(i["block"] == block for li in infos for i in li)
    for (dims, m, U, etas), sol in zip(host, _solutions(host, xs)):
        for r in range(len(etas)):
            assert _true_resid(dims, m, U, etas[r], sol[r]) <= 1e-10 * RESID_SLACK


def test_lattices_full_size_uneven_workload(lqlib):
    """The uneven batch at full size: 8^4, 12^4 and 16^3 x 32, four right-hand sides each,
    Haar links, m_q = 0.1, FP32 inner loop, FP32-pair outer loop, tolerance 1e-10, block size
    tuned; residuals recomputed by the oracle for the first and the last right-hand side of
    every lattice."""
    specs = [((8, 8, 8, 8), 4, 0.1), ((12, 12, 12, 12), 4, 0.1), ((16, 16, 16, 32), 4, 0.1)]
    host, probs = _problems(specs, seed=960, kind="haar")
    xs, infos, st = lqlib.cg_solve_lattices(probs, mode="mixed_f32", tol=1e-10, autotune=True)
    assert st == 0
    for (dims, m, U, etas), sol, inf in zip(host, _solutions(host, xs), infos):
        assert all(i["status"] == 0 and i["true_rel_resid"] <= 1e-10 for i in inf)
        for r in (0, 3):
            assert _true_resid(dims, m, U, etas[r], sol[r]) <= 1e-10 * RESID_SLACK


@pytest.mark.parametrize("mode", ["mixed_f32", "mixed_f16", "f64"])
def test_lattices_cycles_together_equal_cycles_apart(lqlib, mode):
    """Taking the reliable updates of all lattices together (a lattice whose inner loop has
    stopped waits, its blocks idle, until the others' have) changes no lattice's sequence of
    operations: the solutions are the same bits as with each lattice's own cycles."""
    host, probs = _problems(SMALL, seed=930)
    xa, ia, sa = lqlib.cg_solve_lattices(probs, mode=mode, tol=1e-10)
    xb, ib, sb = lqlib.cg_solve_lattices(probs, mode=mode, tol=1e-10, own_cycles=True)
    assert sa == sb == 0
    for a, b in zip(xa, xb):
        assert np.array_equal(to_host(a), to_host(b))
    for la, lb in zip(ia, ib):
        assert [(r["iters"], r["cycles"]) for r in la] == [(r["iters"], r["cycles"]) for r in lb]
