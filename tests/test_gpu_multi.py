"""Several right-hand sides at once: batched operator applies, multi-field conversions and
batched CG solves, against the oracle and against the single-field paths."""
import numpy as np
import pytest

import oracle
import synth
from oracle import formats as F
from fieldio import to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f64x": 1e-13, "f32": 1e-6, "f16s": 1e-3, "i32s": 1e-6}
RESID_SLACK = 1.001


@pytest.mark.parametrize("prec,fmt", [("f64", 18), ("f32", 12), ("f16s", 12), ("f64x", 18), ("i32s", 12)])
@pytest.mark.parametrize("layout,nrhs", [("eo", 2), ("eo", 4), ("eo", 8), ("lex", 3), ("lex", 5)])
@pytest.mark.parametrize("dagger", [False, True])
def test_multi_apply_matches_oracle(lqlib, prec, fmt, layout, nrhs, dagger):
    dims = (4, 6, 2, 4)
    m = 0.1
    U = synth.gauge_field(dims, seed=41)
    psis = [synth.gaussian_spinor(dims, seed=100 + i) for i in range(nrhs)]
    Ub = F.encode_gauge(U, dims, prec, fmt, layout)
    Ud = F.decode_gauge(Ub, dims, prec, fmt, layout)
    pb = F.encode_spinor_multi(psis, dims, prec, layout)
    fn = lqlib.dslash_adjoint_multi if dagger else lqlib.dslash_apply_multi
    out = fn(dims, m, nrhs, to_dev(Ub), to_dev(pb), prec=prec, link_fmt=fmt, layout=layout)
    got = F.decode_spinor_multi(to_host(out), dims, nrhs, prec, layout)
    decoded = F.decode_spinor_multi(pb, dims, nrhs, prec, layout)
    for i in range(nrhs):
        want = oracle.dslash(dims, m, Ud, decoded[i], dagger=dagger)
        assert oracle.rel_l2(got[i], want) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f32", "f64x", "f64"])
def test_multi_apply_equals_single_applies(lqlib, prec):
    """The batched kernel does the single-field arithmetic for every field: bit-identical."""
    dims = (8, 4, 4, 4)
    nrhs = 4
    U = synth.gauge_field(dims, seed=42)
    psis = [synth.gaussian_spinor(dims, seed=200 + i) for i in range(nrhs)]
    Ub = to_dev(F.encode_gauge(U, dims, prec, 18, "eo"))
    multi = lqlib.dslash_apply_multi(dims, 0.2, nrhs, Ub, to_dev(F.encode_spinor_multi(psis, dims, prec, "eo")),
                                     prec=prec, layout="eo")
    got = F.decode_spinor_multi(to_host(multi), dims, nrhs, prec, "eo")
    for i in range(nrhs):
        single = lqlib.dslash_apply(dims, 0.2, Ub, to_dev(F.encode_spinor(psis[i], dims, prec, "eo")),
                                    prec=prec, layout="eo")
        assert np.array_equal(got[i], F.decode_spinor(to_host(single), dims, prec, "eo"))


@pytest.mark.parametrize("prec", ["f32", "f16s", "f64x", "i32s"])
@pytest.mark.parametrize("nrhs", [2, 4])
def test_multi_convert_bit_exact(lqlib, prec, nrhs):
    dims = (4, 4, 2, 6)
    psis = [synth.gaussian_spinor(dims, seed=300 + i) for i in range(nrhs)]
    src = to_dev(F.encode_spinor_multi(psis, dims, "f64", "lex"))
    dst = lqlib.convert_spinor_multi(dims, nrhs, src, "f64", "lex", dst_prec=prec, dst_layout="eo")
    assert np.array_equal(to_host(dst), F.encode_spinor_multi(psis, dims, prec, "eo"))
    back = lqlib.convert_spinor_multi(dims, nrhs, dst, prec, "eo", dst_prec=prec, dst_layout="lex")
    assert np.array_equal(to_host(back), F.encode_spinor_multi(
        F.decode_spinor_multi(to_host(dst), dims, nrhs, prec, "eo"), dims, prec, "lex"))


def _solve_multi(lqlib, dims, m, U, etas, mode, x0s=None, **kw):
    n = len(etas)
    Ud = to_dev(F.encode_gauge(U, dims))
    ed = to_dev(F.encode_spinor_multi(etas, dims, "f64", "lex"))
    x0s = x0s if x0s is not None else [np.zeros_like(e) for e in etas]
    xd = to_dev(F.encode_spinor_multi(x0s, dims, "f64", "lex"))
    x, infos, st = lqlib.cg_solve_multi(dims, m, n, Ud, ed, x=xd, mode=mode, **kw)
    return F.decode_spinor_multi(to_host(x), dims, n, "f64", "lex"), infos, st


def _true_resid(dims, m, U, eta, x):
    r = eta - oracle.normal_op(dims, m, U, x)
    return np.linalg.norm(r.ravel()) / np.linalg.norm(eta.ravel())


@pytest.mark.parametrize("mode", ["mixed_f32", "mixed_f16", "f64x", "f64", "mixed_i32"])
@pytest.mark.parametrize("nrhs", [1, 3, 4, 12])
def test_cg_multi_against_oracle(lqlib, mode, nrhs):
    """nrhs = 3 runs as batches 2 + 1, 12 as 8 + 4; every solve meets the tolerance and
    agrees with the single-right-hand-side solver."""
    dims = (4, 4, 4, 4)
    m = 0.1
    U = synth.gauge_field(dims, seed=51, kind="near_identity", eps=0.5)
    etas = [synth.gaussian_spinor(dims, seed=400 + i) for i in range(nrhs)]
    xs, infos, st = _solve_multi(lqlib, dims, m, U, etas, mode, tol=1e-10)
    assert st == 0
    for i in range(nrhs):
        assert infos[i]["status"] == 0 and infos[i]["true_rel_resid"] <= 1e-10
        assert _true_resid(dims, m, U, etas[i], xs[i]) <= 1e-10 * RESID_SLACK
    Ud = to_dev(F.encode_gauge(U, dims))
    for i in (0, nrhs - 1):
        x1, info1, st1 = lqlib.cg_solve(dims, m, Ud, to_dev(F.encode_spinor(etas[i], dims)), mode=mode, tol=1e-10)
        assert oracle.rel_l2(xs[i], F.decode_spinor(to_host(x1), dims)) <= 1e-7


def test_cg_multi_uneven_right_hand_sides(lqlib, rhs_block=None):
    """Within one batch: a zero right-hand side, one that starts at its solution, one that
    hits the iteration cap, and a regular one; each gets its own status."""
    dims = (4, 4, 2, 4)
    m = 0.05
    U = synth.gauge_field(dims, seed=61, kind="near_identity", eps=0.3)
    e0 = synth.gaussian_spinor(dims, seed=62)
    e1 = np.zeros_like(e0)
    e2 = synth.gaussian_spinor(dims, seed=63)
    e3 = synth.gaussian_spinor(dims, seed=64)
    xsol, _, _ = oracle.cg(dims, m, U, e2, tol=1e-13)
    xs, infos, st = _solve_multi(lqlib, dims, m, U, [e0, e1, e2, e3], "mixed_f32",
                                 x0s=[np.zeros_like(e0), synth.gaussian_spinor(dims, seed=65), xsol,
                                      np.zeros_like(e0)], tol=1e-10, rhs_block=rhs_block)
    assert st == 0
    assert infos[1]["status"] == 0 and np.all(xs[1] == 0)
    assert infos[2]["iters"] == 0 and infos[2]["status"] == 0
    assert infos[0]["iters"] > 0 and infos[3]["iters"] > 0
    for i in (0, 2, 3):
        assert _true_resid(dims, m, U, [e0, e1, e2, e3][i], xs[i]) <= 1e-10 * RESID_SLACK
    # an iteration cap that stops every right-hand side early
    xs, infos, st = _solve_multi(lqlib, dims, m, U, [e0, e2], "mixed_f32", tol=1e-10, max_iter=4,
                                 rhs_block=rhs_block)
    assert st == 1 and all(i["status"] == 1 for i in infos)


@pytest.mark.parametrize("rhs_block", [2, 4])
def test_cg_multi_uneven_right_hand_sides_blocked(lqlib, rhs_block):
    """The same mixed batch with two or four right-hand sides per thread: stopped and idle
    right-hand sides inside one thread's group are skipped while the others go on."""
    test_cg_multi_uneven_right_hand_sides(lqlib, rhs_block=rhs_block)


@pytest.mark.parametrize("mode", ["mixed_f32", "mixed_f16", "mixed_i32"])
@pytest.mark.parametrize("nrhs", [4, 8, 12])
@pytest.mark.parametrize("rhs_block", [1, 2, 4])
def test_cg_multi_register_blocking(lqlib, mode, nrhs, rhs_block):
    """Each blocking factor (right-hand sides per thread in the inner stencil kernels) on a
    lattice with a ragged last tile: every solve meets the tolerance in the oracle's FP64
    residual and agrees with the single-right-hand-side solver; the arithmetic per right-hand
    side is the same, so the iteration counts match those of one thread per right-hand side
    up to the order of the grid reductions."""
    dims = (6, 4, 10, 2)
    m = 0.05
    U = synth.gauge_field(dims, seed=71, kind="near_identity", eps=0.3)
    etas = [synth.gaussian_spinor(dims, seed=700 + i) for i in range(nrhs)]
    xs, infos, st = _solve_multi(lqlib, dims, m, U, etas, mode, tol=1e-10, rhs_block=rhs_block)
    assert st == 0
    assert all(i["rhs_block"] == rhs_block for i in infos)
    _, infos1, _ = _solve_multi(lqlib, dims, m, U, etas, mode, tol=1e-10, rhs_block=1)
    Ud = to_dev(F.encode_gauge(U, dims))
    for i in range(nrhs):
        assert infos[i]["status"] == 0
        assert _true_resid(dims, m, U, etas[i], xs[i]) <= 1e-10 * RESID_SLACK
        assert abs(infos[i]["iters"] - infos1[i]["iters"]) <= 2
    for i in (0, nrhs - 1):
        x1, _, _ = lqlib.cg_solve(dims, m, Ud, to_dev(F.encode_spinor(etas[i], dims)), mode=mode, tol=1e-10)
        assert oracle.rel_l2(xs[i], F.decode_spinor(to_host(x1), dims)) <= 1e-7


@pytest.mark.parametrize("mode", ["mixed_f32", "mixed_f16"])
def test_cg_multi_autotuned_rhs_block(lqlib, mode, tmp_path, monkeypatch):
    """LQ_CG_AUTOTUNE without a blocking flag: the library times the two inner stencil kernels
    with 1, 2 and 4 right-hand sides per thread and keeps the fastest. The choice is reported in every
    info record and appended to the tuning cache file, and the solve gives the same bits and
    counts as a solve with that choice fixed; a batch of one is not tuned."""
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("LQ_TUNE_CACHE", str(cache))
    dims = (8, 6, 4, 6)
    m = 0.05
    U = synth.gauge_field(dims, seed=72, kind="near_identity", eps=0.3)
    etas = [synth.gaussian_spinor(dims, seed=720 + i) for i in range(8)]
    xs, infos, st = _solve_multi(lqlib, dims, m, U, etas, mode, tol=1e-10, autotune=True)
    assert st == 0
    rb = infos[0]["rhs_block"]
    assert rb in (1, 2, 4) and all(i["rhs_block"] == rb for i in infos)
    lines = [ln for ln in cache.read_text().splitlines() if '"what":"rhs_block"' in ln]
    assert len(lines) == 1 and lines[0].startswith('{"block": %d, "key": ' % rb)
    assert '"dims":[8,6,4,6],"nrhs":8' in lines[0]
    xf, infof, stf = _solve_multi(lqlib, dims, m, U, etas, mode, tol=1e-10, rhs_block=rb)
    assert stf == 0 and np.array_equal(xs, xf)
    assert [i["iters"] for i in infos] == [i["iters"] for i in infof]
    for i in (0, 7):
        assert _true_resid(dims, m, U, etas[i], xs[i]) <= 1e-10 * RESID_SLACK
    # a second tuned solve takes the cached choice: nothing more is appended
    _, infos2, _ = _solve_multi(lqlib, dims, m, U, etas, mode, tol=1e-10, autotune=True)
    assert infos2[0]["rhs_block"] == rb
    assert len([ln for ln in cache.read_text().splitlines() if '"what":"rhs_block"' in ln]) == 1
    _, info1, _ = _solve_multi(lqlib, dims, m, U, etas[:1], mode, tol=1e-10, autotune=True)
    assert info1[0]["rhs_block"] == 1


def test_cg_multi_full_size_24x24x24x48(lqlib):
    """The batched workload at full size: 24^3 x 48, Haar links, 12 right-hand sides, FP32
    inner loop, FP64-class outer loop, tolerance 1e-10; residuals recomputed by the oracle for
    two of them."""
    dims = (24, 24, 24, 48)
    m = 0.1
    U = synth.gauge_field(dims, seed=5)
    etas = [synth.gaussian_spinor(dims, seed=500 + i) for i in range(12)]
    xs, infos, st = _solve_multi(lqlib, dims, m, U, etas, "mixed_f32", tol=1e-10)
    assert st == 0
    assert all(i["true_rel_resid"] <= 1e-10 for i in infos)
    for i in (0, 11):
        assert _true_resid(dims, m, U, etas[i], xs[i]) <= 1e-10 * RESID_SLACK


def test_cg_multi_device_loop_equals_host_loop(lqlib):
    """A batch whose right-hand sides stop at different iterations and cycles: the solve run
    on the device (one CUDA graph) and the host-driven one give the same bits and counts."""
    dims = (4, 4, 2, 4)
    m = 0.05
    U = synth.gauge_field(dims, seed=66, kind="near_identity", eps=0.3)
    etas = [synth.gaussian_spinor(dims, seed=67 + i) for i in range(3)]
    etas[1] *= 1e-3
    for mode in ("f64x", "mixed_f16"):
        xg, ig, sg = _solve_multi(lqlib, dims, m, U, etas, mode, tol=1e-10)
        xh, ih, sh = _solve_multi(lqlib, dims, m, U, etas, mode, tol=1e-10, graph=False)
        assert sg == sh == 0
        assert [i["iters"] for i in ig] == [i["iters"] for i in ih]
        assert np.array_equal(xg, xh)
