"""Run the library's entry points on small and ragged lattices with the bounds-checked debug
build (LQ_LIB_VARIANT=checked) and require that no kernel touched a slot outside its field.

Not a test module: tests/test_gpu_bounds.py runs it in a child process, so that the checked
library is the only one that process loads.  Each operation's result is also compared with
the CPU oracle (a skipped access would read zero and show up there too).  Prints one line per
group and "bounds suite ok: <n> operations" at the end; exits non-zero on the first failure.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle                       # noqa: E402
import synth                        # noqa: E402
from oracle import formats as F     # noqa: E402
from fieldio import to_dev, to_host  # noqa: E402
import paper_1904_08616_gb300 as lq  # noqa: E402

TOL = {"f64": 1e-13, "f64x": 1e-13, "f32": 1e-6, "f16s": 1e-3, "i32s": 1e-6}
LATTICES = [(2, 2, 2, 2), (6, 4, 10, 2), (4, 4, 4, 4)]
count = 0


def clean(what):
    global count
    n, first = lq.bounds_violations()
    if n != 0:
        raise SystemExit(f"{what}: {n} out-of-range accesses, first slot {first}")
    count += 1


def main():
    assert lq.checked(), "run with LQ_LIB_VARIANT=checked"
    lq.load()
    n0, _ = lq.bounds_violations()
    assert n0 == 0, "the checked library reports the normal build"
    m = 0.1
    # operator and adjoint, every stored format and layout
    for dims in LATTICES:
        U = synth.gauge_field(dims, seed=1)
        psi = synth.gaussian_spinor(dims, seed=2)
        for prec in ("f64", "f64x", "f32", "f16s", "i32s"):
            for fmt in ((18,) if prec == "f64x" else (18, 12, 10)):
                for layout in ("lex", "eo"):
                    Ub = F.encode_gauge(U, dims, prec, fmt, layout)
                    pb = F.encode_spinor(psi, dims, prec, layout)
                    for dag in (False, True):
                        fn = lq.dslash_adjoint if dag else lq.dslash_apply
                        out = fn(dims, m, to_dev(Ub), to_dev(pb), prec=prec, link_fmt=fmt, layout=layout)
                        got = F.decode_spinor(to_host(out), dims, prec, layout)
                        want = oracle.dslash(dims, m, F.decode_gauge(Ub, dims, prec, fmt, layout),
                                             F.decode_spinor(pb, dims, prec, layout), dagger=dag)
                        err = oracle.rel_l2(got, want)
                        assert err <= TOL[prec], (dims, prec, fmt, layout, dag, err)
                        clean(f"apply {dims} {prec}/{fmt}/{layout} dagger={dag}")
                    if layout == "eo" and dims != (2, 2, 2, 2):
                        # the parity hop onto the even sites from the odd half of psi
                        full = F.encode_spinor(psi, dims, prec, "eo")
                        from fieldio import eo_half
                        odd = eo_half(full, dims, prec, 1)
                        lq.dslash_hop(dims, 0, to_dev(Ub), to_dev(odd), prec=prec, link_fmt=fmt)
                        clean(f"hop {dims} {prec}/{fmt}")
    print(f"operators: {count} calls clean", flush=True)
    # several fields at once (EO interleaved)
    dims = (6, 4, 10, 2)
    U = synth.gauge_field(dims, seed=3)
    for prec in ("f32", "f16s"):
        for nr in (2, 4):
            psis = [synth.gaussian_spinor(dims, seed=10 + i) for i in range(nr)]
            Ub = F.encode_gauge(U, dims, prec, 12, "eo")
            pb = F.encode_spinor_multi(psis, dims, prec, "eo")
            out = lq.dslash_apply_multi(dims, m, nr, to_dev(Ub), to_dev(pb), prec=prec, link_fmt=12, layout="eo")
            got = F.decode_spinor_multi(to_host(out), dims, nr, prec, "eo")
            Ud = F.decode_gauge(Ub, dims, prec, 12, "eo")
            for i in range(nr):
                want = oracle.dslash(dims, m, Ud, F.decode_spinor_multi(pb, dims, nr, prec, "eo")[i])
                assert oracle.rel_l2(got[i], want) <= TOL[prec]
            clean(f"apply_multi {prec} nr={nr}")
    # solvers: every mode, single and several right-hand sides, register blocking, Schur,
    # lattice batches, 10-real inner links, and the no-allocation entry
    for dims, kind in (((2, 2, 2, 2), "haar"), ((6, 4, 10, 2), "near_identity")):
        U = synth.gauge_field(dims, seed=5, kind=kind, eps=0.3)
        Ud = to_dev(F.encode_gauge(U, dims))
        for nr in (1, 3, 4):
            etas = [synth.gaussian_spinor(dims, seed=20 + i) for i in range(nr)]
            ed = to_dev(F.encode_spinor_multi(etas, dims, "f64", "lex"))
            for mode in ("f64", "f64x", "mixed_f32", "mixed_f16", "mixed_i32"):
                for rb in ((1, 2, 4) if nr == 4 and mode.startswith("mixed") else (None,)):
                    x, infos, st = lq.cg_solve_multi(dims, m, nr, Ud, ed, mode=mode, tol=1e-10, rhs_block=rb)
                    assert st == 0, (dims, nr, mode, rb, st)
                    xs = F.decode_spinor_multi(to_host(x), dims, nr, "f64", "lex")
                    for i in range(nr):
                        r = etas[i] - oracle.normal_op(dims, m, U, xs[i])
                        assert np.linalg.norm(r) / np.linalg.norm(etas[i]) <= 1.001e-10
                    clean(f"cg_solve_multi {dims} nr={nr} {mode} rb={rb}")
        e1 = to_dev(F.encode_spinor(synth.gaussian_spinor(dims, seed=30), dims))
        for mode in ("mixed_f32", "mixed_f16"):
            _, _, st = lq.cg_solve(dims, m, Ud, e1, mode=mode, tol=1e-10, link10=True)
            assert st == 0
            clean(f"cg_solve {dims} {mode} link10")
        for mode in ("f64x", "mixed_f32", "mixed_f16", "mixed_i32"):
            _, _, st = lq.cg_solve_schur(dims, m, Ud, e1, mode=mode, tol=1e-10)
            assert st == 0
            clean(f"cg_solve_schur {dims} {mode}")
    probs = []
    for i, (dims, nr) in enumerate((((2, 2, 2, 2), 2), ((6, 4, 10, 2), 4), ((4, 4, 4, 4), 1))):
        U = synth.gauge_field(dims, seed=40 + i)
        etas = [synth.gaussian_spinor(dims, seed=50 + 10 * i + j) for j in range(nr)]
        probs.append({"dims": dims, "m_q": m, "nrhs": nr, "U": to_dev(F.encode_gauge(U, dims)),
                      "eta": to_dev(F.encode_spinor_multi(etas, dims, "f64", "lex"))})
    for mode in ("f64", "f64x", "mixed_f32", "mixed_f16"):
        _, _, st = lq.cg_solve_lattices(probs, mode=mode, tol=1e-10)
        assert st == 0
        clean(f"cg_solve_lattices {mode}")
    print(f"solvers: {count} calls clean", flush=True)
    # conversions, the domain-decomposed operator, the link gradient
    dims = (6, 4, 10, 2)
    U = synth.gauge_field(dims, seed=60)
    psi = synth.gaussian_spinor(dims, seed=61)
    Ud, pd = to_dev(F.encode_gauge(U, dims)), to_dev(F.encode_spinor(psi, dims))
    for prec in ("f32", "f16s", "f64x", "i32s"):
        for layout in ("lex", "eo"):
            lq.convert_spinor(dims, pd, "f64", "lex", dst_prec=prec, dst_layout=layout)
            for fmt in ((18,) if prec == "f64x" else (18, 12, 10)):
                lq.convert_gauge(dims, Ud, "f64", "lex", dst_prec=prec, dst_fmt=fmt, dst_layout=layout)
            clean(f"convert {prec} {layout}")
    g = lq.link_grad(dims, pd, pd)
    clean("link_grad")
    from paper_1904_08616_gb300 import halo
    out = halo.VirtualRanks(dims, 2).apply(m, Ud, pd)
    want = oracle.dslash(dims, m, U, psi)
    assert oracle.rel_l2(F.decode_spinor(to_host(out), dims), want) <= 1e-13
    clean("halo dslash")
    del g
    print(f"bounds suite ok: {count} operations", flush=True)


if __name__ == "__main__":
    main()
