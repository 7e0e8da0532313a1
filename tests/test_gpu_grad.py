"""Link gradients and the autograd functions against the oracle and against finite
differences of the library's own forward passes."""
import numpy as np
import pytest

import oracle
import synth
from fieldio import to_dev, to_host

pytestmark = pytest.mark.gpu

LATTICES = [(2, 2, 2, 2), (4, 6, 2, 4), (6, 4, 10, 2)]


def _cdev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _links_host(buf, dims):
    return to_host(buf).view(np.complex128).reshape(int(np.prod(dims)), 4, 3, 3)


@pytest.mark.parametrize("dims", LATTICES)
def test_link_grad_matches_oracle(lqlib, dims):
    g = synth.gaussian_spinor(dims, seed=701)
    psi = synth.gaussian_spinor(dims, seed=702)
    got = _links_host(lqlib.link_grad(dims, to_dev(g), to_dev(psi)), dims)
    want = oracle.link_grad(dims, g, psi)
    assert oracle.rel_l2(got, want) <= 1e-14


def test_link_grad_scale_and_accumulate(lqlib):
    dims = (4, 4, 2, 4)
    g = synth.gaussian_spinor(dims, seed=711)
    psi = synth.gaussian_spinor(dims, seed=712)
    prev = synth.gauge_field(dims, seed=713)
    out = to_dev(prev)
    lqlib.link_grad(dims, to_dev(g), to_dev(psi), out=out, scale=-2.5, accumulate=True)
    want = prev - 2.5 * oracle.link_grad(dims, g, psi)
    assert oracle.rel_l2(_links_host(out, dims), want) <= 1e-14
    lqlib.link_grad(dims, to_dev(g), to_dev(psi), out=out, scale=0.5)
    assert oracle.rel_l2(_links_host(out, dims), 0.5 * oracle.link_grad(dims, g, psi)) <= 1e-14


def test_link_grad_bad_args(lqlib):
    dims = (4, 4, 4, 4)
    f = to_dev(synth.gaussian_spinor(dims, seed=1))
    with pytest.raises(lqlib.LqError):
        lqlib.link_grad((4, 4, 3, 4), f, f)
    out = lqlib.link_grad(dims, f, f)
    with pytest.raises(lqlib.LqError):
        lqlib.link_grad(dims, out, f, out=out)       # out overlaps g
    with pytest.raises(lqlib.LqError):
        lqlib.link_grad(dims, f, f, scale=float("nan"))
    c = _cdev(synth.gaussian_spinor(dims, seed=2))
    with pytest.raises(ValueError):
        lqlib.link_grad(dims, c.conj(), c)           # a lazy view's memory is not its value


@pytest.mark.parametrize("dagger", [False, True])
def test_dirac_apply_backward_matches_oracle(lqlib, dagger):
    import torch
    from paper_1904_08616_gb300.autograd import dirac_apply
    dims = (4, 6, 2, 4)
    m = 0.1
    U = synth.gauge_field(dims, seed=721)
    psi = synth.gaussian_spinor(dims, seed=722)
    g = synth.gaussian_spinor(dims, seed=723)
    Ut = _cdev(U).requires_grad_()
    pt = _cdev(psi).requires_grad_()
    out = dirac_apply(dims, m, Ut, pt, dagger=dagger)
    assert oracle.rel_l2(out.detach().cpu().numpy(), oracle.dslash(dims, m, U, psi, dagger=dagger)) <= 1e-14
    loss = (out.conj() * _cdev(g)).real.sum()      # Re <out, g> = Re <g, out>
    loss.backward()
    want_psi = oracle.dslash(dims, m, U, g, dagger=not dagger)
    want_U = oracle.link_grad(dims, psi, g) if dagger else oracle.link_grad(dims, g, psi)
    assert oracle.rel_l2(pt.grad.cpu().numpy(), want_psi) <= 1e-14
    assert oracle.rel_l2(Ut.grad.cpu().numpy(), want_U) <= 1e-14
    assert torch.isfinite(loss)


@pytest.mark.parametrize("dagger", [False, True])
def test_dirac_apply_gradcheck(lqlib, dagger):
    """torch.autograd.gradcheck: the analytic vector-Jacobian products against the numerical
    Jacobian of the library's forward kernel (D is linear in each argument, so central
    differences are exact up to rounding)."""
    import torch
    from paper_1904_08616_gb300.autograd import dirac_apply
    dims = (2, 2, 2, 2)
    U = _cdev(synth.gauge_field(dims, seed=731)).requires_grad_()
    psi = _cdev(synth.gaussian_spinor(dims, seed=732)).requires_grad_()
    assert torch.autograd.gradcheck(lambda a, b: dirac_apply(dims, 0.3, a, b, dagger=dagger), (U, psi),
                                    eps=1e-6, atol=1e-8, rtol=1e-6, fast_mode=True)


@pytest.mark.parametrize("mode,tol", [("f64", 1e-12), ("mixed_f32", 1e-12), ("f64x", 1e-12)])
def test_dirac_solve_backward_matches_oracle(lqlib, mode, tol):
    from paper_1904_08616_gb300.autograd import dirac_solve
    dims = (4, 4, 4, 4)
    m = 0.1
    U = synth.gauge_field(dims, seed=741, kind="near_identity", eps=0.5)
    eta = synth.gaussian_spinor(dims, seed=742)
    chi = synth.gaussian_spinor(dims, seed=743)
    Ut = _cdev(U).requires_grad_()
    et = _cdev(eta).requires_grad_()
    x = dirac_solve(dims, m, Ut, et, mode=mode, tol=tol)
    (x.conj() * _cdev(chi)).real.sum().backward()
    want_eta, want_U = oracle.solve_grads(dims, m, U, eta, chi, tol=1e-13)
    assert oracle.rel_l2(et.grad.cpu().numpy(), want_eta) <= 1e-9
    assert oracle.rel_l2(Ut.grad.cpu().numpy(), want_U) <= 1e-9


def test_dirac_solve_finite_differences_16x16x16x16(lqlib):
    """Directional derivatives of L = Re <chi, (D^dag D)^{-1} eta> at 16^4 (exp(0.5 i H)
    links, m = 0.1): the adjoint gradient against central differences of the library's own
    FP64 solves, along random directions in the links and in eta."""
    import torch
    from paper_1904_08616_gb300.autograd import dirac_solve
    dims = (16, 16, 16, 16)
    m = 0.1
    tol = 1e-13
    U = synth.gauge_field(dims, seed=751, kind="near_identity", eps=0.5)
    eta = synth.gaussian_spinor(dims, seed=752)
    chi_t = _cdev(synth.gaussian_spinor(dims, seed=753))
    Ut = _cdev(U).requires_grad_()
    et = _cdev(eta).requires_grad_()
    x = dirac_solve(dims, m, Ut, et, mode="f64", tol=tol)
    (x.conj() * chi_t).real.sum().backward()
    gU, ge = Ut.grad.detach(), et.grad.detach()

    def loss(Uv, ev):
        with torch.no_grad():
            xv = dirac_solve(dims, m, Uv, ev, mode="f64", tol=tol)
            return float((xv.conj() * chi_t).real.sum())

    h = 1e-4
    rng = synth.make_rng(754)
    for k in range(3):
        dU = _cdev(rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape))
        fd = (loss(Ut.detach() + h * dU, et.detach()) - loss(Ut.detach() - h * dU, et.detach())) / (2 * h)
        an = float((gU.conj() * dU).real.sum())     # dL = Re <grad, dU> in the dL/dRe + i dL/dIm convention
        assert abs(fd - an) <= 1e-6 * abs(an), (k, fd, an)
    for k in range(2):
        de = _cdev(rng.standard_normal(eta.shape) + 1j * rng.standard_normal(eta.shape))
        fd = (loss(Ut.detach(), et.detach() + h * de) - loss(Ut.detach(), et.detach() - h * de)) / (2 * h)
        an = float((ge.conj() * de).real.sum())
        assert abs(fd - an) <= 1e-6 * abs(an), (k, fd, an)


def test_dirac_solve_mixed_gradient_matches_fp64(lqlib):
    """At 16^4 the gradient through Algorithm 1 (FP32 inner loop) agrees with the one through
    FP64 CG to the solve tolerance."""
    from paper_1904_08616_gb300.autograd import dirac_solve
    dims = (16, 16, 16, 16)
    m = 0.1
    U = synth.gauge_field(dims, seed=761, kind="near_identity", eps=0.5)
    eta = synth.gaussian_spinor(dims, seed=762)
    chi_t = _cdev(synth.gaussian_spinor(dims, seed=763))
    grads = {}
    for mode in ("f64", "mixed_f32"):
        Ut = _cdev(U).requires_grad_()
        et = _cdev(eta).requires_grad_()
        x = dirac_solve(dims, m, Ut, et, mode=mode, tol=1e-12)
        (x.conj() * chi_t).real.sum().backward()
        grads[mode] = (Ut.grad.cpu().numpy(), et.grad.cpu().numpy())
    assert oracle.rel_l2(grads["mixed_f32"][0], grads["f64"][0]) <= 1e-9
    assert oracle.rel_l2(grads["mixed_f32"][1], grads["f64"][1]) <= 1e-9


def test_dirac_solve_fd_64_link_entries_step_1e6(lqlib):
    """The differentiation workload as stated: 16^4, FP64 links exp(0.5 i H), m = 0.1,
    L = Re <chi, (D^dag D)^{-1} eta>; central differences with step 1e-6 on the real and the
    imaginary part of 64 random link entries, FP64 CG solves to 1e-13, against the adjoint
    gradient; relative L2 error over the 128 derivatives <= 1e-6."""
    import torch
    from paper_1904_08616_gb300.autograd import dirac_solve
    dims = (16, 16, 16, 16)
    m = 0.1
    tol = 1e-13
    U = synth.gauge_field(dims, seed=771, kind="near_identity", eps=0.5)
    eta_t = _cdev(synth.gaussian_spinor(dims, seed=772))
    chi_t = _cdev(synth.gaussian_spinor(dims, seed=773))
    Ut = _cdev(U).requires_grad_()
    x = dirac_solve(dims, m, Ut, eta_t, mode="f64", tol=tol)
    (x.conj() * chi_t).real.sum().backward()
    grad = Ut.grad.detach().cpu().numpy().reshape(-1)
    U0 = Ut.detach().reshape(-1)

    def loss(Uflat):
        with torch.no_grad():
            xv = dirac_solve(dims, m, Uflat.reshape(U.shape), eta_t, mode="f64", tol=tol)
            return float((xv.conj() * chi_t).real.sum())

    h = 1e-6
    idx = synth.make_rng(774).choice(U.size, size=64, replace=False)
    fd, an = [], []
    for i in idx:
        for unit, part in ((1.0, "re"), (1j, "im")):
            Up = U0.clone()
            Um = U0.clone()
            Up[int(i)] += h * unit
            Um[int(i)] -= h * unit
            fd.append((loss(Up) - loss(Um)) / (2 * h))
            an.append(grad[i].real if part == "re" else grad[i].imag)
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(fd - an) <= 1e-6 * np.linalg.norm(an), (np.abs(fd - an).max(), np.linalg.norm(an))
