"""Pins of the oracle's reverse mode (oracle/nadmm_oracle_grad.py) against
things other than itself: central finite differences of the FP64 forward
functions (step 1e-6, so the truncation error is ~1e-12 relative), the
adjoint (dot-product) identity for the linear operators, and a closed form
for one ADMM iteration.  Grids are tiny and inputs smooth and generic, so no
finite-difference step crosses a kink of the piecewise-smooth operators."""
import math

import numpy as np
import pytest
from scipy.ndimage import gaussian_filter

import oracle as O

EPS = 1e-6


def fd(f, x, d):
    return (f(x + EPS * d) - f(x - EPS * d)) / (2.0 * EPS)


def close(a, b, rel=1e-6, abs_=1e-9):
    assert abs(a - b) <= rel * max(abs(a), abs(b)) + abs_, (a, b)


@pytest.fixture
def rng():
    return np.random.default_rng(1234)


def smooth_image(rng, shape, sigma=1.0):
    f = gaussian_filter(rng.random(shape), sigma)
    return (f - f.min()) / (f.max() - f.min())


# ---------------------------------------------------------------- grid ops
def test_trilinear_vjp_values_and_positions(rng):
    nz, ny, nx = 4, 5, 6
    f = rng.random((nz, ny, nx))
    # points inside and outside the clamp range (outside: zero gradient)
    px = rng.uniform(-0.7, nx - 0.3, (3, 7))
    py = rng.uniform(-0.7, ny - 0.3, (3, 7))
    pz = rng.uniform(-0.7, nz - 0.3, (3, 7))
    g = rng.standard_normal(px.shape)
    gf, gx, gy, gz = O.trilinear_vjp(f, px, py, pz, g)
    d = rng.standard_normal(f.shape)
    close(fd(lambda q: (O.trilinear(q, px, py, pz) * g).sum(), f, d), (gf * d).sum())
    dp = rng.standard_normal(px.shape)
    close(fd(lambda q: (O.trilinear(f, q, py, pz) * g).sum(), px, dp), (gx * dp).sum())
    close(fd(lambda q: (O.trilinear(f, px, q, pz) * g).sum(), py, dp), (gy * dp).sum())
    close(fd(lambda q: (O.trilinear(f, px, py, q) * g).sum(), pz, dp), (gz * dp).sum())
    outside = (px < 0) | (px > nx - 1)
    assert outside.any() and np.all(gx[outside] == 0)


def test_central_gradient_vjp_is_the_adjoint(rng):
    f = rng.standard_normal((5, 4, 6))
    g = rng.standard_normal((3, 5, 4, 6))
    lhs = (O.central_gradient(f) * g).sum()
    rhs = (f * O.central_gradient_vjp(g)).sum()
    close(lhs, rhs, rel=1e-12)
    # by hand on a 1D profile along x: f = [a, b, c, d], clamped differences
    # D = [(b-a)/2, (c-a)/2, (d-b)/2, (d-c)/2]; adjoint of g = e_0 along x
    g1 = np.zeros((3, 1, 1, 4))
    g1[0, 0, 0, 0] = 1.0
    np.testing.assert_allclose(O.central_gradient_vjp(g1)[0, 0], [-0.5, 0.5, 0.0, 0.0])
    g1[0, 0, 0, 0] = 0.0
    g1[0, 0, 0, 3] = 1.0
    np.testing.assert_allclose(O.central_gradient_vjp(g1)[0, 0], [0.0, 0.0, -0.5, 0.5])


def test_warp_and_linearise_vjp(rng):
    shape = (5, 6, 7)
    I0, I1 = smooth_image(rng, shape), smooth_image(rng, shape)
    u = 0.8 * rng.standard_normal((3,) + shape)
    gJ = rng.standard_normal((3,) + shape)
    gc = rng.standard_normal(shape)
    gI0, gI1, gu = O.linearise_vjp(I0, I1, u, gJ, gc)

    def obj(a, b, v):
        J, c, _ = O.linearise(a, b, v)
        return (J * gJ).sum() + (c * gc).sum()
    d = rng.standard_normal(shape)
    close(fd(lambda q: obj(q, I1, u), I0, d), (gI0 * d).sum())
    close(fd(lambda q: obj(I0, q, u), I1, d), (gI1 * d).sum())
    du = rng.standard_normal(u.shape)
    close(fd(lambda q: obj(I0, I1, q), u, du), (gu * du).sum())


def test_compose_vjp(rng):
    shape = (4, 5, 6)
    u = 0.7 * rng.standard_normal((3,) + shape)
    v = 0.6 * rng.standard_normal((3,) + shape)
    g = rng.standard_normal((3,) + shape)
    gu, gv = O.compose_vjp(u, v, g)
    du = rng.standard_normal(u.shape)
    close(fd(lambda q: (O.compose(q, v) * g).sum(), u, du), (gu * du).sum())
    close(fd(lambda q: (O.compose(u, q) * g).sum(), v, du), (gv * du).sum())


@pytest.mark.parametrize("kappa,delta,branch", [(0.05, math.inf, "jac"), (math.inf, 0.05, "abs"),
                                                (100.0, 100.0, "one")])
def test_bound_scale_vjp(rng, kappa, delta, branch):
    w = rng.standard_normal((3, 4, 5, 6))
    s, m_abs, m_jac = O.bound_scale(w, kappa, delta)
    expect = {"jac": kappa / m_jac, "abs": delta / m_abs, "one": 1.0}[branch]
    assert s == expect
    gw = O.bound_scale_vjp(w, kappa, delta, 1.7)
    d = rng.standard_normal(w.shape)
    close(fd(lambda q: 1.7 * O.bound_scale(q, kappa, delta)[0], w, d), (gw * d).sum(),
          abs_=1e-10)
    if branch == "one":
        assert not gw.any()


@pytest.mark.parametrize("kappa,delta", [(0.01, math.inf), (math.inf, 0.01)])
def test_bound_scale_vjp_shares_ties(kappa, delta):
    """Reading R16 at a tie: a field mirror-symmetric in x attains its maximum
    Jacobian row sum (and its maximum |w|) at mirrored voxels.  Scaling w by
    (1 + t) moves every tied entry alike, so the derivative of s along w is
    -s whatever the shares, and the shares must add up to the whole gradient."""
    nx = 8
    x = np.arange(nx, dtype=np.float64)
    g = np.exp(-0.5 * ((x - (nx - 1) / 2.0) / 1.5) ** 2)   # g[i] == g[nx - 1 - i]
    w = np.zeros((3, 3, 4, nx))
    w[0] = g[None, None, :]
    s, m_abs, m_jac = O.bound_scale(w, kappa, delta)
    assert s < 1.0
    gw = O.bound_scale_vjp(w, kappa, delta, 1.0)
    assert np.count_nonzero(gw) >= 2                        # several entries share it
    close((gw * w).sum(), -s, rel=1e-12)


# ---------------------------------------------------------------- Eq. 5 / 6
def test_spectral_solve_is_symmetric_and_dgamma(rng):
    a = rng.standard_normal((3, 4, 6, 5))
    b = rng.standard_normal((3, 4, 6, 5))
    lam, theta, n = 3.0, 0.4, 2
    close((O.spectral_solve(a, lam, theta, n) * b).sum(),
          (a * O.spectral_solve(b, lam, theta, n)).sum(), rel=1e-12)
    # d/dgamma with gamma = lam / theta, by finite differences in lambda
    dS = O.spectral_solve_dgamma(a, lam, theta, n)
    num = fd(lambda q: (O.spectral_solve(a, q, theta, n) * b).sum(), lam, 1.0)
    close(num, (dS * b).sum() / theta)


@pytest.mark.parametrize("n,K,acc", [(1, 4, True), (2, 5, True), (3, 3, False), (2, 1, True)])
def test_admm_vjp(rng, n, K, acc):
    shape = (4, 5, 6)
    J = 0.5 * rng.standard_normal((3,) + shape)
    c = 0.3 * rng.standard_normal(shape)
    gw = rng.standard_normal((3,) + shape)
    lam, theta = 2.0, 0.5
    gJ, gc, gl, gt = O.admm_vjp(J, c, lam, theta, n, K, gw, accelerate=acc)

    def f(J_=J, c_=c, lam_=lam, th_=theta):
        return (O.admm(J_, c_, lam_, th_, n, K, accelerate=acc) * gw).sum()
    dJ = rng.standard_normal(J.shape)
    dc = rng.standard_normal(c.shape)
    close(fd(lambda q: f(J_=q), J, dJ), (gJ * dJ).sum())
    close(fd(lambda q: f(c_=q), c, dc), (gc * dc).sum())
    close(fd(lambda q: f(lam_=q), lam, 1.0), gl)
    close(fd(lambda q: f(th_=q), theta, 1.0), gt)


def test_admm_vjp_one_iteration_closed_form(rng):
    """K = 1 from w_hat = b_hat = 0: v = -c J / d, w = S v, so
    d<gw, w>/dc = -(J . S gw) / d with d = theta + |J|^2."""
    shape = (4, 4, 6)
    J = rng.standard_normal((3,) + shape)
    c = rng.standard_normal(shape)
    gw = rng.standard_normal((3,) + shape)
    lam, theta, n = 1.5, 0.3, 1
    _, gc, _, _ = O.admm_vjp(J, c, lam, theta, n, 1, gw)
    d = theta + (J * J).sum(axis=0)
    expect = -(J * O.spectral_solve(gw, lam, theta, n)).sum(axis=0) / d
    np.testing.assert_allclose(gc, expect, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- outer loop
@pytest.mark.parametrize("kappa,delta", [(0.5, 1.0), (0.02, math.inf), (math.inf, 0.05)])
def test_register_vjp(rng, kappa, delta):
    shape = (5, 6, 7)
    I0, I1 = smooth_image(rng, shape), smooth_image(rng, shape)
    kw = dict(lam=1.0, theta=0.5, n=1, outer=3, inner=3, kappa=kappa, delta=delta)
    u, tape = O.register_tape(I0, I1, **kw)
    if kappa < 1 and math.isinf(delta) or delta < 1:
        assert all(t[4] < 1.0 for t in tape)  # the bound is active at every step
    gu = rng.standard_normal(u.shape)
    g0, g1, gl, gt = O.register_vjp(I0, I1, gu, **kw)

    def f(a=I0, b=I1, **o):
        k = dict(kw)
        k.update(o)
        return (O.register_tape(a, b, **k)[0] * gu).sum()
    d = rng.standard_normal(shape)
    close(fd(lambda q: f(a=q), I0, d), (g0 * d).sum())
    close(fd(lambda q: f(b=q), I1, d), (g1 * d).sum())
    close(fd(lambda q: f(lam=q), 1.0, 1.0), gl)
    close(fd(lambda q: f(theta=q), 0.5, 1.0), gt)


def test_ssd_after_warp_vjp(rng):
    shape = (4, 5, 6)
    I0, I1 = smooth_image(rng, shape), smooth_image(rng, shape)
    u = 0.9 * rng.standard_normal((3,) + shape)
    gL = 0.7  # the incoming gradient of the loss scales every output
    g0, g1, gu = O.ssd_after_warp_vjp(I0, I1, u, gL)
    d = rng.standard_normal(shape)
    close(fd(lambda q: gL * O.ssd_after_warp(q, I1, u), I0, d), (g0 * d).sum())
    close(fd(lambda q: gL * O.ssd_after_warp(I0, q, u), I1, d), (g1 * d).sum())
    du = rng.standard_normal(u.shape)
    close(fd(lambda q: gL * O.ssd_after_warp(I0, I1, q), u, du), (gu * du).sum())


def test_loss_and_gradients_chain(rng):
    shape = (6, 6, 8)
    I0, I1 = smooth_image(rng, shape, 1.3), smooth_image(rng, shape, 1.3)
    kw = dict(lam=2.0, theta=0.3, n=2, outer=2, inner=4)
    L, g0, g1, gl, gt = O.loss_and_gradients(I0, I1, **kw)

    def f(a=I0, b=I1, **o):
        k = dict(kw)
        k.update(o)
        return O.ssd_after_warp(a, b, O.register(a, b, **k))
    close(L, f())
    d = rng.standard_normal(shape)
    close(fd(lambda q: f(a=q), I0, d), (g0 * d).sum())
    close(fd(lambda q: f(b=q), I1, d), (g1 * d).sum())
    close(fd(lambda q: f(lam=q), 2.0, 1.0), gl)
    close(fd(lambda q: f(theta=q), 0.3, 1.0), gt)
