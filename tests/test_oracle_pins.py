"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, a dense direct solve built here from the stencil, brute-force
minimisation, exact invariants, and special cases that reduce to textbook
problems.  None of them calls the CUDA path.
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import oracle as O
from paper_2109_12688_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ------------------------------------------------------------ helpers (test-only)
def dense_periodic_laplacian(dims):
    """(-Delta_h) as a dense matrix on a periodic grid, unknown index
    z*ny*nx + y*nx + x, built from the 7-point stencil by explicit loops."""
    nx, ny, nz = dims
    V = nx * ny * nz
    A = np.zeros((V, V))

    def idx(x, y, z):
        return ((z % nz) * ny + (y % ny)) * nx + (x % nx)

    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = idx(x, y, z)
                A[i, i] += 6.0
                for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    A[i, idx(x + d[0], y + d[1], z + d[2])] -= 1.0
    return A


def dense_l2_minimiser_here(J, c, lam, n):
    """(J J^T + lambda L^n) v = -J c assembled from this file's stencil."""
    shape = c.shape
    V = c.size
    L = np.linalg.matrix_power(dense_periodic_laplacian(shape[::-1]), n)
    Jf = J.reshape(3, V).astype(np.float64)
    A = np.kron(np.eye(3), lam * L)
    for i in range(3):
        for j in range(3):
            A[i * V:(i + 1) * V, j * V:(j + 1) * V] += np.diag(Jf[i] * Jf[j])
    rhs = -(Jf * c.reshape(1, V)).ravel()
    return np.linalg.solve(A, rhs).reshape((3,) + shape)


# ------------------------------------------------------------ Eq. 5 scalars
def test_nesterov_sequence_closed_forms():
    alpha, beta = O.nesterov_sequence(40)
    assert alpha[0] == 1.0
    assert beta[0] == 0.0                                   # beta_0 = (alpha^0 - 1)/alpha^1
    assert alpha[1] == pytest.approx((1 + math.sqrt(5)) / 2, abs=1e-15)   # golden ratio
    # alpha^2 = (1 + sqrt(1 + 4 phi^2)) / 2 with phi^2 = phi + 1
    assert alpha[2] == pytest.approx((1 + math.sqrt(1 + 4 * (alpha[1] + 1))) / 2, abs=1e-14)
    for k in range(40):
        # the recurrence is the positive root of a^2 - a - alpha_k^2 = 0
        assert alpha[k + 1] ** 2 - alpha[k + 1] == pytest.approx(alpha[k] ** 2, rel=1e-13)
        assert alpha[k] >= (k + 2) / 2.0 - 1e-12              # standard growth bound
        assert 0.0 <= beta[k] < 1.0
        assert beta[k] == pytest.approx((alpha[k] - 1) / alpha[k + 1], rel=1e-15)
    assert beta[1] == pytest.approx((alpha[1] - 1) / alpha[2], rel=1e-15)
    assert beta[1] == pytest.approx(0.2817535251, abs=1e-9)


# ------------------------------------------------------------ Eq. 6 v-step
def test_data_step_l2_is_the_3x3_solve_and_kkt():
    rng = np.random.default_rng(11)
    theta = 0.07
    u = rng.normal(size=(3, 50, 1, 1))
    J = rng.normal(size=(3, 50, 1, 1))
    c = rng.normal(size=(50, 1, 1))
    v = O.data_step_l2(u, J, c, theta)
    for i in range(50):
        Ji = J[:, i, 0, 0]
        A = np.outer(Ji, Ji) + theta * np.eye(3)           # Eq. 6 middle line
        rhs = theta * u[:, i, 0, 0] - Ji * c[i, 0, 0]
        np.testing.assert_allclose(v[:, i, 0, 0], np.linalg.solve(A, rhs), rtol=1e-11, atol=1e-12)
    rho = (J * v).sum(0) + c
    kkt = J * rho[None] + theta * (v - u)
    assert np.abs(kkt).max() < 1e-12


def test_data_step_l1_matches_brute_force():
    rng = np.random.default_rng(12)
    theta = 0.1
    for _ in range(40):
        u = rng.normal(size=3)
        Jv = rng.normal(size=3) * rng.uniform(0.05, 2.0)
        c = rng.normal() * rng.uniform(0.01, 3.0)
        v = O.data_step_l1(u.reshape(3, 1, 1, 1), Jv.reshape(3, 1, 1, 1),
                           np.array(c).reshape(1, 1, 1), theta, eps=1e-15)[:, 0, 0, 0]

        def f(vv):
            return abs(Jv @ vv + c) + 0.5 * theta * ((vv - u) ** 2).sum()

        # components orthogonal to J only feel the quadratic, so the minimiser
        # is u + tau J; minimise over tau by bounded scalar search
        g = lambda t: f(u + t * Jv)  # noqa: E731
        span = 2.0 / theta                     # |tau| <= 1/theta at the minimiser
        res = minimize_scalar(g, bounds=(-span, span), method="bounded",
                              options={"xatol": 1e-13, "maxiter": 5000})
        grid = np.linspace(res.x - 1e-3, res.x + 1e-3, 20001)
        t_best = grid[np.argmin([g(t) for t in grid])]
        v_bf = u + t_best * Jv
        assert f(v) <= f(v_bf) + 1e-9
        np.testing.assert_allclose(v, v_bf, atol=2e-6 * max(1.0, np.abs(Jv).max()))
        for _ in range(10):
            assert f(v) <= f(v + rng.normal(size=3) * 1e-3) + 1e-12


# ------------------------------------------------------------ Eq. 6 w-step
@pytest.mark.parametrize("dims", [(4, 4, 4), (4, 6, 3), (5, 3, 7)])
@pytest.mark.parametrize("n", [1, 2, 3])
def test_spectral_solve_equals_dense_solve(dims, n):
    lam, theta = 2.5, 0.3
    nx, ny, nz = dims
    y = synth.random_field((3, nz, ny, nx), seed=5).astype(np.float64)
    L = np.linalg.matrix_power(dense_periodic_laplacian(dims), n)
    A = lam * L + theta * np.eye(nx * ny * nz)
    w_fft = O.spectral_solve(y, lam, theta, n)
    for i in range(3):
        w_dense = np.linalg.solve(A, theta * y[i].ravel()).reshape(y[i].shape)
        np.testing.assert_allclose(w_fft[i], w_dense, rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("pqr", [(1, 0, 0), (0, 2, 1), (3, 1, 2), (4, 5, 3)])
def test_spectral_solve_single_mode(pqr):
    dims = (8, 12, 6)
    nx, ny, nz = dims
    p, q, r = pqr
    lam, theta, n = 4.0, 0.2, 2
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mode = np.cos(2 * np.pi * (p * x / nx + q * y / ny + r * z / nz))
    K = (4 * np.sin(np.pi * p / nx) ** 2 + 4 * np.sin(np.pi * q / ny) ** 2
         + 4 * np.sin(np.pi * r / nz) ** 2)
    gain = 1.0 / (1.0 + (lam / theta) * K ** n)
    w = O.spectral_solve(np.stack([mode, 2 * mode, -mode]), lam, theta, n)
    np.testing.assert_allclose(w[0], gain * mode, atol=1e-12)
    np.testing.assert_allclose(w[1], 2 * gain * mode, atol=1e-12)
    np.testing.assert_allclose(w[2], -gain * mode, atol=1e-12)


def test_spectral_solve_keeps_constants():
    y = np.ones((3, 6, 4, 8)) * np.array([0.3, -1.2, 2.0])[:, None, None, None]
    np.testing.assert_allclose(O.spectral_solve(y, 50.0, 0.01, 3), y, atol=1e-13)


def test_symbol_matches_sin_squared_form():
    dims = (6, 10, 4)
    for n in (1, 2, 3):
        K = O.laplacian_symbol(dims, n)
        z, y, x = np.meshgrid(np.arange(4), np.arange(10), np.arange(6), indexing="ij")
        ref = (4 * np.sin(np.pi * x / 6) ** 2 + 4 * np.sin(np.pi * y / 10) ** 2
               + 4 * np.sin(np.pi * z / 4) ** 2) ** n
        np.testing.assert_allclose(K, ref, atol=1e-12)


# ------------------------------------------------------------ Eq. 5 loop
@pytest.mark.parametrize("n", [1, 2, 3])
def test_admm_reaches_dense_minimiser(n):
    dims = (4, 5, 3)
    J, c = synth.random_linearisation(dims, seed=3, grad_scale=0.3, resid_scale=0.5)
    J = J.astype(np.float64)
    c = c.astype(np.float64)
    lam = 2.0
    v_star = dense_l2_minimiser_here(J, c, lam, n)
    np.testing.assert_allclose(O.dense_minimiser_l2(J, c, lam, n), v_star, rtol=1e-10, atol=1e-12)
    scale = np.abs(v_star).max()
    # plain ADMM at two penalties, accelerated ADMM where theta >~ |J|^2
    for theta, acc in ((0.2, False), (1.0, False), (1.0, True)):
        w = O.admm(J, c, lam, theta, n, 600, accelerate=acc)
        assert np.abs(w - v_star).max() / scale < 1e-8, (theta, acc)


def test_hs_special_case_normal_equations():
    """s = 2, n = 1 is Horn-Schunck (Sec. 2): its regularised normal
    equations (J J^T - lambda Delta) v = -J c, solved densely."""
    dims = (4, 4, 4)
    J, c = synth.random_linearisation(dims, seed=21, grad_scale=0.3, resid_scale=0.5)
    J = J.astype(np.float64)
    c = c.astype(np.float64)
    lam = 1.5
    V = c.size
    Lap = dense_periodic_laplacian(dims)
    Jf = J.reshape(3, V)
    A = np.zeros((3 * V, 3 * V))
    for i in range(3):
        A[i * V:(i + 1) * V, i * V:(i + 1) * V] = lam * Lap
        for j in range(3):
            A[i * V:(i + 1) * V, j * V:(j + 1) * V] += np.diag(Jf[i] * Jf[j])
    v_hs = np.linalg.solve(A, -(Jf * c.reshape(1, V)).ravel()).reshape(J.shape)
    w = O.admm(J, c, lam, 0.5, 1, 800, s=2, accelerate=False)
    np.testing.assert_allclose(w, v_hs, atol=1e-9 * np.abs(v_hs).max())


def test_admm_fixed_point_with_dual():
    """At the minimiser v*, the scaled dual of the w-line is
    b* = (lambda/theta) L v*; one iteration of Eq. 5 leaves (v*, b*) fixed."""
    dims = (4, 4, 4)
    J, c = synth.random_linearisation(dims, seed=4, grad_scale=0.5, resid_scale=0.5)
    J = J.astype(np.float64)
    c = c.astype(np.float64)
    lam, theta, n = 3.0, 0.4, 2
    v_star = dense_l2_minimiser_here(J, c, lam, n)
    L = np.linalg.matrix_power(dense_periodic_laplacian(dims), n)
    b_star = np.stack([(lam / theta) * (L @ v_star[i].ravel()).reshape(c.shape) for i in range(3)])
    for beta in (0.0, 0.6):
        w, b, v = O.admm_step(v_star, v_star, b_star, b_star, beta, J, c, lam, theta, n)
        np.testing.assert_allclose(w, v_star, atol=1e-11)
        np.testing.assert_allclose(v, v_star, atol=1e-11)
        np.testing.assert_allclose(b, b_star, atol=1e-11)


def test_nesterov_index_on_one_voxel():
    """On a 1-voxel grid L = 0, so w = v and b = 0, and with J = (j, 0, 0)
    the x-component follows e^k = a (e^{k-1} + beta_{k-1}(e^{k-1} - e^{k-2}))
    with a = theta / (theta + j^2) and e = w - (-c/j); worked by hand here."""
    j, c0, theta = 0.8, 0.3, 0.5
    J = np.zeros((3, 1, 1, 1))
    J[0] = j
    c = np.full((1, 1, 1), c0)
    hist = O.admm(J, c, 1.0, theta, 2, 8, history=True)
    _, beta = O.nesterov_sequence(8)
    a = theta / (theta + j * j)
    u_star = -c0 / j
    e = [a * (0.0 - u_star)]                      # w_hat^0 = 0
    e.append(a * e[0])                            # beta_0 = 0
    for k in range(2, 8):
        e.append(a * (e[k - 1] + beta[k - 1] * (e[k - 1] - e[k - 2])))
    for k in range(8):
        w, b = hist[k]
        assert w[0, 0, 0, 0] - u_star == pytest.approx(e[k], abs=1e-14)
        assert abs(w[1, 0, 0, 0]) < 1e-15 and abs(b).max() < 1e-15


def test_admm_l1_reaches_low_energy():
    dims = (4, 4, 3)
    J, c = synth.random_linearisation(dims, seed=8, grad_scale=0.4, resid_scale=0.3)
    J = J.astype(np.float64)
    c = c.astype(np.float64)
    lam, n = 1.0, 1
    w = O.admm(J, c, lam, 0.3, n, 3000, s=1, eps=1e-12, accelerate=False)
    e0 = O.energy(w, J, c, lam, n, s=1)
    rng = np.random.default_rng(0)
    for _ in range(30):
        d = rng.normal(size=w.shape) * 1e-3
        assert e0 <= O.energy(w + d, J, c, lam, n, s=1) + 1e-9
    assert e0 <= O.energy(np.zeros_like(w), J, c, lam, n, s=1)


def test_energy_and_lagrangian_pins():
    dims = (4, 4, 4)
    J, c = synth.random_linearisation(dims, seed=9, grad_scale=0.5, resid_scale=0.5)
    J = J.astype(np.float64)
    c = c.astype(np.float64)
    lam, n = 2.0, 2
    assert O.energy(np.zeros_like(J), J, c, lam, n, 2) == pytest.approx(0.5 * (c ** 2).sum())
    assert O.energy(np.zeros_like(J), J, c, lam, n, 1) == pytest.approx(np.abs(c).sum())
    v = dense_l2_minimiser_here(J, c, lam, n)
    e = O.energy(v, J, c, lam, n, 2)
    rng = np.random.default_rng(1)
    for _ in range(10):
        d = rng.normal(size=v.shape) * 1e-4
        assert O.energy(v + d, J, c, lam, n, 2) >= e - 1e-12
    b = rng.normal(size=v.shape)
    assert O.augmented_lagrangian(v, v, np.zeros_like(v), J, c, lam, 0.3, n) == pytest.approx(e)
    assert O.augmented_lagrangian(v, v, b, J, c, lam, 0.3, n) == pytest.approx(e + 0.15 * (b ** 2).sum())


# ------------------------------------------------------------ grid primitives
def test_trilinear_reproduces_affine():
    nz, ny, nx = 5, 6, 7
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = 0.3 + 1.1 * x - 0.7 * y + 0.25 * z
    rng = np.random.default_rng(2)
    px = rng.uniform(0, nx - 1, 200)
    py = rng.uniform(0, ny - 1, 200)
    pz = rng.uniform(0, nz - 1, 200)
    np.testing.assert_allclose(O.trilinear(f, px, py, pz), 0.3 + 1.1 * px - 0.7 * py + 0.25 * pz,
                               atol=1e-12)
    # at grid points the samples are exact, outside the box they clamp
    np.testing.assert_allclose(O.trilinear(f, x.astype(float), y.astype(float), z.astype(float)), f)
    assert O.trilinear(f, np.array([-3.0]), np.array([2.0]), np.array([99.0]))[0] == pytest.approx(
        f[nz - 1, 2, 0])


def test_central_gradient_of_ramp():
    nz, ny, nx = 4, 5, 6
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    g = O.central_gradient(2.0 * x - 3.0 * y + 0.5 * z)
    np.testing.assert_allclose(g[0][:, :, 1:-1], 2.0)
    np.testing.assert_allclose(g[1][:, 1:-1, :], -3.0)
    np.testing.assert_allclose(g[2][1:-1], 0.5)
    # clamped index at the border: one-sided difference halved
    np.testing.assert_allclose(g[0][:, :, 0], 1.0)
    np.testing.assert_allclose(g[1][:, -1, :], -1.5)


def test_compose_constant_shifts_add():
    shape = (3, 8, 9, 10)
    u = np.zeros(shape) + np.array([0.4, -0.3, 0.2])[:, None, None, None]
    v = np.zeros(shape) + np.array([-0.7, 0.5, 0.25])[:, None, None, None]
    out = O.compose(u, v)
    np.testing.assert_allclose(out[:, 1:-1, 1:-1, 1:-1],
                               (u + v)[:, 1:-1, 1:-1, 1:-1], atol=1e-14)


def test_warp_by_integer_shift():
    rng = np.random.default_rng(3)
    I1 = rng.normal(size=(6, 7, 8))
    u = np.zeros((3, 6, 7, 8))
    u[0] = 1.0
    u[2] = -1.0
    w = O.warp(I1, u)
    np.testing.assert_allclose(w[1:, :, :-1], I1[:-1, :, 1:], atol=1e-14)


def test_bound_scale_properties():
    rng = np.random.default_rng(4)
    w = rng.normal(size=(3, 6, 7, 8)) * 2.0
    s, m_abs, m_jac = O.bound_scale(w, 0.5, 1.0)
    assert 0 < s <= 1
    _, a2, j2 = O.bound_scale(s * w, math.inf, math.inf)
    assert a2 <= 1.0 + 1e-12 and j2 <= 0.5 + 1e-12
    assert max(a2 / 1.0, j2 / 0.5) == pytest.approx(1.0)
    assert O.bound_scale(w * 1e-4, 0.5, 1.0)[0] == 1.0
    assert O.bound_scale(w, math.inf, math.inf)[0] == 1.0
    det = O.jacobian_determinant(s * w)
    assert det.min() > 0


def test_jacobian_determinant_linear_map():
    nz, ny, nx = 6, 6, 6
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    A = np.array([[0.1, 0.2, -0.1], [0.05, -0.3, 0.0], [0.2, 0.1, 0.15]])
    pos = np.stack([x, y, z]).astype(float)
    u = np.einsum("ij,j...->i...", A, pos)
    det = O.jacobian_determinant(u)
    np.testing.assert_allclose(det[1:-1, 1:-1, 1:-1], np.linalg.det(np.eye(3) + A), rtol=1e-12)
    assert np.all(O.jacobian_determinant(np.zeros((3, 4, 4, 4))) == 1.0)


# ------------------------------------------------------------ whole pipeline
def test_identical_images_give_identity():
    p = synth.make_pair((16, 12, 8), seed=1)
    u = O.register(p["fixed"], p["fixed"], 10.0, 0.1, 2, 3, 5)
    assert np.all(u == 0.0)


def test_recovers_known_translation():
    dims = (24, 20, 16)
    shift = (0.6, -0.4, 0.3)
    I0, I1 = synth.translated_blob_pair(dims, shift, sigma_frac=0.25)
    u = O.register(I0, I1, 10.0, 0.02, 1, 10, 30)
    np.testing.assert_allclose(u[:, 8, 10, 12], -np.array(shift), atol=0.01)


def test_phantom_registration_is_diffeomorphic_and_reduces_ssd():
    p = synth.make_pair((32, 32, 24), seed=0)
    u, scales = O.register(p["fixed"], p["moving"], 10.0, 0.1, 2, 5, 10, return_scales=True)
    assert O.jacobian_determinant(u).min() > 0
    ssd0 = ((p["moving"].astype(float) - p["fixed"]) ** 2).sum()
    ssd1 = ((O.warp(p["moving"], u) - p["fixed"]) ** 2).sum()
    assert ssd1 < 0.6 * ssd0
    assert all(0 < s <= 1 for s in scales)


def test_velocity_bound_is_active_when_needed():
    p = synth.make_pair((32, 32, 24), seed=2)
    u, scales = O.register(p["fixed"], p["moving"], 0.05, 0.01, 1, 3, 10, kappa=0.05,
                           delta=0.2, return_scales=True)
    assert min(scales) < 1.0
    assert O.jacobian_determinant(u).min() > 0


# ------------------------------------------------------------ pins aimed at single-term slips
def test_accelerated_admm_on_one_fourier_mode():
    """With J = (j, 0, 0) uniform and c a single cosine mode, every field of
    Eq. 5 stays a multiple of that mode, so the 3D iteration reduces to a
    scalar recurrence: v = a u + d (Sherman-Morrison with a = theta/(theta +
    j^2), d = -j C/(theta + j^2)), w = g (v + b_hat) (spectral gain g =
    1/(1 + (lambda/theta) K^n)), b = b_hat + v - w, then the Nesterov
    extrapolation of both w and b."""
    dims = (8, 6, 4)
    nx, ny, nz = dims
    p, q, r = 1, 2, 1
    lam, theta, n, j, C = 0.7, 0.9, 2, 0.6, 0.5
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mode = np.cos(2 * np.pi * (p * x / nx + q * y / ny + r * z / nz))
    J = np.zeros((3,) + mode.shape)
    J[0] = j
    c = C * mode
    K = 4 * np.sin(np.pi * p / nx) ** 2 + 4 * np.sin(np.pi * q / ny) ** 2 + 4 * np.sin(np.pi * r / nz) ** 2
    g = 1.0 / (1.0 + (lam / theta) * K ** n)
    a = theta / (theta + j * j)
    d = -j * C / (theta + j * j)
    _, beta = O.nesterov_sequence(12)
    hist = O.admm(J, c, lam, theta, n, 12, history=True)
    w_hat = b_hat = w_prev = b_prev = 0.0
    for k in range(12):
        v = a * (w_hat - b_hat) + d
        w = g * (v + b_hat)
        b = b_hat + v - w
        gw, gb = hist[k]
        np.testing.assert_allclose(gw[0], w * mode, atol=1e-13)
        np.testing.assert_allclose(gb[0], b * mode, atol=1e-13)
        assert np.abs(gw[1:]).max() < 1e-14 and np.abs(gb[1:]).max() < 1e-14
        w_hat = w + beta[k] * (w - w_prev)
        b_hat = b + beta[k] * (b - b_prev)
        w_prev, b_prev = w, b
    assert abs(b) > 1e-3          # the dual is genuinely non-zero here


def test_trilinear_hand_example_and_cell_bounds():
    nz, ny, nx = 4, 4, 6
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = (x ** 2).astype(float)
    # between x = 2 and 3 with weight 0.3: 0.7 * 4 + 0.3 * 9 = 5.5
    assert O.trilinear(f, np.array([2.3]), np.array([1.0]), np.array([2.0]))[0] == pytest.approx(5.5)
    assert O.trilinear(f, np.array([2.7]), np.array([0.5]), np.array([1.5]))[0] == pytest.approx(7.5)
    rng = np.random.default_rng(5)
    g = rng.normal(size=(nz, ny, nx))
    px, py, pz = rng.uniform(0, nx - 1, 300), rng.uniform(0, ny - 1, 300), rng.uniform(0, nz - 1, 300)
    val = O.trilinear(g, px, py, pz)
    for i in range(300):
        x0, y0, z0 = int(px[i]), int(py[i]), int(pz[i])
        cell = g[z0:z0 + 2, y0:y0 + 2, x0:x0 + 2]
        assert cell.min() - 1e-12 <= val[i] <= cell.max() + 1e-12


def test_compose_affine_fields_is_matrix_product():
    """(Id + A1) o (Id + A2) = Id + A2 + A1 + A1 A2 for linear fields, the
    order of Eq. 1: u_new(x) = v(x) + u(x + v(x))."""
    shape = (9, 10, 11)
    z, y, x = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), np.arange(shape[2]), indexing="ij")
    pos = np.stack([x, y, z]).astype(float)
    A1 = np.array([[0.02, -0.05, 0.01], [0.03, 0.01, -0.02], [0.0, 0.04, 0.02]])
    A2 = np.array([[-0.01, 0.02, 0.04], [0.05, 0.0, 0.01], [-0.03, 0.02, 0.01]])
    u = np.einsum("ij,j...->i...", A1, pos)
    v = np.einsum("ij,j...->i...", A2, pos)
    out = O.compose(u, v)
    ref = np.einsum("ij,j...->i...", A1 + A2 + A1 @ A2, pos)
    np.testing.assert_allclose(out[:, 1:-2, 1:-2, 1:-2], ref[:, 1:-2, 1:-2, 1:-2], atol=1e-12)


def test_bound_scale_uses_max_row_sum_of_jacobian():
    shape = (8, 8, 8)
    z, y, x = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    pos = np.stack([x, y, z]).astype(float) - 3.5
    A = np.array([[0.1, -0.3, 0.05], [0.2, 0.2, -0.2], [0.0, 0.1, 0.4]])
    w = np.einsum("ij,j...->i...", A, pos)
    s, m_abs, m_jac = O.bound_scale(w, 0.25, math.inf)
    assert m_jac == pytest.approx(np.linalg.norm(A, np.inf))          # 0.6
    assert m_abs == pytest.approx(np.abs(w).max())
    assert s == pytest.approx(0.25 / 0.6)


def test_outer_loop_composes_in_the_paper_order(monkeypatch):
    """Sec. 2 / Eq. 1 with N = 1: after K outer steps phi = (Id + v_1) o
    (Id + v_2) o ... o (Id + v_K).  The inner solver is replaced by prescribed
    linear velocities v_k(x) = A_k x (trilinear interpolation is exact on
    them), so the composed map must be the matrix product
    (I + s_1 A_1)(I + s_2 A_2)...(I + s_K A_K) in that order, s_k the
    velocity bound of each step."""
    from oracle import nadmm_oracle as M
    shape = (12, 13, 14)
    z, y, x = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
    pos = np.stack([x, y, z]).astype(float) - 6.0
    rng = np.random.default_rng(7)
    mats = [rng.normal(size=(3, 3)) * 0.04 for _ in range(4)]
    calls = iter(mats)
    monkeypatch.setattr(M, "admm", lambda *a, **k: np.einsum("ij,j...->i...", next(calls), pos))
    I0 = np.zeros(shape)
    for delta in (math.inf, 0.1):
        calls = iter(mats)
        u, scales = M.register(I0, I0, outer=4, inner=1, kappa=math.inf, delta=delta,
                               return_scales=True)
        P = np.eye(3)
        for A, sk in zip(mats, scales):
            P = P @ (np.eye(3) + sk * A)
        ref = np.einsum("ij,j...->i...", P - np.eye(3), pos)
        inner = (slice(None),) + (slice(4, -4),) * 3
        np.testing.assert_allclose(u[inner], ref[inner], atol=1e-12)
        if delta == 0.1:
            assert max(scales) < 1.0


# ---------------------------------------------------------------- thresholds (Sec. 4, version 2)
def test_admm_sub_steps_minimise_the_augmented_lagrangian():
    """Eq. 5 lines 1-2 minimise Eq. 4 in v (w, b fixed) and in w (v, b fixed):
    at the sub-step's output the central difference of Eq. 4 along random
    directions vanishes (it is quadratic for s = 2) and moving away raises it."""
    rng = np.random.default_rng(31)
    dims, lam, theta, n = (6, 5, 4), 3.0, 0.4, 2
    shape = (3,) + dims[::-1]
    J, c = rng.normal(size=shape), rng.normal(size=dims[::-1])
    w, b, v = rng.normal(size=shape), rng.normal(size=shape), rng.normal(size=shape)
    v_star = O.data_step_l2(w - b, J, c, theta)
    w_star = O.spectral_solve(v + b, lam, theta, n)
    h = 1e-3
    for _ in range(3):
        d = rng.normal(size=shape)
        Lv = [O.augmented_lagrangian(v_star + t * d, w, b, J, c, lam, theta, n) for t in (-h, 0.0, h)]
        Lw = [O.augmented_lagrangian(v, w_star + t * d, b, J, c, lam, theta, n) for t in (-h, 0.0, h)]
        for L in (Lv, Lw):
            assert abs(L[2] - L[0]) / (2 * h) <= 1e-6 * max(1.0, abs(L[1]))
            assert L[0] > L[1] and L[2] > L[1]


def test_register_resumes_from_u0():
    """Outer steps restart the ADMM state (reading R7), so a + b compositions
    equal b compositions started from the result of a (the first
    linearisation is taken at u0)."""
    p = synth.make_pair((16, 16, 12), seed=6)
    kw = dict(lam=10.0, theta=0.1, n=2, inner=5)
    u3 = O.register(p["fixed"], p["moving"], outer=3, **kw)
    u1 = O.register(p["fixed"], p["moving"], outer=1, **kw)
    u12 = O.register(p["fixed"], p["moving"], outer=2, u0=u1, **kw)
    np.testing.assert_array_equal(u12, u3)


def test_admm_until_stops_at_the_first_small_change():
    p = synth.make_pair((16, 16, 12), seed=2)
    J, c, _ = O.linearise(p["fixed"], p["moving"], np.zeros((3, 12, 16, 16)))
    hist = O.admm(J, c, 10.0, 0.1, 2, 30, history=True)
    rel = [np.linalg.norm(hist[k][0] - hist[k - 1][0]) / np.linalg.norm(hist[k][0])
           for k in range(1, 30)]
    tol = 0.5 * (rel[4] + rel[5]) if rel[5] < rel[4] else rel[5] * 1.0001
    k_expect = 1 + next(i for i, r in enumerate(rel) if r <= tol) + 1
    w, k = O.admm_until(J, c, 10.0, 0.1, 2, 30, tol)
    assert k == k_expect
    np.testing.assert_array_equal(w, hist[k - 1][0])
    w0, k0 = O.admm_until(J, c, 10.0, 0.1, 2, 7, 1e-30)  # never met: the cap
    assert k0 == 7 and np.array_equal(w0, hist[6][0])


def test_admm_threshold_can_stop_after_the_second_iteration():
    """The ADMM test starts at k = 1 (reading R19): a threshold just above the
    first change ||w^1 - w^0|| / ||w^1|| stops after two iterations, one just
    below it does not."""
    p = synth.make_pair((16, 16, 12), seed=2)
    J, c, _ = O.linearise(p["fixed"], p["moving"], np.zeros((3, 12, 16, 16)))
    hist = O.admm(J, c, 10.0, 0.1, 2, 12, history=True)
    r1 = np.linalg.norm(hist[1][0] - hist[0][0]) / np.linalg.norm(hist[1][0])
    _, k = O.admm_until(J, c, 10.0, 0.1, 2, 12, r1 * (1 + 1e-9))
    assert k == 2
    _, k = O.admm_until(J, c, 10.0, 0.1, 2, 12, r1 * (1 - 1e-9))
    assert k > 2


def test_warp_threshold_rule():
    """Outer stop (reading R19): after the re-warp of composition j, stop when
    ||I1w_j - I1w_{j-1}|| <= tol ||I1w_{j-1}||.  The warped images I1w_j are
    taken from threshold-free runs of j compositions; thresholds just above
    and just below each ratio give the first j whose ratio is within tol."""
    p = synth.make_pair((16, 16, 12), seed=4)
    kw = dict(lam=10.0, theta=0.1, n=2, inner=6)
    zero = np.zeros((3, 12, 16, 16))
    I1w = [O.linearise(p["fixed"], p["moving"], zero)[2]]
    for j in range(1, 4):
        u_j = O.register(p["fixed"], p["moving"], outer=j, **kw)
        I1w.append(O.linearise(p["fixed"], p["moving"], u_j)[2])
    r = [np.linalg.norm(I1w[j] - I1w[j - 1]) / np.linalg.norm(I1w[j - 1]) for j in range(1, 4)]
    for j in range(3):
        for f in (1 + 1e-9, 1 - 1e-9):
            tol = r[j] * f
            expect = next((i + 1 for i in range(3) if r[i] <= tol), 4)
            _, counts = O.register(p["fixed"], p["moving"], outer=4, warp_tol=tol,
                                   return_counts=True, **kw)
            assert len(counts) == expect, (j, f, r)


def test_register_thresholds_reduce_to_caps_and_stop_early():
    p = synth.make_pair((16, 16, 12), seed=4)
    kw = dict(lam=10.0, theta=0.1, n=2, outer=4, inner=6)
    base = O.register(p["fixed"], p["moving"], **kw)
    tiny = O.register(p["fixed"], p["moving"], admm_tol=1e-30, warp_tol=1e-30, **kw)
    np.testing.assert_array_equal(base, tiny)          # thresholds never met = caps
    u, counts = O.register(p["fixed"], p["moving"], admm_tol=0.3, warp_tol=0.5,
                           return_counts=True, **kw)
    assert all(k < 6 for k in counts) and len(counts) < 4  # both stop early
    # the outer loop stopped right after the first composition whose re-warp
    # changed the warped image by at most 50 %
    u1 = O.register(p["fixed"], p["moving"], admm_tol=0.3, outer=len(counts), inner=6,
                    lam=10.0, theta=0.1, n=2)
    np.testing.assert_array_equal(u, u1)


# ------------------------------------------------------------ adaptive restart (R20)
def _weakly_convex_case(seed=3):
    """theta << |J|^2: Eq. 5 as printed diverges here while plain ADMM
    converges (|J| = 1 at every voxel, theta = 0.05)."""
    rng = np.random.default_rng(seed)
    J = rng.normal(size=(3, 4, 4, 4))
    J /= np.sqrt((J ** 2).sum(0, keepdims=True))
    c = 0.5 * rng.normal(size=(4, 4, 4))
    return J, c, 1.0, 0.05, 1


def test_restart_extremes_are_plain_and_printed_admm():
    """eta = 0 restarts at every test: every momentum factor is 0, i.e. plain
    ADMM; eta = inf never restarts: Eq. 5 as printed (same arithmetic,
    bit-identical)."""
    rng = np.random.default_rng(21)
    J = rng.normal(scale=0.4, size=(3, 6, 5, 4))
    c = rng.normal(scale=0.3, size=(6, 5, 4))
    for n in (1, 2):
        plain = O.admm(J, c, 2.0, 0.3, n, 9, accelerate=False)
        assert np.array_equal(O.admm_restart(J, c, 2.0, 0.3, n, 9, eta=0.0), plain)
        printed = O.admm(J, c, 2.0, 0.3, n, 9)
        assert np.array_equal(O.admm_restart(J, c, 2.0, 0.3, n, 9, eta=math.inf), printed)


def test_restart_makes_the_weakly_convex_case_converge():
    J, c, lam, theta, n = _weakly_convex_case()
    ref = O.dense_minimiser_l2(J, c, lam, n)
    printed = O.admm(J, c, lam, theta, n, 300)
    assert np.abs(printed).max() > 1e6                       # Eq. 5 as printed blows up
    w = O.admm_restart(J, c, lam, theta, n, 300)
    assert np.abs(w - ref).max() < 1e-6 * np.abs(ref).max()   # restart reaches the minimiser
    plain = O.admm(J, c, lam, theta, n, 300, accelerate=False)
    assert np.abs(w - ref).max() <= np.abs(plain - ref).max()  # and no slower than plain ADMM


def test_restart_rule_against_the_iterates():
    """The recorded factors follow the rule from residuals recomputed from the
    recorded iterates: c_k = ||w^k - w_hat^k||^2 + ||b^k - b_hat^k||^2, a test
    fails when c_k >= eta cbar (cbar then divided by eta, else cbar = c_k),
    and a restart found at k zeroes the factor forming w_hat^{k+2}, after
    which the factors run beta_1, beta_2, ..."""
    J, c, lam, theta, n = _weakly_convex_case(5)
    for eta in (0.999, 0.5):
        _check_restart_rule(J, c, lam, theta, n, eta)


def _check_restart_rule(J, c, lam, theta, n, eta):
    h = O.admm_restart(J, c, lam, theta, n, 60, eta=eta, history=True)
    _, beta = O.nesterov_sequence(61)
    cbar, found = math.inf, []
    for k in range(60):
        ck = ((h["w"][k] - h["w_hat"][k]) ** 2).sum() + ((h["b"][k] - h["b_hat"][k]) ** 2).sum()
        if ck < eta * cbar:
            cbar = ck
        else:
            cbar /= eta
            found.append(k)
    assert found == h["restart"] and len(found) >= 3
    last_zero = 1
    for k in range(2, 60):
        if k - 2 in found:
            last_zero = k
        assert h["factor"][k] == (0.0 if k == last_zero else beta[k - last_zero])
        # the extrapolation really used that factor
        np.testing.assert_allclose(h["w_hat"][k], h["w"][k - 1] + h["factor"][k]
                                   * (h["w"][k - 1] - h["w"][k - 2]), rtol=0, atol=1e-12)


def test_register_with_restart_matches_printed_when_never_triggered():
    pair = synth.make_pair((16, 16, 12), seed=4)
    a = O.register(pair["fixed"], pair["moving"], n=2, outer=2, inner=6, restart_eta=math.inf)
    b = O.register(pair["fixed"], pair["moving"], n=2, outer=2, inner=6)
    assert np.array_equal(a, b)
