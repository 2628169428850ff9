"""FP64 CPU oracle for Nesterov-accelerated ADMM diffeomorphic registration.

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by ``bench.py``'s CPU-baseline / reference
arm.  The product path (the CUDA library and its Python binding) never imports
or calls it, and it shares no code, tables or helpers with that path.

It restates, plainly and slowly, what the method computes (arXiv 2109.12688):

* Sec. 2, Eq. 1 and the text after it: the greedy composition
  phi <- phi o (Id + v) with N = 1, re-warping the ORIGINAL source image each
  time and re-linearising the data term around the warped image;
* Eq. 2: the convex model (1/s)||rho(v)||^s + (lambda/2)||grad^n v||^2 with
  rho(v) = <grad I1, v> + I1 - I0;
* Eq. 4: the augmented Lagrangian;
* Eq. 5: the Nesterov-accelerated ADMM iteration (v, w, b, alpha, w_hat,
  b_hat) with w_hat^0 = b_hat^0 = 0 and alpha^0 = 1;
* Eq. 6: the closed-form v-step (s = 1 thresholding, s = 2 Sherman-Morrison)
  and the w-step solved by a division in the 3D DFT spectrum.

Readings where the paper is silent or garbled (each also listed in the design
notes of the repository):

* R1 (Eq. 6, w-step): the printed F(v+b)/(lambda F(Delta^n) + theta) lacks
  theta in the numerator; the optimality condition of Eq. 5's w-line is
  (lambda L + theta) w = theta (v + b_hat), so w = F^-1[theta F(y) /
  (lambda K^n + theta)].
* R2 (Eq. 2 vs Eq. 6): ||grad^n w||^2 is read as <w, L w> with
  L = (-Delta_h)^n, the operator whose DFT symbol the paper prints:
  K^n = 2^n (3 - cos 2pi p/M - cos 2pi q/N - cos 2pi r/H)^n.
* R3: periodic boundary conditions for L (implied by the DFT).
* R4: trilinear interpolation clamps sample coordinates to [0, dim-1]
  (border replicate); gradients are central differences with clamped
  indices, (f[min(i+1,n-1)] - f[max(i-1,0)]) / 2.
* R5: J = grad(I1 o phi), the gradient of the re-warped image.
* R6: ADMM state (w, b, w_hat, b_hat, alpha) is reset at every outer step;
  w^{-1} = b^{-1} = 0 (never used because beta_0 = 0).
* R7: the velocity composed at each outer step is the regularised iterate
  w^K (equal to v at convergence).
* R8: "sufficiently small" velocity (Sec. 2, after Eq. 1) is enforced by a
  global rescale v = s w^K, s = min(1, kappa / max_x ||D w(x)||_inf,
  delta / max_x |w(x)|_inf); kappa = delta = inf is the paper-literal
  (no rescale).  ||.||_inf of the 3x3 Jacobian is the max absolute row sum.
* R9: eps = 1e-6 for s = 1.
* R10: grid spacing 1 voxel on every axis.

Array conventions: scalars are ``[nz][ny][nx]`` (x fastest), vector fields
``[3][nz][ny][nx]`` with component 0 along x; dims are (nx, ny, nz) =
(M, N, H) in the paper's notation; displacements are in voxels and
phi(x) = x + u(x).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "nesterov_sequence", "data_step_l2", "data_step_l1", "laplacian_symbol",
    "spectral_solve", "apply_periodic_laplacian", "admm_step", "admm",
    "trilinear", "warp", "central_gradient", "linearise", "compose",
    "bound_scale", "jacobian_determinant", "register", "admm_until", "energy",
    "augmented_lagrangian", "dense_minimiser_l2", "admm_restart",
]


# ---------------------------------------------------------------- Eq. 5 scalars
def nesterov_sequence(K):
    """alpha^0..alpha^K and beta_0..beta_{K-1} of Eq. 5 (lines 4-6).

    alpha^0 = 1 (Sec. 3, after Eq. 5); alpha^{k+1} = (1 + sqrt(1 + 4
    (alpha^k)^2)) / 2; beta_k = (alpha^k - 1) / alpha^{k+1} is the factor in
    w_hat^{k+1} = w^k + beta_k (w^k - w^{k-1}).
    """
    alpha = [1.0]
    beta = []
    for k in range(K):
        a_next = (1.0 + math.sqrt(1.0 + 4.0 * alpha[k] * alpha[k])) / 2.0
        beta.append((alpha[k] - 1.0) / a_next)
        alpha.append(a_next)
    return alpha, beta


# ---------------------------------------------------------------- Eq. 6 v-step
def data_step_l2(u, J, c, theta):
    """s = 2 v-subproblem (Eq. 5 line 1, closed form Eq. 6 middle).

    Solves (J J^T + theta I) v = theta u - J c per voxel, with u = w_hat -
    b_hat and c = I1 - I0, by Sherman-Morrison:
    v = u - (J.u + c) J / (theta + |J|^2).
    """
    u = np.asarray(u, np.float64)
    J = np.asarray(J, np.float64)
    c = np.asarray(c, np.float64)
    rho = (J * u).sum(axis=0) + c
    return u - (rho / (theta + (J * J).sum(axis=0)))[None] * J


def data_step_l1(u, J, c, theta, eps=1e-6):
    """s = 1 v-subproblem (Eq. 5 line 1, closed form Eq. 6 top and the text
    after Eq. 6): z = theta rho(u) / (|J|^2 + eps),
    v = u - z / max(|z|, 1) * J / theta."""
    u = np.asarray(u, np.float64)
    J = np.asarray(J, np.float64)
    c = np.asarray(c, np.float64)
    rho = (J * u).sum(axis=0) + c
    z = theta * rho / ((J * J).sum(axis=0) + eps)
    t = z / np.maximum(np.abs(z), 1.0)
    return u - (t / theta)[None] * J


# ---------------------------------------------------------------- Eq. 6 w-step
def laplacian_symbol(dims, n):
    """F((-Delta_h)^n) on the DFT grid (text after Eq. 6, readings R2/R3):
    2^n (3 - cos(2 pi p/M) - cos(2 pi q/N) - cos(2 pi r/H))^n, returned as a
    [H][N][M] array (p along x, q along y, r along z)."""
    nx, ny, nz = dims
    p = np.arange(nx, dtype=np.float64)
    q = np.arange(ny, dtype=np.float64)
    r = np.arange(nz, dtype=np.float64)
    base = (3.0 - np.cos(2.0 * np.pi * r / nz)[:, None, None]
            - np.cos(2.0 * np.pi * q / ny)[None, :, None]
            - np.cos(2.0 * np.pi * p / nx)[None, None, :])
    return (2.0 ** n) * base ** n


def spectral_solve(y, lam, theta, n):
    """w-subproblem of Eq. 5 line 2 by Eq. 6 bottom (reading R1):
    w = F^-1[ theta F(y) / (lambda F((-Delta)^n) + theta) ], per component,
    with F the 3D DFT (periodic)."""
    y = np.asarray(y, np.float64)
    nz, ny, nx = y.shape[1:]
    denom = lam * laplacian_symbol((nx, ny, nz), n) + theta
    out = np.empty_like(y)
    for i in range(y.shape[0]):
        out[i] = np.real(np.fft.ifftn(theta * np.fft.fftn(y[i]) / denom))
    return out


def apply_periodic_laplacian(f, n=1):
    """(-Delta_h)^n f with the periodic 7-point stencil (unit spacing),
    applied n times; acts on the last three axes."""
    g = np.asarray(f, np.float64)
    for _ in range(n):
        acc = 6.0 * g
        for ax in (-1, -2, -3):
            acc = acc - np.roll(g, 1, axis=ax) - np.roll(g, -1, axis=ax)
        g = acc
    return g


# ---------------------------------------------------------------- Eq. 5 loop
def _v_step(u, J, c, theta, s, eps):
    if s == 2:
        return data_step_l2(u, J, c, theta)
    if s == 1:
        return data_step_l1(u, J, c, theta, eps)
    raise ValueError("s must be 1 or 2")


def admm_step(w_km1, w_km2, b_km1, b_km2, beta_km1, J, c, lam, theta, n,
              s=2, eps=1e-6):
    """One iteration k of Eq. 5 from the state after iteration k-1.

    w_hat^k = w^{k-1} + beta_{k-1} (w^{k-1} - w^{k-2}), b_hat^k likewise;
    v^k = v-step(w_hat^k - b_hat^k); w^k = w-step(v^k + b_hat^k);
    b^k = b_hat^k + v^k - w^k.  Returns (w^k, b^k, v^k).
    """
    w_hat = w_km1 + beta_km1 * (w_km1 - w_km2)
    b_hat = b_km1 + beta_km1 * (b_km1 - b_km2)
    v = _v_step(w_hat - b_hat, J, c, theta, s, eps)
    w = spectral_solve(v + b_hat, lam, theta, n)
    b = b_hat + v - w
    return w, b, v


def admm(J, c, lam, theta, n, iters, s=2, eps=1e-6, accelerate=True,
         history=False):
    """Nesterov-accelerated ADMM (Eq. 5) for the model of Eq. 2 linearised
    at the current warp.  Initial w_hat^0 = b_hat^0 = 0, alpha^0 = 1 (Sec. 3);
    ``accelerate=False`` sets every beta to 0 (plain ADMM).

    Returns w^{iters-1} (reading R7), or the list of (w^k, b^k) when
    ``history`` is set.
    """
    J = np.asarray(J, np.float64)
    c = np.asarray(c, np.float64)
    _, beta = nesterov_sequence(max(iters, 1))
    zero = np.zeros_like(J)
    w_km1, w_km2, b_km1, b_km2 = zero, zero, zero, zero
    hist = []
    for k in range(iters):
        bk = 0.0 if (k == 0 or not accelerate) else beta[k - 1]
        w, b, _ = admm_step(w_km1, w_km2, b_km1, b_km2, bk, J, c, lam, theta,
                            n, s, eps)
        w_km2, b_km2 = w_km1, b_km1
        w_km1, b_km1 = w, b
        if history:
            hist.append((w, b))
    return hist if history else w_km1


def admm_restart(J, c, lam, theta, n, iters, s=2, eps=1e-6, eta=0.999,
                 history=False):
    """Eq. 5 with adaptive restart (reading R20; not in the paper: the
    restart rule of Goldstein et al.'s fast ADMM, whose O(1/k^2) rate the
    paper cites after Eq. 5).

    Combined residual of iteration k: c_k = ||w^k - w_hat^k||^2 +
    ||b^k - b_hat^k||^2 over the grid (Goldstein et al.'s residual divided by
    the common factor theta).  With the reference cbar (+inf before the
    first test): if c_k < eta cbar, no restart and cbar = c_k; otherwise a
    restart and cbar = cbar / eta.  A restart found at iteration k restarts
    the momentum of the extrapolation that forms w_hat^{k+2}, b_hat^{k+2}
    (one iteration late, the first that can see the grid-wide c_k): the
    factor forming w_hat^j is beta_{j - r}, r the latest iteration whose
    factor a restart set to zero (r = 1 from the start, as beta_0 = 0), so
    the factors after a restart run 0, beta_1, beta_2, ...  eta = 0 restarts
    at every test (plain ADMM); eta = inf never restarts (Eq. 5 as printed).

    Returns w^{iters-1}, or with ``history`` a dict with lists "w", "b",
    "w_hat", "b_hat" (per iteration), "factor" (factor forming w_hat^k) and
    "restart" (iterations k whose test restarted)."""
    J = np.asarray(J, np.float64)
    c = np.asarray(c, np.float64)
    _, beta = nesterov_sequence(max(iters, 1) + 1)
    zero = np.zeros_like(J)
    w_km1, w_km2, b_km1, b_km2 = zero, zero, zero, zero
    r = 1                       # latest iteration whose factor is forced to 0
    pending = []                # iterations at which a found restart takes effect
    cbar = math.inf
    hist = {"w": [], "b": [], "w_hat": [], "b_hat": [], "factor": [], "restart": []}
    for k in range(iters):
        if k in pending:
            r = k
        f = 0.0 if k == 0 else beta[k - r]
        w_hat = w_km1 + f * (w_km1 - w_km2)
        b_hat = b_km1 + f * (b_km1 - b_km2)
        v = _v_step(w_hat - b_hat, J, c, theta, s, eps)
        w = spectral_solve(v + b_hat, lam, theta, n)
        b = b_hat + v - w
        ck = float(((w - w_hat) ** 2).sum() + ((b - b_hat) ** 2).sum())
        if eta > 0.0 and ck < eta * cbar:
            cbar = ck
        else:
            cbar = cbar / eta if eta > 0.0 else cbar
            pending.append(k + 2)
            hist["restart"].append(k)
        w_km2, b_km2 = w_km1, b_km1
        w_km1, b_km1 = w, b
        if history:
            for key, val in (("w", w), ("b", b), ("w_hat", w_hat), ("b_hat", b_hat),
                             ("factor", f)):
                hist[key].append(val)
    return hist if history else w_km1


# ---------------------------------------------------------------- grid ops
def trilinear(f, px, py, pz):
    """Trilinear interpolation of f [nz][ny][nx] at points (px, py, pz) in
    voxel units, coordinates clamped to [0, dim-1] (reading R4)."""
    f = np.asarray(f, np.float64)
    nz, ny, nx = f.shape
    px = np.clip(np.asarray(px, np.float64), 0.0, nx - 1.0)
    py = np.clip(np.asarray(py, np.float64), 0.0, ny - 1.0)
    pz = np.clip(np.asarray(pz, np.float64), 0.0, nz - 1.0)
    ix = np.minimum(np.floor(px).astype(np.int64), nx - 2)
    iy = np.minimum(np.floor(py).astype(np.int64), ny - 2)
    iz = np.minimum(np.floor(pz).astype(np.int64), nz - 2)
    fx, fy, fz = px - ix, py - iy, pz - iz
    c000 = f[iz, iy, ix]
    c001 = f[iz, iy, ix + 1]
    c010 = f[iz, iy + 1, ix]
    c011 = f[iz, iy + 1, ix + 1]
    c100 = f[iz + 1, iy, ix]
    c101 = f[iz + 1, iy, ix + 1]
    c110 = f[iz + 1, iy + 1, ix]
    c111 = f[iz + 1, iy + 1, ix + 1]
    c00 = c000 * (1 - fx) + c001 * fx
    c01 = c010 * (1 - fx) + c011 * fx
    c10 = c100 * (1 - fx) + c101 * fx
    c11 = c110 * (1 - fx) + c111 * fx
    c0 = c00 * (1 - fy) + c01 * fy
    c1 = c10 * (1 - fy) + c11 * fy
    return c0 * (1 - fz) + c1 * fz


def _grid(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64),
                          np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def warp(I1, u):
    """I1 o (Id + u): the re-warp of the source image (Sec. 2, text after
    Eq. 2, with N = 1)."""
    u = np.asarray(u, np.float64)
    x, y, z = _grid(u.shape[1:])
    return trilinear(I1, x + u[0], y + u[1], z + u[2])


def central_gradient(f):
    """Central differences with clamped indices along x, y, z (reading R4).
    Returns [3][nz][ny][nx]."""
    f = np.asarray(f, np.float64)
    out = np.empty((3,) + f.shape)
    for comp, ax in ((0, 2), (1, 1), (2, 0)):
        n = f.shape[ax]
        idx = np.arange(n)
        hi = np.take(f, np.minimum(idx + 1, n - 1), axis=ax)
        lo = np.take(f, np.maximum(idx - 1, 0), axis=ax)
        out[comp] = 0.5 * (hi - lo)
    return out


def linearise(I0, I1, u):
    """Data-term linearisation at the current warp (Eq. 2, reading R5):
    I1w = I1 o (Id + u), J = grad I1w, c = I1w - I0."""
    I1w = warp(I1, u)
    return central_gradient(I1w), I1w - np.asarray(I0, np.float64), I1w


def compose(u, v):
    """phi_new = phi o (Id + v) (Eq. 1 with N = 1): u_new(x) = v(x) +
    u(x + v(x))."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    x, y, z = _grid(u.shape[1:])
    px, py, pz = x + v[0], y + v[1], z + v[2]
    return v + np.stack([trilinear(u[i], px, py, pz) for i in range(3)])


def bound_scale(w, kappa=0.5, delta=1.0):
    """Global velocity rescale s of reading R8.  Returns (s, max |w|_inf,
    max ||Dw||_inf)."""
    w = np.asarray(w, np.float64)
    m_abs = float(np.abs(w).max()) if w.size else 0.0
    jac = np.zeros(w.shape[1:])
    for i in range(3):
        jac = np.maximum(jac, np.abs(central_gradient(w[i])).sum(axis=0))
    m_jac = float(jac.max()) if jac.size else 0.0
    s = 1.0
    if math.isfinite(kappa) and m_jac > 0.0:
        s = min(s, kappa / m_jac)
    if math.isfinite(delta) and m_abs > 0.0:
        s = min(s, delta / m_abs)
    return s, m_abs, m_jac


def jacobian_determinant(u):
    """det(I + Du) per voxel with the central differences of reading R4
    (the diffeomorphism check of Sec. 4, "Quantitative results")."""
    u = np.asarray(u, np.float64)
    D = np.stack([central_gradient(u[i]) for i in range(3)])  # D[i][j] = d u_i / d x_j
    A = D + np.eye(3)[:, :, None, None, None]
    return (A[0, 0] * (A[1, 1] * A[2, 2] - A[1, 2] * A[2, 1])
            - A[0, 1] * (A[1, 0] * A[2, 2] - A[1, 2] * A[2, 0])
            + A[0, 2] * (A[1, 0] * A[2, 1] - A[1, 1] * A[2, 0]))


# ---------------------------------------------------------------- outer loop
def admm_until(J, c, lam, theta, n, max_iters, tol, s=2, eps=1e-6):
    """Eq. 5 stopped by a threshold (Sec. 4, second hyper-parameter version;
    reading R18): after iteration k >= 1 stop when
    ||w^k - w^{k-1}||_2 <= tol ||w^k||_2, at most max_iters iterations.
    Returns (w, iterations run)."""
    J = np.asarray(J, np.float64)
    c = np.asarray(c, np.float64)
    _, beta = nesterov_sequence(max(max_iters, 1))
    zero = np.zeros_like(J)
    w_km1, w_km2, b_km1, b_km2 = zero, zero, zero, zero
    for k in range(max_iters):
        bk = 0.0 if k == 0 else beta[k - 1]
        w, b, _ = admm_step(w_km1, w_km2, b_km1, b_km2, bk, J, c, lam, theta, n, s, eps)
        w_km2, b_km2 = w_km1, b_km1
        w_km1, b_km1 = w, b
        if k >= 1 and np.sqrt(((w_km1 - w_km2) ** 2).sum()) <= tol * np.sqrt((w_km1 ** 2).sum()):
            return w_km1, k + 1
    return w_km1, max_iters


def register(I0, I1, lam=10.0, theta=0.1, n=2, outer=5, inner=10, s=2,
             eps=1e-6, kappa=0.5, delta=1.0, accelerate=True,
             return_scales=False, u0=None, admm_tol=0.0, warp_tol=0.0,
             return_counts=False, restart_eta=None):
    """Greedy diffeomorphic registration (Sec. 2, text after Eq. 2; Eq. 1
    with N = 1): u <- u0 (default 0); repeat ``outer`` times: linearise at
    the current warp of the original I1, run ``inner`` iterations of Eq. 5,
    bound the velocity (R8), compose phi <- phi o (Id + v).  Returns u with
    I1 o (Id + u) ~ I0.

    Thresholds (Sec. 4, second version; reading R18), 0 = off: ADMM stops
    early as in admm_until (then outer/inner are caps); the outer loop stops
    after the re-warp of step o when ||I1w_o - I1w_{o-1}||_2 <= warp_tol
    ||I1w_{o-1}||_2.  return_counts adds the list of ADMM iterations run per
    outer step.  ``restart_eta`` (not None) runs each inner loop as
    admm_restart with that eta (reading R20)."""
    I0 = np.asarray(I0, np.float64)
    I1 = np.asarray(I1, np.float64)
    u = np.zeros((3,) + I0.shape) if u0 is None else np.array(u0, np.float64)
    scales = []
    counts = []
    J, c, I1w = linearise(I0, I1, u)
    for o in range(outer):
        if admm_tol > 0.0:
            w, k = admm_until(J, c, lam, theta, n, inner, admm_tol, s, eps)
        elif restart_eta is not None:
            w, k = admm_restart(J, c, lam, theta, n, inner, s, eps, restart_eta), inner
        else:
            w, k = admm(J, c, lam, theta, n, inner, s, eps, accelerate), inner
        counts.append(k)
        sc, _, _ = bound_scale(w, kappa, delta)
        scales.append(sc)
        u = compose(u, sc * w)
        if o + 1 < outer:
            J, c, I1w_new = linearise(I0, I1, u)
            stop = warp_tol > 0.0 and (np.sqrt(((I1w_new - I1w) ** 2).sum())
                                       <= warp_tol * np.sqrt((I1w ** 2).sum()))
            I1w = I1w_new
            if stop:
                break
    out = [u]
    if return_scales:
        out.append(scales)
    if return_counts:
        out.append(counts)
    return out[0] if len(out) == 1 else tuple(out)


# ---------------------------------------------------------------- energies
def energy(v, J, c, lam, n, s=2):
    """Eq. 2 with reading R2: (1/s) sum |rho(v)|^s + (lambda/2) <v, L v>,
    L = (-Delta_h)^n applied per component (periodic stencil)."""
    v = np.asarray(v, np.float64)
    rho = (np.asarray(J, np.float64) * v).sum(axis=0) + np.asarray(c, np.float64)
    data = (np.abs(rho) ** s).sum() / s
    reg = sum(float((v[i] * apply_periodic_laplacian(v[i], n)).sum()) for i in range(3))
    return data + 0.5 * lam * reg


def augmented_lagrangian(v, w, b, J, c, lam, theta, n, s=2):
    """Eq. 4: (1/s)||rho(v)||^s + lambda/2 ||grad^n w||^2 +
    theta/2 ||w - v - b||^2 (reading R2 for the regulariser)."""
    v = np.asarray(v, np.float64)
    w = np.asarray(w, np.float64)
    b = np.asarray(b, np.float64)
    rho = (np.asarray(J, np.float64) * v).sum(axis=0) + np.asarray(c, np.float64)
    data = (np.abs(rho) ** s).sum() / s
    reg = sum(float((w[i] * apply_periodic_laplacian(w[i], n)).sum()) for i in range(3))
    return data + 0.5 * lam * reg + 0.5 * theta * float(((w - v - b) ** 2).sum())


def dense_minimiser_l2(J, c, lam, n):
    """Exact minimiser of Eq. 2 for s = 2 on a tiny grid by a dense direct
    solve of the normal equations (J J^T + lambda L) v = -J c, with L built
    from the periodic 7-point stencil (no FFT).  Unknowns ordered
    component-major."""
    J = np.asarray(J, np.float64)
    c = np.asarray(c, np.float64)
    shape = c.shape
    V = c.size
    eye = np.eye(V).reshape((V,) + shape)
    lap = np.stack([apply_periodic_laplacian(eye[i], n).ravel() for i in range(V)], axis=1)
    Jf = J.reshape(3, V)
    A = np.zeros((3 * V, 3 * V))
    for i in range(3):
        A[i * V:(i + 1) * V, i * V:(i + 1) * V] += lam * lap
        for j in range(3):
            A[i * V:(i + 1) * V, j * V:(j + 1) * V] += np.diag(Jf[i] * Jf[j])
    rhs = -(Jf * c.reshape(1, V)).ravel()
    return np.linalg.solve(A, rhs).reshape((3,) + shape)
