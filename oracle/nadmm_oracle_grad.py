"""FP64 reverse mode of the registration (vector-Jacobian products).

TEST INFRASTRUCTURE ONLY, like ``nadmm_oracle``: imported by ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs, never by the
product path, and sharing no code with it.

Each ``*_vjp`` function is the adjoint of the forward function of the same
name in ``nadmm_oracle``: given the gradient g of a scalar with respect to
the forward output, it returns the gradients with respect to the inputs.
They are written out by hand from the forward formulas (no automatic
differentiation) and pinned by finite differences in the tests.

Conventions at the non-smooth points (measure zero for generic inputs):
* trilinear sampling: the clamp of a coordinate to [0, dim-1] passes no
  gradient to the coordinate unless it lies strictly inside;
* |.|: sign(0) = 0;
* the maxima of the velocity bound (reading R8): the gradient is shared
  equally by all entries attaining the maximum; s = min(1, kappa/m_jac,
  delta/m_abs) follows the first candidate, in that order, that attains it.

The data term is s = 2 (Eq. 6, middle): the s = 1 thresholding is piecewise
and not differentiated here.
"""
from __future__ import annotations

import math

import numpy as np

from .nadmm_oracle import (_grid, admm, bound_scale, central_gradient, compose,
                           laplacian_symbol, linearise, nesterov_sequence,
                           spectral_solve, trilinear, warp)

__all__ = [
    "trilinear_vjp", "warp_vjp", "central_gradient_vjp", "linearise_vjp",
    "compose_vjp", "bound_scale_vjp", "spectral_solve_dgamma", "admm_vjp",
    "register_tape", "register_vjp", "ssd_after_warp", "ssd_after_warp_vjp",
    "loss_and_gradients",
]


# ---------------------------------------------------------------- grid ops
def trilinear_vjp(f, px, py, pz, g):
    """Adjoint of trilinear(f, px, py, pz) (reading R4): returns
    (g_f [nz][ny][nx], g_px, g_py, g_pz) for the output gradient g."""
    f = np.asarray(f, np.float64)
    g = np.asarray(g, np.float64)
    nz, ny, nx = f.shape
    px = np.asarray(px, np.float64)
    py = np.asarray(py, np.float64)
    pz = np.asarray(pz, np.float64)
    cx = np.clip(px, 0.0, nx - 1.0)
    cy = np.clip(py, 0.0, ny - 1.0)
    cz = np.clip(pz, 0.0, nz - 1.0)
    inside_x = (px > 0.0) & (px < nx - 1.0)
    inside_y = (py > 0.0) & (py < ny - 1.0)
    inside_z = (pz > 0.0) & (pz < nz - 1.0)
    ix = np.minimum(np.floor(cx).astype(np.int64), nx - 2)
    iy = np.minimum(np.floor(cy).astype(np.int64), ny - 2)
    iz = np.minimum(np.floor(cz).astype(np.int64), nz - 2)
    fx, fy, fz = cx - ix, cy - iy, cz - iz
    wx = (1.0 - fx, fx)
    wy = (1.0 - fy, fy)
    wz = (1.0 - fz, fz)
    gf = np.zeros_like(f)
    corner = {}
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                idx = (iz + dz, iy + dy, ix + dx)
                np.add.at(gf, idx, g * wz[dz] * wy[dy] * wx[dx])
                corner[dz, dy, dx] = f[idx]
    # partial derivatives of the trilinear polynomial in (fx, fy, fz)
    d_fx = sum((corner[dz, dy, 1] - corner[dz, dy, 0]) * wy[dy] * wz[dz]
               for dz in (0, 1) for dy in (0, 1))
    d_fy = sum((corner[dz, 1, dx] - corner[dz, 0, dx]) * wx[dx] * wz[dz]
               for dz in (0, 1) for dx in (0, 1))
    d_fz = sum((corner[1, dy, dx] - corner[0, dy, dx]) * wx[dx] * wy[dy]
               for dy in (0, 1) for dx in (0, 1))
    return gf, g * d_fx * inside_x, g * d_fy * inside_y, g * d_fz * inside_z


def warp_vjp(I1, u, g):
    """Adjoint of warp(I1, u) = I1 o (Id + u): returns (g_I1, g_u)."""
    u = np.asarray(u, np.float64)
    x, y, z = _grid(u.shape[1:])
    gI1, gx, gy, gz = trilinear_vjp(I1, x + u[0], y + u[1], z + u[2], g)
    return gI1, np.stack([gx, gy, gz])


def central_gradient_vjp(g):
    """Adjoint of central_gradient (clamped central differences, R4):
    g [3][nz][ny][nx] -> gradient [nz][ny][nx] of the input field."""
    g = np.asarray(g, np.float64)
    out = np.zeros(g.shape[1:])
    for comp, ax in ((0, 2), (1, 1), (2, 0)):
        n = g.shape[1 + ax]
        idx = np.arange(n)
        gc = np.moveaxis(g[comp], ax, 0)
        acc = np.zeros_like(gc)
        np.add.at(acc, np.minimum(idx + 1, n - 1), 0.5 * gc)
        np.add.at(acc, np.maximum(idx - 1, 0), -0.5 * gc)
        out += np.moveaxis(acc, 0, ax)
    return out


def linearise_vjp(I0, I1, u, gJ, gc, gI1w=None):
    """Adjoint of linearise: (J, c, I1w) = (grad I1w, I1w - I0, I1 o (Id+u)).
    Returns (g_I0, g_I1, g_u)."""
    g_w = central_gradient_vjp(gJ) + np.asarray(gc, np.float64)
    if gI1w is not None:
        g_w = g_w + gI1w
    gI1, gu = warp_vjp(I1, u, g_w)
    return -np.asarray(gc, np.float64), gI1, gu


def compose_vjp(u, v, g):
    """Adjoint of compose(u, v) = v + u(x + v(x)): returns (g_u, g_v)."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    g = np.asarray(g, np.float64)
    x, y, z = _grid(u.shape[1:])
    px, py, pz = x + v[0], y + v[1], z + v[2]
    gu = np.zeros_like(u)
    gv = g.copy()
    for i in range(3):
        gf, gx, gy, gz = trilinear_vjp(u[i], px, py, pz, g[i])
        gu[i] = gf
        gv[0] += gx
        gv[1] += gy
        gv[2] += gz
    return gu, gv


def bound_scale_vjp(w, kappa, delta, gs):
    """Adjoint of the scale s = bound_scale(w, kappa, delta)[0] (R8) for the
    scalar output gradient gs: returns g_w."""
    w = np.asarray(w, np.float64)
    s, m_abs, m_jac = bound_scale(w, kappa, delta)
    cands = [("one", 1.0)]
    if math.isfinite(kappa) and m_jac > 0.0:
        cands.append(("jac", kappa / m_jac))
    if math.isfinite(delta) and m_abs > 0.0:
        cands.append(("abs", delta / m_abs))
    active = next(name for name, val in cands if val == s)
    gw = np.zeros_like(w)
    if active == "jac":
        ds = -kappa / (m_jac * m_jac) * gs
        D = [central_gradient(w[i]) for i in range(3)]          # D[i][j] = d w_i / d x_j
        rows = [np.abs(D[i]).sum(axis=0) for i in range(3)]     # ||row i||_1 per voxel
        hits = [r == m_jac for r in rows]
        count = sum(int(h.sum()) for h in hits)
        for i in range(3):
            G = np.sign(D[i]) * hits[i][None] * (ds / count)
            gw[i] += central_gradient_vjp(G)
    elif active == "abs":
        ds = -delta / (m_abs * m_abs) * gs
        hits = np.abs(w) == m_abs
        gw += np.sign(w) * hits * (ds / int(hits.sum()))
    return gw


# ---------------------------------------------------------------- Eq. 5 / 6
def spectral_solve_dgamma(y, lam, theta, n):
    """d/dgamma of spectral_solve(y) with gamma = lambda / theta:
    F^-1[ -K^n / (1 + gamma K^n)^2 F(y) ] per component."""
    y = np.asarray(y, np.float64)
    nz, ny, nx = y.shape[1:]
    Kn = laplacian_symbol((nx, ny, nz), n)
    gamma = lam / theta
    mult = -Kn / (1.0 + gamma * Kn) ** 2
    out = np.empty_like(y)
    for i in range(y.shape[0]):
        out[i] = np.real(np.fft.ifftn(mult * np.fft.fftn(y[i])))
    return out


def admm_vjp(J, c, lam, theta, n, iters, gw, accelerate=True):
    """Adjoint of admm(J, c, lam, theta, n, iters) (s = 2) for the gradient
    gw of its output w^{iters-1}.  Returns (g_J, g_c, g_lambda, g_theta).

    Forward, per iteration k (Eq. 5): w_hat = w^{k-1} + beta'(w^{k-1} -
    w^{k-2}), b_hat likewise, u = w_hat - b_hat, rho = J.u + c,
    v = u - rho J / d with d = theta + |J|^2, y = v + b_hat, w^k = S y with
    S = 1/(1 + gamma K^n), gamma = lambda/theta, b^k = y - w^k.
    The reverse sweep takes these steps backwards; S is symmetric, so the
    adjoint of w = S y, b = y - S y is y_bar = S(w_bar - b_bar) + b_bar.
    """
    J = np.asarray(J, np.float64)
    c = np.asarray(c, np.float64)
    hist = admm(J, c, lam, theta, n, iters, history=True, accelerate=accelerate)
    _, beta = nesterov_sequence(max(iters, 1))
    K = iters
    zero = np.zeros_like(J)
    W = [h[0] for h in hist]
    B = [h[1] for h in hist]

    def state(k):
        return (W[k], B[k]) if k >= 0 else (zero, zero)

    d = theta + (J * J).sum(axis=0)
    Wbar = [np.zeros_like(J) for _ in range(K)]
    Bbar = [np.zeros_like(J) for _ in range(K)]
    Wbar[K - 1] = np.asarray(gw, np.float64).copy()
    gJ = np.zeros_like(J)
    gc = np.zeros_like(c)
    g_gamma = 0.0
    g_theta = 0.0
    for k in range(K - 1, -1, -1):
        bp = 0.0 if (k == 0 or not accelerate) else beta[k - 1]
        w1, b1 = state(k - 1)
        w2, b2 = state(k - 2)
        w_hat = w1 + bp * (w1 - w2)
        b_hat = b1 + bp * (b1 - b2)
        u = w_hat - b_hat
        rho = (J * u).sum(axis=0) + c
        y = W[k] + B[k]
        wbar, bbar = Wbar[k], Bbar[k]
        ybar = spectral_solve(wbar - bbar, lam, theta, n) + bbar
        g_gamma += float(((wbar - bbar) * spectral_solve_dgamma(y, lam, theta, n)).sum())
        vbar = ybar
        Jv = (J * vbar).sum(axis=0)
        ubar = vbar - J * (Jv / d)[None]
        gc += -Jv / d
        gJ += -(rho / d)[None] * vbar - (Jv / d)[None] * u + (2.0 * rho * Jv / (d * d))[None] * J
        g_theta += float((rho * Jv / (d * d)).sum())
        what_bar = ubar
        bhat_bar = ybar - ubar
        if k - 1 >= 0:
            Wbar[k - 1] += (1.0 + bp) * what_bar
            Bbar[k - 1] += (1.0 + bp) * bhat_bar
        if k - 2 >= 0 and bp != 0.0:
            Wbar[k - 2] += -bp * what_bar
            Bbar[k - 2] += -bp * bhat_bar
    g_lam = g_gamma / theta
    g_theta += -g_gamma * lam / (theta * theta)
    return gJ, gc, g_lam, g_theta


# ---------------------------------------------------------------- outer loop
def register_tape(I0, I1, lam=10.0, theta=0.1, n=2, outer=5, inner=10,
                  kappa=0.5, delta=1.0):
    """register(..., s=2) keeping what the reverse sweep needs: the list of
    per-outer-step (u_o, J_o, c_o, w_o, s_o) and the final u."""
    I0 = np.asarray(I0, np.float64)
    I1 = np.asarray(I1, np.float64)
    u = np.zeros((3,) + I0.shape)
    tape = []
    for _ in range(outer):
        J, c, _ = linearise(I0, I1, u)
        w = admm(J, c, lam, theta, n, inner)
        s, _, _ = bound_scale(w, kappa, delta)
        tape.append((u, J, c, w, s))
        u = compose(u, s * w)
    return u, tape


def register_vjp(I0, I1, gu, lam=10.0, theta=0.1, n=2, outer=5, inner=10,
                 kappa=0.5, delta=1.0):
    """Adjoint of register(I0, I1, ..., s=2): for the gradient gu of the
    final displacement, returns (g_I0, g_I1, g_lambda, g_theta)."""
    I0 = np.asarray(I0, np.float64)
    I1 = np.asarray(I1, np.float64)
    _, tape = register_tape(I0, I1, lam, theta, n, outer, inner, kappa, delta)
    gI0 = np.zeros_like(I0)
    gI1 = np.zeros_like(I1)
    g_lam = 0.0
    g_theta = 0.0
    ubar = np.asarray(gu, np.float64).copy()
    for (u, J, c, w, s) in reversed(tape):
        gu_prev, vbar = compose_vjp(u, s * w, ubar)
        wbar = s * vbar
        sbar = float((vbar * w).sum())
        wbar = wbar + bound_scale_vjp(w, kappa, delta, sbar)
        gJ, gc, gl, gt = admm_vjp(J, c, lam, theta, n, inner, wbar)
        g_lam += gl
        g_theta += gt
        a0, a1, gu_lin = linearise_vjp(I0, I1, u, gJ, gc)
        gI0 += a0
        gI1 += a1
        ubar = gu_prev + gu_lin
    return gI0, gI1, g_lam, g_theta


def ssd_after_warp(I0, I1, u):
    """L = 1/2 sum (I1 o (Id + u) - I0)^2 (the loss the gradients are taken of)."""
    r = warp(I1, u) - np.asarray(I0, np.float64)
    return 0.5 * float((r * r).sum())


def ssd_after_warp_vjp(I0, I1, u, gL=1.0):
    """Adjoint of ssd_after_warp: returns (g_I0, g_I1, g_u)."""
    r = warp(I1, u) - np.asarray(I0, np.float64)
    gI1, gu = warp_vjp(I1, u, gL * r)
    return -gL * r, gI1, gu


def loss_and_gradients(I0, I1, lam=10.0, theta=0.1, n=2, outer=5, inner=10,
                       kappa=0.5, delta=1.0):
    """L = ssd_after_warp(I0, I1, register(I0, I1)) and its gradients with
    respect to I0, I1, lambda and theta: (L, g_I0, g_I1, g_lambda, g_theta)."""
    u, _ = register_tape(I0, I1, lam, theta, n, outer, inner, kappa, delta)
    L = ssd_after_warp(I0, I1, u)
    d0, d1, gu = ssd_after_warp_vjp(I0, I1, u)
    r0, r1, gl, gt = register_vjp(I0, I1, gu, lam, theta, n, outer, inner, kappa, delta)
    return L, d0 + r0, d1 + r1, gl, gt
