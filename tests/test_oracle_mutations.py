"""The oracle's pins catch plausible mistakes.

Each case plants one single-term mistake (a dropped term, a flipped sign, a
wrong index or operand order, a swapped component) into a temporary copy of
`oracle/`, on the CPU, and runs the pin file that covers that function
against the copy: the run must end with at least one failing test (pytest
exit status 1, not a collection or import error).  A control run of the
unmodified copy must pass.  Nothing here touches the repository's own files.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FWD, GRAD = "nadmm_oracle.py", "nadmm_oracle_grad.py"
EVAL, PYR = "nadmm_oracle_eval.py", "nadmm_oracle_pyramid.py"
PINS = {FWD: "test_oracle_pins.py", GRAD: "test_oracle_grad_pins.py",
        EVAL: "test_oracle_eval_pins.py", PYR: "test_oracle_pyramid_pins.py"}

# (oracle file, text as it stands, planted mistake)
MUTATIONS = [
    # Eq. 6 regulariser step and symbol
    (FWD, "theta * np.fft.fftn(y[i]) / denom", "np.fft.fftn(y[i]) / denom"),
    (FWD, "(2.0 ** n) * base ** n", "(2.0 ** n) * base"),
    (FWD, "- np.cos(2.0 * np.pi * q / ny)[None, :, None]",
     "- np.cos(2.0 * np.pi * q / nx)[None, :, None]"),
    # Eq. 5 dual update and Nesterov extrapolation
    (FWD, "b = b_hat + v - w", "b = b_hat - v + w"),
    (FWD, "else beta[k - 1]", "else beta[k]"),
    (FWD, "w_hat = w_km1 + beta_km1 * (w_km1 - w_km2)",
     "w_hat = w_km1 - beta_km1 * (w_km1 - w_km2)"),
    (FWD, "b_hat = b_km1 + beta_km1 * (b_km1 - b_km2)", "b_hat = b_km1"),
    (FWD, "w_km2, b_km2 = w_km1, b_km1", "w_km2, b_km2 = w_km1 * 0, b_km1"),
    (FWD, "a_next = (1.0 + math.sqrt(1.0 + 4.0 * alpha[k] * alpha[k])) / 2.0",
     "a_next = (1.0 + math.sqrt(1.0 + 2.0 * alpha[k] * alpha[k])) / 2.0"),
    # Eq. 6 data steps (s = 2, s = 1)
    (FWD, "[None] * J\n\n\ndef data_step_l1", "[None] * J[::-1]\n\n\ndef data_step_l1"),
    (FWD, "z = theta * rho / ((J * J).sum(axis=0) + eps)", "z = rho / ((J * J).sum(axis=0) + eps)"),
    (FWD, "return u - (t / theta)[None] * J", "return u - t[None] * J"),
    # gradient, interpolation, composition, bound, linearisation
    (FWD, "for comp, ax in ((0, 2), (1, 1), (2, 0)):", "for comp, ax in ((0, 0), (1, 1), (2, 2)):"),
    (FWD, "return c0 * (1 - fz) + c1 * fz", "return c0 * (1 - fy) + c1 * fy"),
    (FWD, "ix = np.minimum(np.floor(px).astype(np.int64), nx - 2)",
     "ix = np.minimum(np.rint(px).astype(np.int64), nx - 2)"),
    (FWD, "return v + np.stack([trilinear(u[i], px, py, pz) for i in range(3)])", "return v + u"),
    (FWD, "    return v + np.stack", "    return u + np.stack"),
    (FWD, "px, py, pz = x + v[0], y + v[1], z + v[2]", "px, py, pz = x + v[1], y + v[0], z + v[2]"),
    (FWD, "s = min(s, kappa / m_jac)", "s = min(s, m_jac / kappa)"),
    (FWD, "jac = np.maximum(jac, np.abs(central_gradient(w[i])).sum(axis=0))",
     "jac = np.maximum(jac, np.abs(central_gradient(w[i])).max(axis=0))"),
    (FWD, "return central_gradient(I1w), I1w - np.asarray(I0, np.float64), I1w",
     "return central_gradient(I1w), np.asarray(I0, np.float64) - I1w, I1w"),
    (FWD, "u = compose(u, sc * w)", "u = compose(sc * w, u)"),
    # Nesterov scalars, data steps, symbol and stencil, interpolation and
    # differences, bound and determinant, energies, dense minimiser, loop wiring
    (FWD, "beta.append((alpha[k] - 1.0) / a_next)", "beta.append(alpha[k] / a_next)"),
    (FWD, "t = z / np.maximum(np.abs(z), 1.0)", "t = z / np.maximum(np.abs(z), 2.0)"),
    (FWD, "rho = (J * u).sum(axis=0) + c\n    return u - (rho",
     "rho = (J * u).sum(axis=0) - c\n    return u - (rho"),
    (FWD, "return u - (rho / (theta + (J * J).sum(axis=0)))[None] * J",
     "return u - (rho / (1.0 + (J * J).sum(axis=0)))[None] * J"),
    (FWD, "base = (3.0 - np.cos", "base = (6.0 - np.cos"),
    (FWD, "acc = 6.0 * g", "acc = 4.0 * g"),
    (FWD, "acc = acc - np.roll(g, 1, axis=ax) - np.roll(g, -1, axis=ax)",
     "acc = acc - np.roll(g, 1, axis=ax) - np.roll(g, 1, axis=ax)"),
    (FWD, "px = np.clip(np.asarray(px, np.float64), 0.0, nx - 1.0)",
     "px = np.asarray(px, np.float64)"),
    (FWD, "c01 = c010 * (1 - fx) + c011 * fx", "c01 = c010 * (1 - fx) + c001 * fx"),
    (FWD, "return trilinear(I1, x + u[0], y + u[1], z + u[2])",
     "return trilinear(I1, x + u[0], y + u[2], z + u[1])"),
    (FWD, "out[comp] = 0.5 * (hi - lo)", "out[comp] = (hi - lo)"),
    (FWD, "lo = np.take(f, np.maximum(idx - 1, 0), axis=ax)", "lo = np.take(f, idx, axis=ax)"),
    (FWD, "s = min(s, delta / m_abs)", "s = min(s, m_abs / delta)"),
    (FWD, "m_abs = float(np.abs(w).max()) if w.size else 0.0",
     "m_abs = float(np.abs(w[0]).max()) if w.size else 0.0"),
    (FWD, "A = D + np.eye(3)[:, :, None, None, None]", "A = D"),
    (FWD, "- A[0, 1] * (A[1, 0] * A[2, 2] - A[1, 2] * A[2, 0])",
     "+ A[0, 1] * (A[1, 0] * A[2, 2] - A[1, 2] * A[2, 0])"),
    (FWD, "return data + 0.5 * lam * reg\n", "return data + lam * reg\n"),
    (FWD, "data = (np.abs(rho) ** s).sum() / s\n    reg = sum(float((v[i]",
     "data = (np.abs(rho) ** s).sum()\n    reg = sum(float((v[i]"),
    (FWD, "0.5 * theta * float(((w - v - b) ** 2).sum())",
     "0.5 * theta * float(((w - v + b) ** 2).sum())"),
    (FWD, "rhs = -(Jf * c.reshape(1, V)).ravel()", "rhs = (Jf * c.reshape(1, V)).ravel()"),
    (FWD, "A[i * V:(i + 1) * V, i * V:(i + 1) * V] += lam * lap",
     "A[i * V:(i + 1) * V, i * V:(i + 1) * V] += lap"),
    (FWD, "bk = 0.0 if (k == 0 or not accelerate) else beta[k - 1]",
     "bk = 0.0 if (k == 0) else beta[k - 1]"),
    (FWD, "w = spectral_solve(v + b_hat, lam, theta, n)", "w = spectral_solve(v, lam, theta, n)"),
    (FWD, "v = _v_step(w_hat - b_hat, J, c, theta, s, eps)",
     "v = _v_step(w_hat + b_hat, J, c, theta, s, eps)"),
    (FWD, "J, c, I1w = linearise(I0, I1, u)\n    for o",
     "J, c, I1w = linearise(I0, I1, np.zeros_like(u))\n    for o"),
    # adaptive restart (reading R20)
    (FWD, "pending.append(k + 2)", "pending.append(k + 1)"),
    (FWD, "            cbar = cbar / eta if eta > 0.0 else cbar", "            cbar = ck"),
    (FWD, "ck = float(((w - w_hat) ** 2).sum() + ((b - b_hat) ** 2).sum())",
     "ck = float(((w - w_hat) ** 2).sum())"),
    (FWD, "f = 0.0 if k == 0 else beta[k - r]", "f = 0.0 if k == 0 else beta[k - r + 1]"),
    (FWD, "        if k in pending:\n            r = k", "        if k in pending:\n            r = k - 1"),
    # threshold stopping (Sec. 4, second version)
    (FWD, "<= tol * np.sqrt((w_km1 ** 2).sum())", "<= tol * np.sqrt((w_km2 ** 2).sum())"),
    (FWD, "return w_km1, k + 1", "return w_km1, k"),
    (FWD, "if k >= 1 and np.sqrt(((w_km1 - w_km2) ** 2).sum())",
     "if k >= 2 and np.sqrt(((w_km1 - w_km2) ** 2).sum())"),
    (FWD, "<= warp_tol * np.sqrt((I1w ** 2).sum()))",
     "<= warp_tol * np.sqrt((I1w_new ** 2).sum()))"),
    (FWD, "            I1w = I1w_new\n", "\n"),
    (FWD, "            if stop:\n                break",
     "            if stop and o > 0:\n                break"),
    # reverse mode
    (GRAD, "(2.0 * rho * Jv / (d * d))[None] * J", "(1.0 * rho * Jv / (d * d))[None] * J"),
    (GRAD, "g_theta += float((rho * Jv / (d * d)).sum())", "g_theta += 0.0"),
    (GRAD, "Wbar[k - 1] += (1.0 + bp) * what_bar", "Wbar[k - 1] += what_bar"),
    (GRAD, "Bbar[k - 2] += -bp * bhat_bar", "Bbar[k - 2] += bp * bhat_bar"),
    (GRAD, "bhat_bar = ybar - ubar", "bhat_bar = ybar"),
    (GRAD, "ybar = spectral_solve(wbar - bbar, lam, theta, n) + bbar",
     "ybar = spectral_solve(wbar - bbar, lam, theta, n)"),
    (GRAD, "np.add.at(acc, np.maximum(idx - 1, 0), -0.5 * gc)",
     "np.add.at(acc, np.maximum(idx - 1, 0), 0.5 * gc)"),
    (GRAD, "gv[1] += gy", "gv[1] += gx"),
    (GRAD, "ds = -kappa / (m_jac * m_jac) * gs", "ds = -kappa / m_jac * gs"),
    (GRAD, "g_theta += -g_gamma * lam / (theta * theta)", "g_theta += g_gamma * lam / (theta * theta)"),
    (GRAD, "return -np.asarray(gc, np.float64), gI1, gu", "return np.asarray(gc, np.float64), gI1, gu"),
    (GRAD, "return -gL * r, gI1, gu", "return gL * r, gI1, gu"),
    (GRAD, "ubar = gu_prev + gu_lin", "ubar = gu_prev"),
    (GRAD, "wbar = wbar + bound_scale_vjp(w, kappa, delta, sbar)", "wbar = wbar"),
    (GRAD, "mult = -Kn / (1.0 + gamma * Kn) ** 2", "mult = -Kn / (1.0 + gamma * Kn)"),
    (GRAD, "inside_x = (px > 0.0) & (px < nx - 1.0)", "inside_x = np.ones_like(px, bool)"),
    # more reverse mode: adjoint weights and clamp masks, warp and compose
    # wiring, bound shares at ties, the ADMM recursion
    (GRAD, "d_fx = sum((corner[dz, dy, 1] - corner[dz, dy, 0]) * wy[dy] * wz[dz]",
     "d_fx = sum((corner[dz, dy, 1] - corner[dz, dy, 0]) * wy[dy] * wy[dz]"),
    (GRAD, "return gf, g * d_fx * inside_x, g * d_fy * inside_y, g * d_fz * inside_z",
     "return gf, g * d_fx * inside_x, g * d_fy * inside_y, g * d_fz * inside_y"),
    (GRAD, "wx = (1.0 - fx, fx)", "wx = (fx, 1.0 - fx)"),
    (GRAD, "gI1, gx, gy, gz = trilinear_vjp(I1, x + u[0], y + u[1], z + u[2], g)",
     "gI1, gx, gy, gz = trilinear_vjp(I1, x + u[0], y + u[1], z + u[1], g)"),
    (GRAD, "g_w = central_gradient_vjp(gJ) + np.asarray(gc, np.float64)",
     "g_w = central_gradient_vjp(gJ) - np.asarray(gc, np.float64)"),
    (GRAD, "gv = g.copy()", "gv = np.zeros_like(g)"),
    (GRAD, "count = sum(int(h.sum()) for h in hits)", "count = 1"),
    (GRAD, "gw += np.sign(w) * hits * (ds / int(hits.sum()))", "gw += np.sign(w) * hits * ds"),
    (GRAD, "G = np.sign(D[i]) * hits[i][None] * (ds / count)",
     "G = D[i] * hits[i][None] * (ds / count)"),
    (GRAD, "ds = -delta / (m_abs * m_abs) * gs", "ds = -delta / m_abs * gs"),
    (GRAD, "gw += np.sign(w) * hits * (ds / int(hits.sum()))",
     "gw += hits * (ds / int(hits.sum()))"),
    (GRAD, "u = w_hat - b_hat\n        rho", "u = w_hat + b_hat\n        rho"),
    (GRAD, "y = W[k] + B[k]", "y = W[k] - B[k]"),
    (GRAD, "ubar = vbar - J * (Jv / d)[None]", "ubar = vbar"),
    (GRAD, "gc += -Jv / d", "gc += Jv / d"),
    (GRAD, "gJ += -(rho / d)[None] * vbar - (Jv / d)[None] * u", "gJ += -(rho / d)[None] * vbar"),
    (GRAD, "g_lam = g_gamma / theta", "g_lam = g_gamma * theta"),
    (GRAD, "Bbar[k - 1] += (1.0 + bp) * bhat_bar", "Bbar[k - 1] += bhat_bar"),
    (GRAD, "if k - 2 >= 0 and bp != 0.0:", "if k - 2 >= 1 and bp != 0.0:"),
    (GRAD, "bp = 0.0 if (k == 0 or not accelerate) else beta[k - 1]",
     "bp = 0.0 if (k == 0 or not accelerate) else beta[k]"),
    (GRAD, "g_gamma += float(((wbar - bbar) * spectral_solve_dgamma(y, lam, theta, n)).sum())",
     "g_gamma += float((wbar * spectral_solve_dgamma(y, lam, theta, n)).sum())"),
    # reverse sweep wiring and the SSD loss
    (GRAD, "wbar = s * vbar", "wbar = vbar"),
    (GRAD, "sbar = float((vbar * w).sum())", "sbar = float((vbar * s * w).sum())"),
    (GRAD, "gu_prev, vbar = compose_vjp(u, s * w, ubar)",
     "gu_prev, vbar = compose_vjp(u, w, ubar)"),
    (GRAD, "        g_lam += gl\n", "\n"),
    (GRAD, "        gI0 += a0\n", "\n"),
    (GRAD, "for (u, J, c, w, s) in reversed(tape):", "for (u, J, c, w, s) in tape:"),
    (GRAD, "r = warp(I1, u) - np.asarray(I0, np.float64)\n    return 0.5",
     "r = warp(I1, u) - np.asarray(I0, np.float64)\n    return 1.0"),
    (GRAD, "gI1, gu = warp_vjp(I1, u, gL * r)", "gI1, gu = warp_vjp(I1, u, r)"),
    (GRAD, "return L, d0 + r0, d1 + r1, gl, gt", "return L, d0, d1 + r1, gl, gt"),
    (GRAD, "J, c, _ = linearise(I0, I1, u)\n        w = admm(",
     "J, c, _ = linearise(I0, I1, np.zeros_like(u))\n        w = admm("),
    # Sec. 4 measures
    (EVAL, "return 1.0 if s == 0 else 2.0 * int((A & B).sum()) / s",
     "return 1.0 if s == 0 else int((A & B).sum()) / s"),
    (EVAL, "vals.append(max(_directed(A, B), _directed(B, A)) * spacing)",
     "vals.append(_directed(A, B) * spacing)"),
    (EVAL, "return np.clip(np.floor(p + 0.5), 0, n - 1).astype(np.int64)",
     "return np.clip(np.floor(p), 0, n - 1).astype(np.int64)"),
    (EVAL, "return 100.0 * float((det <= 0).sum()) / det.size",
     "return 100.0 * float((det < 0).sum()) / det.size"),
    # pyramid
    (PYR, "px, py, pz = (x - 0.5) / 2.0, (y - 0.5) / 2.0, (z - 0.5) / 2.0",
     "px, py, pz = x / 2.0, y / 2.0, z / 2.0"),
    (PYR, "return np.stack([2.0 * trilinear(uc[i], px, py, pz) for i in range(3)])",
     "return np.stack([trilinear(uc[i], px, py, pz) for i in range(3)])"),
    (PYR, "return f.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(1, 3, 5))",
     "return f[::2, ::2, ::2]"),
    # more measures and pyramid: axes, rounding, empty cases, spacing, level
    # order and inputs, the coarse start, the upsampling axes
    (EVAL, "return labels[near(z + u[2], nz), near(y + u[1], ny), near(x + u[0], nx)]",
     "return labels[near(z + u[2], nz), near(y + u[0], ny), near(x + u[1], nx)]"),
    (EVAL, "return np.clip(np.floor(p + 0.5), 0, n - 1).astype(np.int64)",
     "return np.floor(p + 0.5).astype(np.int64) % n"),
    (EVAL, "return 1.0 if s == 0 else 2.0", "return 0.0 if s == 0 else 2.0"),
    (EVAL, "d = distance_transform_edt(~B)", "d = distance_transform_edt(B)"),
    (EVAL, "if A.any() and B.any():", "if A.any() or B.any():"),
    (EVAL, "return float(np.mean(vals)) if vals else float(\"nan\")",
     "return float(np.max(vals)) if vals else float(\"nan\")"),
    (EVAL, "def hausdorff_per_slice(a, b, label, spacing=1.2):",
     "def hausdorff_per_slice(a, b, label, spacing=1.0):"),
    (PYR, "        I1s.append(downsample2(I1s[-1]))", "        I1s.append(downsample2(I0s[-2]))"),
    (PYR, "lvl = levels - 1 - i", "lvl = i"),
    (PYR, "u = register(I0s[lvl], I1s[lvl], outer=outer[i], inner=inner[i], u0=u, **kw)",
     "u = register(I0s[lvl], I1s[lvl], outer=outer[i], inner=inner[i], **kw)"),
    (PYR, "px, py, pz = (x - 0.5) / 2.0, (y - 0.5) / 2.0, (z - 0.5) / 2.0",
     "px, py, pz = (x - 0.5) / 2.0, (z - 0.5) / 2.0, (y - 0.5) / 2.0"),
]

CONFTEST = '''import os, sys
HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
'''


def _stage(dst, oracle_file=None, old=None, new=None):
    """Copy of oracle/, synth and one pin file under dst, with one edit."""
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__", "*.so", "*.o"))
    pkg = os.path.join(dst, "paper_2109_12688_gb300")
    os.makedirs(pkg)
    open(os.path.join(pkg, "__init__.py"), "w").close()
    shutil.copy(os.path.join(ROOT, "paper_2109_12688_gb300", "synth.py"), pkg)
    with open(os.path.join(dst, "conftest.py"), "w") as fh:
        fh.write(CONFTEST)
    if oracle_file is not None:
        path = os.path.join(dst, "oracle", oracle_file)
        src = open(path).read()
        assert old in src, f"{oracle_file} no longer contains {old!r}: update the case"
        with open(path, "w") as fh:
            fh.write(src.replace(old, new, 1))


def _run_pins(dst, pin_file):
    shutil.copy(os.path.join(ROOT, "tests", pin_file), dst)
    # one thread per run: the runs themselves go in parallel
    env = dict(os.environ, PYTHONPATH=dst, PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="1",
               OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "--rootdir", dst, os.path.join(dst, pin_file)],
                       cwd=dst, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-400:]


def test_unmodified_copy_passes_every_pin_file(tmp_path):
    _stage(str(tmp_path))
    for pin_file in sorted(set(PINS.values())):
        rc, out = _run_pins(str(tmp_path), pin_file)
        assert rc == 0, (pin_file, out)


def test_every_planted_mistake_fails_a_pin(tmp_path):
    def one(i):
        oracle_file, old, new = MUTATIONS[i]
        dst = str(tmp_path / f"m{i:02d}")
        os.makedirs(dst)
        _stage(dst, oracle_file, old, new)
        return i, *_run_pins(dst, PINS[oracle_file])

    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(one, range(len(MUTATIONS))))
    missed = [(MUTATIONS[i][0], MUTATIONS[i][2][:70], rc, out) for i, rc, out in results if rc != 1]
    assert not missed, missed
