"""Threshold stopping (Sec. 4, second version; the oracle's admm_until and
register(admm_tol, warp_tol)): the GPU stops after the same ADMM iteration
and the same outer step as the FP64 oracle and returns the same displacement
(max |du| <= 1e-3 voxel).  Thresholds are placed between the oracle's
residuals with a margin, so FP32 rounding cannot flip a decision."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2109_12688_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2109_12688_gb300 import nadmm
    return nadmm


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def oracle_decisions(p, outer, inner, admm_tol, warp_tol, n=2):
    """Every residual the oracle compares with a threshold, as ratios
    residual / threshold (a decision is safe when the ratio is not ~1)."""
    I0, I1 = p["fixed"].astype(float), p["moving"].astype(float)
    u = np.zeros((3,) + I0.shape)
    ratios = []
    J, c, I1w = O.linearise(I0, I1, u)
    for o in range(outer):
        hist = O.admm(J, c, 10.0, 0.1, n, inner, history=True)
        for k in range(1, inner):
            r = np.linalg.norm(hist[k][0] - hist[k - 1][0]) / np.linalg.norm(hist[k][0])
            ratios.append(r / admm_tol)
            if r <= admm_tol:
                w = hist[k][0]
                break
        else:
            w = hist[inner - 1][0]
        s, _, _ = O.bound_scale(w, 0.5, 1.0)
        u = O.compose(u, s * w)
        if o + 1 < outer:
            J, c, I1w_new = O.linearise(I0, I1, u)
            r = np.linalg.norm(I1w_new - I1w) / np.linalg.norm(I1w)
            I1w = I1w_new
            if warp_tol > 0:
                ratios.append(r / warp_tol)
                if r <= warp_tol:
                    break
    return ratios


@pytest.mark.parametrize("dims,seed,outer,inner,admm_tol,warp_tol", [
    ((32, 32, 24), 1, 12, 30, 0.06, 0.02),
    ((32, 32, 24), 2, 12, 30, 0.03, 0.01),
    ((64, 64, 48), 3, 12, 30, 0.1, 0.015),
    ((128, 128, 96), 0, 3, 12, 0.1, 0.0),
])
def test_thresholds_match_the_oracle(lib, dims, seed, outer, inner, admm_tol, warp_tol):
    p = synth.make_pair(dims, seed=seed)
    ratios = oracle_decisions(p, outer, inner, admm_tol, warp_tol)
    assert min(abs(math.log(r)) for r in ratios) > 0.005, "threshold too close to a residual"
    u_ref, counts = O.register(p["fixed"], p["moving"], lam=10.0, theta=0.1, n=2, outer=outer,
                               inner=inner, admm_tol=admm_tol, warp_tol=warp_tol,
                               return_counts=True)
    reg = lib.Registration(dims, device=DEV, outer=outer, inner=inner, admm_tol=admm_tol,
                           warp_tol=warp_tol)
    u = reg.register(dev(p["fixed"]), dev(p["moving"]))
    assert lib.nadmm_get_status(reg.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    o_run, a_run = lib.nadmm_get_iterations(reg.handle, torch.cuda.current_stream())
    assert (o_run, a_run) == (len(counts), sum(counts))
    assert np.abs(u.cpu().numpy() - u_ref).max() <= 1e-3
    if warp_tol > 0:
        assert len(counts) < outer  # the outer loop stopped early
    assert sum(counts) < len(counts) * inner  # some ADMM loop stopped before its cap
    # a second run on the same handle (graph replay) repeats it
    u2 = reg.register(dev(p["fixed"]), dev(p["moving"]))
    assert torch.equal(u, u2)
    assert lib.nadmm_get_iterations(reg.handle, torch.cuda.current_stream()) == (o_run, a_run)


def test_thresholds_off_are_the_fixed_schedule(lib):
    dims = (32, 32, 24)
    p = synth.make_pair(dims, seed=7)
    # threshold handles run the four-kernel path (its kernels read the stop words)
    a = lib.Registration(dims, device=DEV, outer=3, inner=5, flags=lib.NADMM_FLAG_FOUR_PASS)
    b = lib.Registration(dims, device=DEV, outer=3, inner=5, warp_tol=1e-12)
    ua = a.register(dev(p["fixed"]), dev(p["moving"]))
    ub = b.register(dev(p["fixed"]), dev(p["moving"]))
    assert torch.equal(ua, ub)
    assert lib.nadmm_get_iterations(b.handle, torch.cuda.current_stream()) == (3, 15)
