"""Grids whose sides have prime factors above 7 (no FFT codelet): those
factors run as direct-sum stages of the mixed-radix transform, first in the
plan.  CUDA path vs the FP64 oracle (numpy's FFT handles any length) on the
spectral solve (Eq. 6), teacher-forced ADMM iterates (Eq. 5) and whole
registrations, with the tolerances of the smooth grids."""
import numpy as np
import pytest

import oracle as O
from paper_2109_12688_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"
# x: 44 = 11 x 4, 88 = 11 x 8, 100 = 25 x 4; y: 26 = 13 x 2, 52 = 13 x 4;
# z: 23, 97, 251 (prime), 34 = 17 x 2, 143 = 11 x 13 (every stage generic)
PRIME_GRIDS = [(44, 26, 23), (88, 52, 34), (100, 98, 97), (20, 22, 143), (4, 4, 251),
               (44, 8, 8), (8, 8, 13)]


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


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-30))


@pytest.mark.parametrize("dims", PRIME_GRIDS)
@pytest.mark.parametrize("n", [1, 3])
def test_spectral_solve_prime_sizes(lib, dims, n):
    nx, ny, nz = dims
    reg = lib.Registration(dims, device=DEV, order_n=n, lam=10.0, theta=0.1)
    y = synth.random_field((3, nz, ny, nx), seed=n + nz)
    w = torch.empty((3, nz, ny, nx), device=DEV)
    lib.nadmm_spectral_solve(reg.handle, dev(y), w, torch.cuda.current_stream())
    ref = O.spectral_solve(y, 10.0, 0.1, n)
    got = host(w)
    # a direct r-term sum rounds like r additions: allow 5e-6 of max |y|
    assert np.abs(got - ref).max() <= 5e-6 * np.abs(y).max()
    assert rel_l2(got, ref) <= 2e-6


@pytest.mark.parametrize("dims", [(44, 26, 23), (88, 52, 34)])
def test_admm_iterates_teacher_forced_prime_sizes(lib, dims):
    nx, ny, nz = dims
    lam, theta, n, K = 10.0, 0.1, 2, 6
    p = synth.make_pair(dims, seed=5)
    J, c, _ = O.linearise(p["fixed"], p["moving"], np.zeros((3,) + p["fixed"].shape))
    hist = O.admm(J, c, lam, theta, n, K, history=True)
    reg = lib.Registration(dims, device=DEV, order_n=n, lam=lam, theta=theta)
    shape = (3, nz, ny, nx)
    zero = np.zeros(shape, np.float32)
    w_out = torch.empty(shape, device=DEV)
    b_out = torch.empty(shape, device=DEV)
    Jd, cd = dev(J), dev(c)
    for k in range(K):
        wk1, bk1 = hist[k - 1] if k >= 1 else (zero, zero)
        wk2, bk2 = hist[k - 2] if k >= 2 else (zero, zero)
        lib.nadmm_admm_run(reg.handle, Jd, cd, dev(wk1), dev(wk2), dev(bk1), dev(bk2), k, 1,
                           w_out, b_out, torch.cuda.current_stream())
        w_ref, b_ref = hist[k]
        assert rel_l2(host(w_out), w_ref) <= 1e-5, k
        assert rel_l2(host(b_out), b_ref) <= 1e-5, k


@pytest.mark.parametrize("dims", [(44, 26, 23), (88, 52, 34), (100, 98, 97)])
def test_register_prime_sizes(lib, dims):
    pair = synth.make_pair(dims, seed=3)
    u_ref = O.register(pair["fixed"], pair["moving"], lam=10.0, theta=0.1, n=2, outer=2, inner=4)
    reg = lib.Registration(dims, device=DEV, order_n=2, lam=10.0, theta=0.1, outer=2, inner=4)
    u = reg.register(dev(pair["fixed"]), dev(pair["moving"]))
    assert lib.nadmm_get_status(reg.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    assert np.abs(host(u) - u_ref).max() <= 1e-3


def test_batched_mixes_prime_and_smooth_sizes(lib):
    """A batch with prime-factor and smooth grids: each pair as the oracle."""
    dims = [(32, 32, 24), (44, 26, 23), (20, 22, 143)]
    pairs = [synth.make_pair(d, seed=7 + i) for i, d in enumerate(dims)]
    b = lib.BatchedRegistration(dims, device=DEV, order_n=2, lam=10.0, theta=0.1, outer=2,
                                inner=3)
    us = b.register([dev(p["fixed"]) for p in pairs], [dev(p["moving"]) for p in pairs])
    for p, d, u in zip(pairs, dims, us):
        ref = O.register(p["fixed"], p["moving"], lam=10.0, theta=0.1, n=2, outer=2, inner=3)
        assert np.abs(host(u) - ref).max() <= 1e-3, d


def test_backward_prime_size(lib):
    """Reverse mode on a grid with prime factors 11, 13, 23: the adjoint's
    spectral solves run the same generic stages."""
    dims = (44, 26, 23)
    p = synth.make_pair(dims, seed=8)
    gu = synth.random_field((3,) + dims[::-1], seed=48)
    kw = dict(lam=10.0, theta=0.1, n=2, outer=2, inner=4, kappa=0.5, delta=1.0)
    reg = lib.Registration(dims, device=DEV, requires_grad=True, order_n=2, lam=10.0, theta=0.1,
                           outer=2, inner=4, kappa=0.5, delta=1.0)
    f, m = dev(p["fixed"]), dev(p["moving"])
    u = reg.register(f, m)
    u_ref, _ = O.register_tape(p["fixed"], p["moving"], **kw)
    assert np.abs(host(u) - u_ref).max() <= 1e-3
    g0, g1, gl, gt = reg.backward(f, m, dev(gu))
    r0, r1, rl, rt = O.register_vjp(p["fixed"], p["moving"], gu, **kw)
    assert rel_l2(host(g0), r0) <= 1e-4
    assert rel_l2(host(g1), r1) <= 1e-4
    assert abs(float(gl) - rl) <= 1e-4 * abs(rl) + 1e-7
    assert abs(float(gt) - rt) <= 1e-4 * abs(rt) + 1e-7


def test_pyramid_prime_size(lib):
    """Three levels 44 x 26 x 22 -> 88 x 52 x 44 -> 176 x 104 x 88 (factors
    11 and 13 on every level), short schedule."""
    dims = (176, 104, 88)
    p = synth.make_pair(dims, seed=9)
    outer, inner = (2, 2, 1), (3, 3, 2)
    reg = lib.PyramidRegistration(dims, outer=outer, inner=inner, device=DEV, order_n=2)
    u = reg.register(dev(p["fixed"]), dev(p["moving"]))
    assert lib.nadmm_get_status(reg.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    ref = O.register_pyramid(p["fixed"], p["moving"], outer=outer, inner=inner, lam=10.0,
                             theta=0.1, n=2)
    assert np.abs(host(u) - ref).max() <= 1e-3
