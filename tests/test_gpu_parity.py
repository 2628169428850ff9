"""CUDA path vs FP64 oracle, element by element, on seeded synthetic inputs.

Every call goes through the C ABI (libnadmm.so via the ctypes binding).
Tolerances: per ADMM iterate (teacher-forced: the GPU starts from the
oracle's state) relative L2 <= 1e-5; final deformation after a fixed
iteration count max |u_gpu - u_oracle| <= 1e-3 voxel; spectral solve and
grid operations at FP32 rounding level.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2109_12688_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2109_12688_gb300 import nadmm
    return nadmm


DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def empty(shape):
    return torch.empty(shape, dtype=torch.float32, device=DEV)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-30))


def position_tol(dims, f):
    """Bound for sampling f at x + u computed in FP32: the position carries a
    rounding error <= ulp(max dim) / 2 = 2^-24 * 2^ceil(log2(max dim)), times
    the largest neighbour difference of f, doubled, plus FP32 arithmetic."""
    f = np.asarray(f, np.float64)
    slope = max(np.abs(np.diff(f, axis=a)).max() for a in range(f.ndim))
    return 2.0 * 2.0 ** -24 * 2.0 ** math.ceil(math.log2(max(dims))) * slope + 1e-6


def smooth_field(dims, seed, amp):
    v = synth.random_velocity(dims, np.random.default_rng(seed), max_amp=amp)
    return v.astype(np.float32)


# ------------------------------------------------------------------ a3
@pytest.mark.parametrize("dims", [(32, 32, 24), (20, 12, 14), (4, 4, 4), (12, 6, 7),
                                  (128, 128, 96), (160, 160, 112), (96, 112, 80)])
@pytest.mark.parametrize("n", [1, 2, 3])
def test_spectral_solve(lib, dims, n):
    nx, ny, nz = dims
    lam, theta = 10.0, 0.1
    reg = lib.Registration(dims, device=DEV, order_n=n, lam=lam, theta=theta)
    y = synth.random_field((3, nz, ny, nx), seed=n)
    w = empty((3, nz, ny, nx))
    lib.nadmm_spectral_solve(reg.handle, dev(y), w, torch.cuda.current_stream())
    ref = O.spectral_solve(y, lam, theta, n)
    got = host(w)
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(y).max()
    assert rel_l2(got, ref) <= 1e-6


# ------------------------------------------------------------------ a1-a5
def _phantom_linearisation(dims, seed):
    p = synth.make_pair(dims, seed)
    J, c, _ = O.linearise(p["fixed"], p["moving"], np.zeros((3,) + p["fixed"].shape))
    return J.astype(np.float32), c.astype(np.float32)


@pytest.mark.parametrize("s", [2, 1])
@pytest.mark.parametrize("dims", [(32, 32, 24), (20, 12, 14)])
def test_admm_iterates_teacher_forced(lib, s, dims):
    """Each iterate k of Eq. 5 from the oracle's state after k-1."""
    nx, ny, nz = dims
    lam, theta, n, K = 10.0, 0.1, 2, 10
    J, c = _phantom_linearisation(dims, seed=3)
    hist = O.admm(J, c, lam, theta, n, K, s=s, history=True)
    reg = lib.Registration(dims, device=DEV, order_n=n, lam=lam, theta=theta, data_term=s)
    Jd, cd = dev(J), dev(c)
    shape = (3, nz, ny, nx)
    zero = np.zeros(shape, np.float32)
    w_out, b_out = empty(shape), empty(shape)
    for k in range(K):
        wk1, bk1 = hist[k - 1] if k >= 1 else (zero, zero)
        wk2, bk2 = hist[k - 2] if k >= 2 else (zero, zero)
        lib.nadmm_admm_run(reg.handle, Jd, cd, dev(wk1), dev(wk2), dev(bk1), dev(bk2), k, 1,
                           w_out, b_out, torch.cuda.current_stream())
        w_ref, b_ref = hist[k]
        assert rel_l2(host(w_out), w_ref) <= 1e-5, k
        assert rel_l2(host(b_out), b_ref) <= 1e-5, k


@pytest.mark.parametrize("s", [2, 1])
def test_admm_free_running(lib, s):
    dims = (32, 32, 24)
    nx, ny, nz = dims
    lam, theta, n, K = 10.0, 0.1, 3, 10
    J, c = _phantom_linearisation(dims, seed=4)
    w_ref, b_ref = O.admm(J, c, lam, theta, n, K, s=s, history=True)[-1]
    reg = lib.Registration(dims, device=DEV, order_n=n, lam=lam, theta=theta, data_term=s)
    shape = (3, nz, ny, nx)
    w_out, b_out = empty(shape), empty(shape)
    z = torch.zeros(shape, device=DEV)
    lib.nadmm_admm_run(reg.handle, dev(J), dev(c), z, z, z, z, 0, K, w_out, b_out,
                       torch.cuda.current_stream())
    assert rel_l2(host(w_out), w_ref) <= 1e-5
    assert rel_l2(host(b_out), b_ref) <= 1e-5


def test_admm_resumes_mid_sequence(lib):
    """Starting at k = 4 from the oracle state and running 5 steps equals
    the oracle's iterate 8 (checks the beta index across launches)."""
    dims = (32, 32, 24)
    nx, ny, nz = dims
    J, c = _phantom_linearisation(dims, seed=5)
    hist = O.admm(J, c, 10.0, 0.1, 2, 9, history=True)
    reg = lib.Registration(dims, device=DEV, order_n=2, lam=10.0, theta=0.1)
    shape = (3, nz, ny, nx)
    w_out, b_out = empty(shape), empty(shape)
    lib.nadmm_admm_run(reg.handle, dev(J), dev(c), dev(hist[3][0]), dev(hist[2][0]),
                       dev(hist[3][1]), dev(hist[2][1]), 4, 5, w_out, b_out,
                       torch.cuda.current_stream())
    assert rel_l2(host(w_out), hist[8][0]) <= 1e-5
    assert rel_l2(host(b_out), hist[8][1]) <= 1e-5


# ------------------------------------------------------------------ a6-a8
@pytest.mark.parametrize("dims", [(32, 32, 24), (128, 128, 96), (20, 12, 14)])
def test_linearise(lib, dims):
    nx, ny, nz = dims
    p = synth.make_pair(dims, seed=7)
    u = smooth_field(dims, 8, amp=2.5)
    reg = lib.Registration(dims, device=DEV)
    J, c, I1w = empty((3, nz, ny, nx)), empty((nz, ny, nx)), empty((nz, ny, nx))
    lib.nadmm_linearise(reg.handle, dev(p["fixed"]), dev(p["moving"]), dev(u), J, c, I1w,
                        torch.cuda.current_stream())
    J_ref, c_ref, I1w_ref = O.linearise(p["fixed"], p["moving"], u.astype(np.float64))
    tol = position_tol(dims, p["moving"])
    assert np.abs(host(I1w) - I1w_ref).max() <= tol
    assert np.abs(host(c) - c_ref).max() <= tol
    assert np.abs(host(J) - J_ref).max() <= tol


@pytest.mark.parametrize("kappa,delta", [(0.5, 1.0), (math.inf, math.inf), (0.05, 0.3)])
def test_bound_compose(lib, kappa, delta):
    dims = (32, 32, 24)
    nx, ny, nz = dims
    w = smooth_field(dims, 9, amp=1.7)
    u = smooth_field(dims, 10, amp=2.0)
    reg = lib.Registration(dims, device=DEV, kappa=kappa, delta=delta)
    u_out, sc = empty((3, nz, ny, nx)), empty((1,))
    lib.nadmm_bound_compose(reg.handle, dev(w), dev(u), u_out, sc, torch.cuda.current_stream())
    s_ref, _, _ = O.bound_scale(w.astype(np.float64), kappa, delta)
    assert float(host(sc)[0]) == pytest.approx(s_ref, rel=1e-6)
    ref = O.compose(u.astype(np.float64), s_ref * w.astype(np.float64))
    tol = max(position_tol(dims, u[i]) for i in range(3)) + 1e-6 * np.abs(w).max()
    assert np.abs(host(u_out) - ref).max() <= tol


@pytest.mark.parametrize("dims", [(40, 20, 13), (36, 18, 9), (128, 128, 96)])
@pytest.mark.parametrize("kappa,delta,amp", [(0.5, 1.0, 1.7), (math.inf, math.inf, 0.9),
                                             (math.inf, math.inf, 2.5)])
def test_compose_ragged_grids(lib, dims, kappa, delta, amp):
    """Bound and compose on grids with partial 32 x 8 tiles, for steps within
    one voxel (first two cases) and beyond it (third)."""
    nx, ny, nz = dims
    w = smooth_field(dims, 11, amp=amp)
    u = smooth_field(dims, 12, amp=2.0)
    reg = lib.Registration(dims, device=DEV, kappa=kappa, delta=delta)
    u_out, sc = empty((3, nz, ny, nx)), empty((1,))
    lib.nadmm_bound_compose(reg.handle, dev(w), dev(u), u_out, sc, torch.cuda.current_stream())
    s_ref, _, _ = O.bound_scale(w.astype(np.float64), kappa, delta)
    ref = O.compose(u.astype(np.float64), s_ref * w.astype(np.float64))
    tol = max(position_tol(dims, u[i]) for i in range(3)) + 1e-6 * np.abs(w).max()
    assert np.abs(host(u_out) - ref).max() <= tol


def test_jacobian_det(lib):
    dims = (32, 32, 24)
    nx, ny, nz = dims
    u = smooth_field(dims, 11, amp=2.0)
    reg = lib.Registration(dims, device=DEV)
    det = empty((nz, ny, nx))
    cnt = torch.zeros(1, dtype=torch.int32, device=DEV)
    lib.nadmm_jacobian_det(reg.handle, dev(u), det, cnt, torch.cuda.current_stream())
    ref = O.jacobian_determinant(u.astype(np.float64))
    assert np.abs(host(det) - ref).max() <= 1e-5
    assert int(cnt.item()) == int((ref <= 0).sum())


# ------------------------------------------------------------------ whole path
def _register_gpu(lib, pair, dims, **kw):
    reg = lib.Registration(dims, device=DEV, **kw)
    u = reg.register(dev(pair["fixed"]), dev(pair["moving"]))
    st = lib.nadmm_get_status(reg.handle, torch.cuda.current_stream())
    assert st == lib.NADMM_OK
    return host(u), reg


def _nonpositive(lib, reg, u):
    cnt = torch.zeros(1, dtype=torch.int32, device=DEV)
    lib.nadmm_jacobian_det(reg.handle, dev(u), None, cnt, torch.cuda.current_stream())
    return int(cnt.item())


@pytest.mark.parametrize("seed", range(10))
def test_register_32x32x24_n2(lib, seed):
    dims = (32, 32, 24)
    pair = synth.make_pair(dims, seed)
    kw = dict(lam=10.0, theta=0.1, n=2, outer=5, inner=10)
    u_ref = O.register(pair["fixed"], pair["moving"], **kw)
    u, reg = _register_gpu(lib, pair, dims, order_n=2, lam=10.0, theta=0.1, outer=5, inner=10)
    assert np.abs(u - u_ref).max() <= 1e-3
    assert O.jacobian_determinant(u_ref).min() > 0
    assert _nonpositive(lib, reg, u) == 0


@pytest.mark.parametrize("seed,n", [(0, 1), (1, 3)])
def test_register_32x32x24_l1(lib, seed, n):
    dims = (32, 32, 24)
    pair = synth.make_pair(dims, seed)
    u_ref = O.register(pair["fixed"], pair["moving"], lam=10.0, theta=0.1, n=n, outer=5,
                       inner=10, s=1)
    u, reg = _register_gpu(lib, pair, dims, order_n=n, lam=10.0, theta=0.1, outer=5, inner=10,
                           data_term=1)
    assert np.abs(u - u_ref).max() <= 1e-3
    assert _nonpositive(lib, reg, u) == 0


@pytest.mark.parametrize("n", [1, 2, 3])
def test_register_128x128x96_short_schedule(lib, n):
    """Full-size grid, same kernels and launch shapes as the benchmark,
    2 compositions x 5 ADMM iterations so the oracle stays in seconds."""
    dims = (128, 128, 96)
    pair = synth.make_pair(dims, seed=n)
    u_ref = O.register(pair["fixed"], pair["moving"], lam=10.0, theta=0.1, n=n, outer=2, inner=5)
    u, _ = _register_gpu(lib, pair, dims, order_n=n, lam=10.0, theta=0.1, outer=2, inner=5)
    assert np.abs(u - u_ref).max() <= 1e-3


def test_register_128x128x96_full_schedule_properties(lib):
    """The benchmarked schedule (10 x 10): diffeomorphic and SSD-reducing."""
    dims = (128, 128, 96)
    pair = synth.make_pair(dims, seed=0)
    u, reg = _register_gpu(lib, pair, dims, order_n=2, lam=10.0, theta=0.1, outer=10, inner=10)
    assert _nonpositive(lib, reg, u) == 0
    warped = O.warp(pair["moving"], u)
    ssd0 = ((pair["moving"].astype(float) - pair["fixed"]) ** 2).sum()
    assert ((warped - pair["fixed"]) ** 2).sum() < 0.7 * ssd0


@pytest.mark.parametrize("dims", [(160, 160, 112), (96, 96, 64), (20, 12, 14), (12, 6, 7),
                                  (4, 4, 4)])
def test_register_edge_sizes(lib, dims):
    pair = synth.make_pair(dims, seed=2)
    u_ref = O.register(pair["fixed"], pair["moving"], lam=10.0, theta=0.1, n=2, outer=2, inner=3)
    u, _ = _register_gpu(lib, pair, dims, order_n=2, lam=10.0, theta=0.1, outer=2, inner=3)
    assert np.abs(u - u_ref).max() <= 1e-3


def test_single_iteration_schedule(lib):
    dims = (32, 32, 24)
    pair = synth.make_pair(dims, seed=6)
    u_ref = O.register(pair["fixed"], pair["moving"], lam=5.0, theta=0.05, n=1, outer=1, inner=1)
    u, _ = _register_gpu(lib, pair, dims, order_n=1, lam=5.0, theta=0.05, outer=1, inner=1)
    assert np.abs(u - u_ref).max() <= 1e-4


def test_identical_images_give_zero(lib):
    dims = (32, 32, 24)
    pair = synth.make_pair(dims, seed=1)
    same = dict(pair, moving=pair["fixed"])
    u, _ = _register_gpu(lib, same, dims, outer=3, inner=5)
    assert np.all(u == 0.0)


def test_translation_recovered(lib):
    dims = (24, 20, 16)
    shift = (0.6, -0.4, 0.3)
    I0, I1 = synth.translated_blob_pair(dims, shift, sigma_frac=0.25)
    u, _ = _register_gpu(lib, {"fixed": I0, "moving": I1}, dims, order_n=1, lam=10.0,
                         theta=0.02, outer=10, inner=30)
    np.testing.assert_allclose(u[:, 8, 10, 12], -np.array(shift), atol=0.01)


def test_graph_direct_host_paths_agree_and_repeat(lib):
    dims = (32, 32, 24)
    nx, ny, nz = dims
    pair = synth.make_pair(dims, seed=5)
    I0, I1 = dev(pair["fixed"]), dev(pair["moving"])
    a = lib.Registration(dims, device=DEV, outer=3, inner=6)
    b = lib.Registration(dims, device=DEV, outer=3, inner=6, flags=lib.NADMM_FLAG_NO_GRAPH)
    u1 = host(a.register(I0, I1))
    u2 = host(a.register(I0, I1))
    u3 = host(b.register(I0, I1))
    assert np.array_equal(u1, u2) and np.array_equal(u1, u3)
    hf = torch.from_numpy(pair["fixed"]).pin_memory()
    hm = torch.from_numpy(pair["moving"]).pin_memory()
    hu = torch.empty((3, nz, ny, nx), dtype=torch.float32).pin_memory()
    lib.nadmm_register_host(a.handle, hf, hm, hu, torch.cuda.current_stream())
    assert np.array_equal(hu.numpy().astype(np.float64), u1)
    prof = lib.nadmm_register_profiled(a.handle, I0, I1, empty((3, nz, ny, nx)),
                                       torch.cuda.current_stream())
    # 24 z-planes fill a small part of the GPU: four kernels per ADMM iteration
    assert prof["plane"][1] == 3 * 4 and prof["pencil"][1] == 3 * 6
    assert prof["plane_first"][1] == 3 and prof["plane_final"][1] == 3
    assert prof["slab"][1] == 0 and prof["zslab"][1] == 0
    assert all(ms >= 0 for ms, _ in prof.values())
    slab = lib.Registration(dims, device=DEV, outer=3, inner=6, flags=lib.NADMM_FLAG_SLAB_PATH)
    prof = lib.nadmm_register_profiled(slab.handle, I0, I1, empty((3, nz, ny, nx)),
                                       torch.cuda.current_stream())
    assert prof["slab"][1] == 3 * 4 and prof["zslab"][1] == 3 * 6
    assert prof["slab_first"][1] == 3 and prof["slab_final"][1] == 3


def test_nonfinite_input_sets_status(lib):
    dims = (32, 32, 24)
    pair = synth.make_pair(dims, seed=1)
    bad = pair["moving"].copy()
    bad[12, 16, 16] = np.nan
    reg = lib.Registration(dims, device=DEV, outer=2, inner=2)
    reg.register(dev(pair["fixed"]), dev(bad))
    assert lib.nadmm_get_status(reg.handle, torch.cuda.current_stream()) == lib.NADMM_ERR_NONFINITE
    # the status word is cleared by the read, and a clean call reports OK
    reg.register(dev(pair["fixed"]), dev(pair["moving"]))
    assert lib.nadmm_get_status(reg.handle, torch.cuda.current_stream()) == lib.NADMM_OK


@pytest.mark.parametrize("attempts", [1, 4096])
def test_expired_wait_sets_timeout_and_context_survives(lib, attempts):
    """A bounded mbarrier wait that nothing completes reports
    NADMM_ERR_TIMEOUT through the status word; the next registration on the
    same context runs and matches the oracle."""
    dims = (32, 32, 24)
    reg = lib.Registration(dims, device=DEV, outer=2, inner=3)
    lib.nadmm_selftest_wait_timeout(reg.handle, attempts, torch.cuda.current_stream())
    assert lib.nadmm_get_status(reg.handle, torch.cuda.current_stream()) == lib.NADMM_ERR_TIMEOUT
    assert lib.nadmm_get_status(reg.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    pair = synth.make_pair(dims, seed=6)
    u = host(reg.register(dev(pair["fixed"]), dev(pair["moving"])))
    assert lib.nadmm_get_status(reg.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    ref = O.register(pair["fixed"], pair["moving"], lam=10.0, theta=0.1, n=2, outer=2, inner=3)
    assert np.abs(u - ref).max() <= 1e-3


# ------------------------------------------------------------------ 256 x 256 x 192
LARGE = (256, 256, 192)


@pytest.fixture(scope="module")
def large_pair():
    return synth.phase_pair(LARGE, seed=0)


def test_large_spectral_solve_n3(lib):
    nx, ny, nz = LARGE
    reg = lib.Registration(LARGE, device=DEV, order_n=3)
    y = synth.random_field((3, nz, ny, nx), seed=5)
    w = empty((3, nz, ny, nx))
    lib.nadmm_spectral_solve(reg.handle, dev(y), w, torch.cuda.current_stream())
    ref = O.spectral_solve(y, 10.0, 0.1, 3)
    got = host(w)
    assert rel_l2(got, ref) <= 1e-6
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(y).max()


def test_large_register_short_schedule_n3(lib, large_pair):
    fixed, moving = large_pair
    u_ref = O.register(fixed, moving, lam=10.0, theta=0.1, n=3, outer=1, inner=3)
    reg = lib.Registration(LARGE, device=DEV, order_n=3, outer=1, inner=3)
    u = host(reg.register(dev(fixed), dev(moving)))
    assert np.abs(u - u_ref).max() <= 1e-3


def test_large_register_full_schedule_n3(lib, large_pair):
    """256 x 256 x 192, n = 3, 10 x 10: no folds, lower SSD, and the device
    memory it needs (workspace + inputs + output) stays below 2 GB."""
    fixed, moving = large_pair
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    base = torch.cuda.memory_allocated()
    reg = lib.Registration(LARGE, device=DEV, order_n=3, outer=10, inner=10)
    f, m = dev(fixed), dev(moving)
    u = reg.register(f, m)
    assert lib.nadmm_get_status(reg.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    torch.cuda.synchronize()
    peak = torch.cuda.max_memory_allocated() - base
    assert peak < 2 * 1024 ** 3
    assert torch.isfinite(u).all()
    cnt = torch.zeros(1, dtype=torch.int32, device=DEV)
    lib.nadmm_jacobian_det(reg.handle, u, None, cnt, torch.cuda.current_stream())
    assert int(cnt.item()) == 0
    warped = O.warp(moving, host(u))
    ssd0 = ((moving.astype(float) - fixed) ** 2).sum()
    assert ((warped - fixed) ** 2).sum() < ssd0


@pytest.mark.parametrize("seed,n", [(0, 1), (1, 2), (2, 3)])
def test_register_128x128x96_label_metrics(lib, seed, n):
    """The paper's measures on the synthetic labels (Sec. 4): after the
    10 x 10 registration the warped source labels overlap the target labels
    better (mean Dice over LV, LVM, RV), lie closer (mean per-slice
    Hausdorff) and no voxel folds."""
    dims = (128, 128, 96)
    pair = synth.make_pair(dims, seed=seed)
    u, reg = _register_gpu(lib, pair, dims, order_n=n, lam=10.0, theta=0.1, outer=10, inner=10)
    fixed_lab, moving_lab = pair["labels_fixed"], pair["labels_moving"]
    warped = O.warp_labels(moving_lab, u)
    d0 = np.mean([O.dice(moving_lab, fixed_lab, k) for k in (1, 2, 3)])
    d1 = np.mean([O.dice(warped, fixed_lab, k) for k in (1, 2, 3)])
    h0 = np.mean([O.hausdorff_per_slice(moving_lab, fixed_lab, k) for k in (1, 2, 3)])
    h1 = np.mean([O.hausdorff_per_slice(warped, fixed_lab, k) for k in (1, 2, 3)])
    assert d1 > d0
    assert h1 < h0
    assert O.nonpositive_jacobian_percent(u) == 0.0
