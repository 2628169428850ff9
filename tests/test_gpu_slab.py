"""The two-kernel slab path of the ADMM iteration against the four-kernel
path and the FP64 oracle.

Both paths compute Eq. 5 / Eq. 6 with the same arithmetic in a different
rounding order: the slab path transforms whole z-planes (x- and y-DFTs, the
x-DFT as a half-length complex DFT) in a cluster of three CTAs and runs one
z-pass; NADMM_FLAG_FOUR_PASS forces the plane pass + y/z/y passes.  Every
call goes through the C ABI.
"""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _classes(lib, reg, pair):
    u = torch.empty((3,) + tuple(reversed(reg.dims)), device="cuda:0")
    prof = lib.nadmm_register_profiled(reg.handle, _dev(pair["fixed"]), _dev(pair["moving"]), u,
                                       torch.cuda.current_stream())
    return {k: n for k, (_, n) in prof.items() if n > 0}


@pytest.mark.parametrize("dims,default,eligible", [((128, 128, 96), True, True),
                                                   ((32, 32, 24), False, True),
                                                   ((160, 160, 112), True, True),
                                                   ((96, 112, 80), True, True),
                                                   ((20, 12, 14), False, False),
                                                   ((256, 256, 192), False, False)])
def test_path_selection(lib, dims, default, eligible):
    """Grids whose planes fit a CTA and whose axes have lane plans can take
    the slab path (two kernels per iteration): by default when their
    three-CTA clusters fill at least 80 % of the device's waves (96 z-planes
    on 97 resident clusters at 128 x 128 x 96, 80 of 97 at 96 x 112 x 80,
    24 of several hundred at 32 x 32 x 24; 112 z-planes of 160 x 160 one CTA
    per SM: 3 waves, 81 %), always with NADMM_FLAG_SLAB_PATH; the
    four-kernel flag keeps the plane pass and its y/z/y passes."""
    pair = synth.make_pair(dims, seed=1) if max(dims) <= 160 else None
    if pair is None:
        f, m = synth.phase_pair(dims, seed=1)
        pair = {"fixed": f, "moving": m}

    def classes(flags):
        reg = lib.Registration(dims, device="cuda:0", outer=1, inner=4, flags=flags)
        return _classes(lib, reg, pair)

    for flags, slab in ((0, default), (lib.NADMM_FLAG_SLAB_PATH, eligible),
                        (lib.NADMM_FLAG_FOUR_PASS, False)):
        n = classes(flags)
        if slab:
            assert n.get("slab_first") == 1 and n.get("slab_k1") == 1 and n.get("slab") == 2
            assert n.get("zslab") == 4 and n.get("slab_final") == 1 and "plane" not in n
        else:
            assert "slab" not in n and n.get("plane") == 2, (flags, n)


@pytest.mark.parametrize("dims,n", [((128, 128, 96), 2), ((32, 32, 24), 1), ((96, 112, 80), 3),
                                    ((160, 160, 112), 2), ((64, 48, 48), 2)])
def test_slab_registration_matches_four_pass_and_oracle(lib, dims, n):
    pair = synth.make_pair(dims, seed=n + 3)
    kw = dict(order_n=n, lam=10.0, theta=0.1, outer=2, inner=6)
    I0, I1 = _dev(pair["fixed"]), _dev(pair["moving"])
    slab = lib.Registration(dims, device="cuda:0", flags=lib.NADMM_FLAG_SLAB_PATH,
                            **kw).register(I0, I1)
    four = lib.Registration(dims, device="cuda:0", flags=lib.NADMM_FLAG_FOUR_PASS,
                            **kw).register(I0, I1)
    torch.cuda.synchronize()
    a = slab.cpu().numpy().astype(np.float64)
    b = four.cpu().numpy().astype(np.float64)
    assert np.isfinite(a).all()
    assert np.abs(a - b).max() <= 1e-4
    ref = O.register(pair["fixed"], pair["moving"], lam=10.0, theta=0.1, n=n, outer=2, inner=6)
    assert np.abs(a - ref).max() <= 1e-3


@pytest.mark.parametrize("dims", [(128, 128, 96), (32, 32, 24), (96, 112, 80), (160, 160, 112),
                                  (64, 48, 48)])
@pytest.mark.parametrize("n", [1, 3])
def test_slab_spectral_solve_matches_oracle(lib, dims, n):
    """The w-step alone (Eq. 6 last line) through the slab kernels: forward
    x/y DFTs of a field, the z-pass, the inverse x/y DFTs."""
    nx, ny, nz = dims
    y = synth.random_field((3, nz, ny, nx), seed=7 + n)
    reg = lib.Registration(dims, device="cuda:0", order_n=n, lam=10.0, theta=0.1,
                           flags=lib.NADMM_FLAG_SLAB_PATH)
    yd = _dev(y)
    w = torch.full_like(yd, float("nan"))
    lib.nadmm_spectral_solve(reg.handle, yd, w, torch.cuda.current_stream())
    torch.cuda.synchronize()
    got = w.cpu().numpy().astype(np.float64)
    ref = O.spectral_solve(y, 10.0, 0.1, n)
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(y).max()


@pytest.mark.parametrize("k", [0, 1, 2, 5])
def test_slab_teacher_forced_iterate(lib, k):
    """One ADMM iteration from a given state (nadmm_admm_run, slab STATE
    modes) against the oracle's admm_step: relative L2 <= 1e-5."""
    dims = (128, 128, 96)
    nx, ny, nz = dims
    J, c = synth.random_linearisation(dims, seed=30 + k)
    shape = (3, nz, ny, nx)
    st = [synth.random_field(shape, seed=40 + k + i, scale=0.3) for i in range(4)]
    reg = lib.Registration(dims, device="cuda:0", order_n=2, lam=10.0, theta=0.1, inner=12,
                           flags=lib.NADMM_FLAG_SLAB_PATH)
    _, beta = O.nesterov_sequence(12)
    bk = 0.0 if k == 0 else beta[k - 1]
    zero = np.zeros(shape)
    w1, w2, b1, b2 = (st if k >= 2 else (st[0], zero, st[2], zero)) if k >= 1 else (zero,) * 4
    w_ref, b_ref, _ = O.admm_step(w1, w2, b1, b2, bk, J, c, 10.0, 0.1, 2)
    w_out, b_out = torch.empty(shape, device="cuda:0"), torch.empty(shape, device="cuda:0")
    args = [_dev(w1), _dev(w2), _dev(b1), _dev(b2)]
    lib.nadmm_admm_run(reg.handle, _dev(J), _dev(c), *args, k, 1, w_out, b_out,
                       torch.cuda.current_stream())
    torch.cuda.synchronize()
    for got, ref in ((w_out, w_ref), (b_out, b_ref)):
        g = got.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(g - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("dims", [(128, 128, 96), (64, 48, 48), (96, 112, 80)])
def test_two_planes_per_cluster_is_the_same_pass(lib, dims):
    """NADMM_FLAG_SLAB_PAIRS: every cluster takes two z-planes in turn (half
    the clusters; an odd plane count leaves one cluster a single plane); the
    arithmetic per plane is unchanged, so the registrations are bit-identical,
    with and without adaptive restart."""
    pair = synth.make_pair(dims, seed=21)
    I0, I1 = _dev(pair["fixed"]), _dev(pair["moving"])
    for extra in ({}, {"restart_eta": 0.999, "theta": 0.02}):
        kw = dict(order_n=2, outer=2, inner=8, **extra)
        a = lib.Registration(dims, device="cuda:0", flags=lib.NADMM_FLAG_SLAB_PATH,
                             **kw).register(I0, I1)
        b = lib.Registration(dims, device="cuda:0", flags=lib.NADMM_FLAG_SLAB_PAIRS,
                             **kw).register(I0, I1)
        torch.cuda.synchronize()
        assert torch.equal(a, b), extra
