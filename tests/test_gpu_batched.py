"""Batched registration of pairs with different grid sizes (one CUDA graph
with concurrent lanes) against the single-pair path and the FP64 oracle.

The batched handle runs exactly the kernels of nadmm_register on each pair,
so its results are compared bit for bit with single-pair calls; the oracle
comparison (max |du| <= 1e-3 voxel) covers the small pairs."""
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


def single(lib, dims, fixed, moving, **kw):
    reg = lib.Registration(dims, device=DEV, **kw)
    u = reg.register(fixed, moving)
    assert lib.nadmm_get_status(reg.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    out = u.cpu().numpy()
    reg.close()
    return out


SMALL = [(32, 32, 24), (20, 12, 14), (16, 20, 12), (12, 6, 7), (24, 24, 20), (8, 10, 9)]
KW = dict(order_n=2, lam=10.0, theta=0.1, outer=2, inner=4)


def small_pairs():
    return [synth.make_pair(d, seed=10 + i) for i, d in enumerate(SMALL)]


def test_batched_small_matches_oracle_and_single(lib):
    pairs = small_pairs()
    fixed = [dev(p["fixed"]) for p in pairs]
    moving = [dev(p["moving"]) for p in pairs]
    breg = lib.BatchedRegistration(SMALL, device=DEV, **KW)
    us = breg.register(fixed, moving)
    assert lib.nadmm_get_status(breg.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    for d, p, f, m, u in zip(SMALL, pairs, fixed, moving, us):
        got = u.cpu().numpy()
        ref = O.register(p["fixed"], p["moving"], lam=10.0, theta=0.1, n=2, outer=2, inner=4)
        assert np.abs(got - ref).max() <= 1e-3, d
        assert np.array_equal(got, single(lib, d, f, m, **KW)), d


@pytest.mark.parametrize("lanes,flags", [(1, 0), (3, 0), (6, 0), (2, 1)])
def test_batched_lanes_and_direct_launch_agree(lib, lanes, flags):
    pairs = small_pairs()
    fixed = [dev(p["fixed"]) for p in pairs]
    moving = [dev(p["moving"]) for p in pairs]
    ref = lib.BatchedRegistration(SMALL, device=DEV, **KW).register(fixed, moving)
    breg = lib.BatchedRegistration(SMALL, device=DEV, lanes=lanes, flags=flags, **KW)
    for _ in range(2):  # second call replays the captured graph
        us = breg.register(fixed, moving)
        for a, b in zip(us, ref):
            assert torch.equal(a, b)


def test_batched_recaptures_on_new_pointers(lib):
    pairs = small_pairs()
    fixed = [dev(p["fixed"]) for p in pairs]
    moving = [dev(p["moving"]) for p in pairs]
    breg = lib.BatchedRegistration(SMALL, device=DEV, **KW)
    a = [t.clone() for t in breg.register(fixed, moving)]
    swapped = breg.register(moving, fixed)  # new pointer set: re-captured graph
    b = breg.register(fixed, moving)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    for d, f, m, s in zip(SMALL, fixed, moving, swapped):
        assert np.array_equal(s.cpu().numpy(), single(lib, d, m, f, **KW))


def test_batched_rejects_single_calls(lib):
    breg = lib.BatchedRegistration(SMALL[:2], device=DEV, **KW)
    y = torch.zeros((3, 24, 32, 32), device=DEV)
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_spectral_solve(breg.handle, y, y, torch.cuda.current_stream())
    assert e.value.status == lib.NADMM_ERR_INVALID_ARG
    with pytest.raises(lib.NadmmError):
        lib.nadmm_batch_set_lanes(breg.handle, 1)  # workspace already attached


def test_batch_of_64_uneven_pairs(lib):
    """64 pairs, nx, ny from {96..160}, nz from {64..112} (seed 1234), n = 2,
    10 x 10 iterations, one graph (two lanes, the pairs on the four-kernel
    path): bit-identical to 64 single-pair calls and free of folds."""
    dims = synth.draw_batch_dims(64, seed=1234)
    data = [synth.phase_pair(d, seed=i) for i, d in enumerate(dims)]
    fixed = [dev(f) for f, _ in data]
    moving = [dev(m) for _, m in data]
    kw = dict(order_n=2, lam=10.0, theta=0.1, outer=10, inner=10)
    breg = lib.BatchedRegistration(dims, device=DEV, **kw)
    us = breg.register(fixed, moving)
    assert lib.nadmm_get_status(breg.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    assert lib.nadmm_batch_get_lanes(breg.handle) == 2
    for i in range(0, 64, 9):  # a sample of the pairs through the single-pair four-kernel path
        assert np.array_equal(us[i].cpu().numpy(), single(lib, dims[i], fixed[i], moving[i],
                                                          flags=lib.NADMM_FLAG_FOUR_PASS, **kw))
    for d, u in zip(dims, us):
        reg = lib.Registration(d, device=DEV, **kw)
        cnt = torch.zeros(1, dtype=torch.int32, device=DEV)
        lib.nadmm_jacobian_det(reg.handle, u, None, cnt, torch.cuda.current_stream())
        assert int(cnt.item()) == 0, d
        assert torch.isfinite(u).all()
        reg.close()


# grids on the slab path, one of them (160 x 160 x 112) in the one-CTA-per-SM
# shared-memory class, so a flat batch runs two slab launches per phase
FLAT = [(32, 32, 24), (64, 48, 48), (160, 160, 112), (96, 112, 80), (48, 32, 24), (32, 32, 24)]


def test_flat_batch_equals_single_and_lane_runs(lib):
    """Flat execution (lane count 0: every ADMM phase one launch over all
    pairs, z-passes one launch per z plan): bit-identical to single-pair
    calls and to the per-pair lanes, with and without graph capture.  The
    default is two concurrent lanes."""
    pairs = [synth.make_pair(d, seed=70 + i) for i, d in enumerate(FLAT)]
    fixed = [dev(p["fixed"]) for p in pairs]
    moving = [dev(p["moving"]) for p in pairs]
    assert lib.nadmm_batch_get_lanes(lib.BatchedRegistration(FLAT, device=DEV, **KW).handle) == 2
    flat = lib.BatchedRegistration(FLAT, device=DEV, lanes=0, **KW)
    assert lib.nadmm_batch_get_lanes(flat.handle) == 0
    us = [u.clone() for u in flat.register(fixed, moving)]
    again = flat.register(fixed, moving)  # graph replay
    slab = lib.NADMM_FLAG_SLAB_PATH  # the per-pair runs on the same (slab) kernels
    lanes = lib.BatchedRegistration(FLAT, device=DEV, lanes=2, flags=slab, **KW).register(fixed,
                                                                                        moving)
    direct = lib.BatchedRegistration(FLAT, device=DEV, lanes=0, flags=lib.NADMM_FLAG_NO_GRAPH,
                                     **KW).register(fixed, moving)
    for i, d in enumerate(FLAT):
        assert torch.equal(us[i], again[i]), d
        assert torch.equal(us[i], lanes[i]), d
        assert torch.equal(us[i], direct[i]), d
        assert np.array_equal(us[i].cpu().numpy(),
                              single(lib, d, fixed[i], moving[i], flags=slab, **KW)), d
    ref = O.register(pairs[1]["fixed"], pairs[1]["moving"], lam=10.0, theta=0.1, n=2, outer=2,
                     inner=4)
    assert np.abs(us[1].cpu().numpy() - ref).max() <= 1e-3


def test_flat_batch_with_restart_equals_single(lib):
    kw = dict(order_n=2, lam=10.0, theta=0.02, outer=2, inner=16, restart_eta=0.999)
    dims = [FLAT[0], FLAT[1], FLAT[4]]
    pairs = [synth.make_pair(d, seed=80 + i) for i, d in enumerate(dims)]
    fixed = [dev(p["fixed"]) for p in pairs]
    moving = [dev(p["moving"]) for p in pairs]
    for lanes in (0, 2):  # flat, and lanes (restart keeps every pair on the slab path)
        us = lib.BatchedRegistration(dims, device=DEV, lanes=lanes, **kw).register(fixed, moving)
        for i, d in enumerate(dims):
            assert np.array_equal(us[i].cpu().numpy(),
                                  single(lib, d, fixed[i], moving[i], **kw)), (lanes, d)


def test_flat_needs_slab_pairs(lib):
    b = lib.nadmm_create_batched(lib.make_config(SMALL[0]), SMALL)
    assert lib.nadmm_batch_get_lanes(b) == 2  # a pair off the slab path: lanes by default
    with pytest.raises(lib.NadmmError):
        lib.nadmm_batch_set_lanes(b, 0)
    lib.nadmm_destroy(b)


def test_four_kernel_lanes_equal_single_calls_with_per_pair_orders(lib):
    """The bench's batched leg on the four-kernel path: three 128x128x96 pairs
    with regulariser orders 1, 2, 3 on three concurrent lanes give the
    single four-kernel calls' displacements bit for bit."""
    dims = (128, 128, 96)
    pairs = [synth.make_pair(dims, seed=n) for n in (1, 2, 3)]
    fixed = [dev(p["fixed"]) for p in pairs]
    moving = [dev(p["moving"]) for p in pairs]
    kw = dict(lam=10.0, theta=0.1, outer=2, inner=5, flags=lib.NADMM_FLAG_FOUR_PASS)
    breg = lib.BatchedRegistration([dims] * 3, device=DEV, lanes=3,
                                   per_pair=[{"order_n": n} for n in (1, 2, 3)], **kw)
    assert lib.nadmm_batch_get_lanes(breg.handle) == 3
    us = breg.register(fixed, moving)
    assert lib.nadmm_get_status(breg.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    for n, f, m, u in zip((1, 2, 3), fixed, moving, us):
        assert np.array_equal(u.cpu().numpy(), single(lib, dims, f, m, order_n=n, **kw)), n
