"""FFT plan choices and the autotuner: every lane split of a 96x96x64 grid
(x, y: 12 x 8 or 6 x 16; z: 8 x 8 or 4 x 16) solves the regulariser step like
the FP64 oracle, nadmm_autotune returns one of them, and a registration with
the tuned plan matches the oracle; the JSON cache is written and reused."""
import itertools
import json

import numpy as np
import pytest

import oracle as O
from paper_2109_12688_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"
DIMS = (96, 96, 64)


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


@pytest.mark.parametrize("combo", list(itertools.product((8, 16), repeat=3)))
@pytest.mark.parametrize("four", [False, True])
def test_every_plan_solves_like_the_oracle(lib, combo, four):
    flags = lib.NADMM_FLAG_FOUR_PASS if four else 0
    for ax, r2 in enumerate(combo):
        flags |= lib.NADMM_FLAG_LANE8(ax) if r2 == 8 else lib.NADMM_FLAG_LANE16(ax)
    nx, ny, nz = DIMS
    reg = lib.Registration(DIMS, device=DEV, order_n=2, flags=flags)
    y = synth.random_field((3, nz, ny, nx), seed=sum(combo))
    w = torch.empty((3, nz, ny, nx), device=DEV)
    lib.nadmm_spectral_solve(reg.handle, dev(y), w, torch.cuda.current_stream())
    ref = O.spectral_solve(y, 10.0, 0.1, 2)
    got = w.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(y).max()


def test_autotune_and_cache(lib, tmp_path):
    cache = str(tmp_path / "plans.json")
    plan = lib.autotune(DIMS, DEV, cache)
    assert plan & ~lib.PLAN_FLAGS == 0
    table = json.load(open(cache))
    (key, rec), = table.items()
    assert key.startswith("96,96,64|") and rec["plan_flags"] == plan and rec["ms_per_iteration"] > 0
    rec["plan_flags"] = lib.NADMM_FLAG_LANE16(2)   # the cache wins over a new timing
    json.dump(table, open(cache, "w"))
    assert lib.autotune(DIMS, DEV, cache) == lib.NADMM_FLAG_LANE16(2)
    pair = synth.make_pair(DIMS, seed=3)
    reg = lib.Registration(DIMS, device=DEV, outer=2, inner=3, tune=True)
    u = reg.register(dev(pair["fixed"]), dev(pair["moving"])).cpu().numpy()
    ref = O.register(pair["fixed"], pair["moving"], lam=10.0, theta=0.1, n=2, outer=2, inner=3)
    assert np.abs(u - ref).max() <= 1e-3


def test_batched_with_tuned_plans(lib, tmp_path):
    dims = [(96, 96, 64), (128, 128, 96), (96, 96, 64)]
    pairs = [synth.make_pair(d, seed=30 + i) for i, d in enumerate(dims)]
    f = [dev(p["fixed"]) for p in pairs]
    m = [dev(p["moving"]) for p in pairs]
    breg = lib.BatchedRegistration(dims, device=DEV, outer=2, inner=3,
                                   autotune_cache=str(tmp_path / "p.json"))
    us = breg.register(f, m)
    for i in (0, 1):
        ref = O.register(pairs[i]["fixed"], pairs[i]["moving"], lam=10.0, theta=0.1, n=2,
                         outer=2, inner=3)
        assert np.abs(us[i].cpu().numpy() - ref).max() <= 1e-3


@pytest.mark.parametrize("dims", [(128, 128, 96), (96, 96, 64), (160, 160, 112), (32, 32, 24)])
def test_fused_pencil_is_the_split_pass(lib, dims):
    """The fused y/z/y cluster kernel computes exactly what the three split
    kernels compute (same transforms, same order of operations), so the
    registrations are bit-identical; grids it does not cover fall back."""
    pair = synth.make_pair(dims, seed=11)
    kw = dict(outer=2, inner=4)
    a = lib.Registration(dims, device=DEV, flags=lib.NADMM_FLAG_FOUR_PASS, **kw)
    b = lib.Registration(dims, device=DEV, flags=lib.NADMM_FLAG_FUSED_PENCIL, **kw)
    ua = a.register(dev(pair["fixed"]), dev(pair["moving"]))
    ub = b.register(dev(pair["fixed"]), dev(pair["moving"]))
    assert lib.nadmm_get_status(b.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    assert torch.equal(ua, ub)


@pytest.mark.parametrize("dims", [(128, 128, 96), (96, 96, 64), (160, 160, 112), (32, 32, 24)])
def test_pipelined_plane_pass_is_the_per_tile_pass(lib, dims):
    """The persistent, double-buffered plane pass (k >= 2 of a fixed schedule)
    runs the per-tile kernel's arithmetic on the same tiles, so registrations
    with and without it are bit-identical; grids with fewer tiles than CTAs
    and tile counts that do not divide evenly over the CTAs are included."""
    pair = synth.make_pair(dims, seed=12)
    kw = dict(outer=2, inner=5)
    a = lib.Registration(dims, device=DEV, flags=lib.NADMM_FLAG_FOUR_PASS, **kw)
    b = lib.Registration(dims, device=DEV, flags=lib.NADMM_FLAG_PIPELINED_PLANE, **kw)
    ua = a.register(dev(pair["fixed"]), dev(pair["moving"]))
    ub = b.register(dev(pair["fixed"]), dev(pair["moving"]))
    assert lib.nadmm_get_status(b.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    assert torch.equal(ua, ub)


@pytest.mark.parametrize("dims", [(128, 128, 96), (20, 12, 14), (96, 112, 80)])
def test_outer_step_slices_per_thread_give_the_same_result(lib, dims):
    """The re-warp, gradient and compose kernels with 1, 2 or 4 z-slices per
    thread (an odd nz leaves a ragged last group) compute the same
    registration bit for bit."""
    pair = synth.make_pair(dims, seed=13)
    kw = dict(outer=3, inner=3)
    ref = None
    for f in (0, lib.NADMM_FLAG_OUTER_Z2, lib.NADMM_FLAG_OUTER_Z4):
        u = lib.Registration(dims, device=DEV, flags=f, **kw).register(dev(pair["fixed"]),
                                                                       dev(pair["moving"]))
        if ref is None:
            ref = u
        else:
            assert torch.equal(u, ref), f


def test_autotune_picks_outer_slices(lib):
    cfg = lib.make_config((96, 112, 80))
    need = lib.nadmm_autotune_workspace_size(cfg)
    ws = torch.empty(need + 256, dtype=torch.uint8, device=DEV)
    ptr = (ws.data_ptr() + 255) // 256 * 256
    flags, ms = lib.nadmm_autotune(cfg, ptr, need, torch.cuda.current_stream())
    assert flags & lib.NADMM_FLAG_OUTER_MASK != lib.NADMM_FLAG_OUTER_MASK
    assert flags & ~lib.PLAN_FLAGS == 0 and ms > 0
