"""C-ABI checks that need no GPU: the library loads, exports every symbol
declared in include/nadmm.h, and its host-side validation behaves as
documented.  No call here touches a CUDA device."""
import math
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2109_12688_gb300 import nadmm
    return nadmm


def declared_functions():
    text = open(os.path.join(ROOT, "include", "nadmm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nadmm_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 17
    so = lib.load()
    for n in names:
        assert hasattr(so, n), n
    # and the binding exposes the same names
    for n in names:
        assert hasattr(lib, n), n


def test_config_defaults(lib):
    cfg = lib.nadmm_config_init(128, 128, 96)
    assert (cfg.nx, cfg.ny, cfg.nz) == (128, 128, 96)
    assert cfg.order_n == 2 and cfg.data_term == 2
    assert cfg.lambda_ == pytest.approx(10.0) and cfg.theta == pytest.approx(0.1)
    assert cfg.outer_iters == 10 and cfg.inner_iters == 10
    assert cfg.bound_kappa == pytest.approx(0.5) and cfg.bound_delta == pytest.approx(1.0)


@pytest.mark.parametrize("dims", [(128, 128, 96), (32, 32, 24), (160, 160, 112), (96, 96, 64),
                                  (20, 12, 14), (4, 4, 4), (12, 6, 7), (256, 256, 192)])
def test_create_and_workspace_size(lib, dims):
    h = lib.nadmm_create(lib.make_config(dims))
    nx, ny, nz = dims
    V = nx * ny * nz
    ws = lib.nadmm_workspace_size(h)
    # half spectrum + 6 vector fields + 4 scalar fields, plus small tables
    expect = 3 * (nx // 2 + 1) * ny * nz * 8 + (6 * 3 + 4) * V * 4
    assert expect <= ws <= expect + 64 * 1024
    lib.nadmm_destroy(h)


@pytest.mark.parametrize("dims,why", [((3, 8, 8), "dimension"), ((10, 8, 8), "multiple of 4"),
                                      ((8, 7, 8), "even"), ((8, 2 * 521, 8), "prime factor"),
                                      ((4 * 521, 8, 8), "prime factor"), ((512, 64, 64), "shared"),
                                      ((64, 64, 320), "nz must be")])
def test_unsupported_sizes_are_rejected(lib, dims, why):
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_create(lib.make_config(dims))
    assert e.value.status == lib.NADMM_ERR_UNSUPPORTED_SIZE
    assert why in str(e.value)


@pytest.mark.parametrize("dims", [(44, 8, 8), (8, 8, 13), (44, 26, 23), (88, 52, 34),
                                  (100, 98, 97), (4, 4, 251), (20, 22, 11 * 13)])
def test_sizes_with_prime_factors_above_7_are_planned(lib, dims):
    """Prime factors above 7 get direct-sum FFT stages, so these grids plan
    and size their workspace like smooth ones (host only)."""
    h = lib.nadmm_create(lib.make_config(dims))
    nx, ny, nz = dims
    assert lib.nadmm_workspace_size(h) >= 3 * (nx // 2 + 1) * ny * nz * 8
    lib.nadmm_destroy(h)


@pytest.mark.parametrize("field,value", [("order_n", 0), ("order_n", 9), ("theta", 0.0),
                                         ("theta", -1.0), ("lambda_", -0.5),
                                         ("lambda_", float("nan")), ("outer_iters", 0),
                                         ("inner_iters", 0), ("data_term", 3), ("eps", 0.0),
                                         ("bound_kappa", 0.0), ("bound_delta", -1.0),
                                         ("flags", 0x8000), ("flags", 0x3000), ("flags", 12),
                                         ("flags", 0x400 | 0x800)])
def test_bad_parameters_are_rejected(lib, field, value):
    cfg = lib.make_config((32, 32, 24))
    setattr(cfg, field, value)
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_create(cfg)
    assert e.value.status == lib.NADMM_ERR_INVALID_ARG


def test_infinite_bounds_allowed(lib):
    h = lib.nadmm_create(lib.make_config((32, 32, 24), kappa=math.inf, delta=math.inf))
    lib.nadmm_destroy(h)


def test_calls_without_workspace_fail_before_any_device_work(lib):
    h = lib.nadmm_create(lib.make_config((32, 32, 24)))
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_register(h, 256, 512, 768)
    assert e.value.status == lib.NADMM_ERR_NO_WORKSPACE
    for fn, args in ((lib.nadmm_spectral_solve, (256, 512)),
                     (lib.nadmm_bound_compose, (256, 512, 768))):
        with pytest.raises(lib.NadmmError) as e:
            fn(h, *args)
        assert e.value.status == lib.NADMM_ERR_NO_WORKSPACE
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_set_workspace(h, 1000, 1 << 30)
    assert e.value.status == lib.NADMM_ERR_ALIGNMENT
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_set_workspace(h, 4096, 16)
    assert e.value.status == lib.NADMM_ERR_NO_WORKSPACE
    with pytest.raises(lib.NadmmError):
        lib.nadmm_set_params(h, 1.0, 0.0)
    lib.nadmm_set_params(h, 1.0, 0.5)
    lib.nadmm_destroy(h)
    lib.nadmm_destroy(None)


def test_status_strings(lib):
    assert lib.nadmm_status_string(0) == "NADMM_OK"
    assert lib.nadmm_status_string(lib.NADMM_ERR_NONFINITE) == "NADMM_ERR_NONFINITE"
    assert "unknown" in lib.nadmm_status_string(99)


def _ws_parts(dims):
    nx, ny, nz = dims
    V = nx * ny * nz
    return 3 * (nx // 2 + 1) * ny * nz * 8 + (6 * 3 + 4) * V * 4


def test_batched_create_layout(lib):
    dims = [(32, 32, 24), (96, 96, 64), (20, 12, 14), (160, 160, 112), (12, 6, 7)]
    h = lib.nadmm_create_batched(lib.make_config(dims[0]), dims)
    two = lib.nadmm_workspace_size(h)  # default: two lanes -> {160^2x112}, {the rest}
    assert lib.nadmm_batch_get_lanes(h) == 2
    big, second = _ws_parts((160, 160, 112)), _ws_parts((96, 96, 64))
    assert big + second <= two <= big + second + 5 * 64 * 1024
    lib.nadmm_batch_set_lanes(h, 4)
    ws = lib.nadmm_workspace_size(h)
    # 4 lanes, largest pairs first -> lanes hold {160^2x112}, {96^2x64},
    # {32^2x24, 12x6x7}, {20x12x14}: one state region per lane plus tables
    states = [_ws_parts((160, 160, 112)), _ws_parts((96, 96, 64)), _ws_parts((32, 32, 24)),
              _ws_parts((20, 12, 14))]
    assert sum(states) <= ws <= sum(states) + 5 * 64 * 1024
    lib.nadmm_batch_set_lanes(h, 1)  # one lane: the largest pair's state only
    ws1 = lib.nadmm_workspace_size(h)
    assert _ws_parts((160, 160, 112)) <= ws1 <= _ws_parts((160, 160, 112)) + 5 * 64 * 1024
    lib.nadmm_batch_set_lanes(h, 99)  # clamped to npairs
    assert lib.nadmm_batch_get_lanes(h) == len(dims)
    assert lib.nadmm_workspace_size(h) >= sum(_ws_parts(d) for d in dims)
    lib.nadmm_destroy(h)


def test_batched_default_lanes_and_flat_on_request(lib):
    """Batched handles start with two concurrent lanes even when every pair
    can take the slab path; flat execution (lane count 0) is on request and
    refused with the reverse-mode tape (host logic, no device work)."""
    dims = [(32, 32, 24), (64, 48, 48), (96, 112, 80)]
    h = lib.nadmm_create_batched(lib.make_config(dims[0]), dims)
    assert lib.nadmm_batch_get_lanes(h) == 2
    lib.nadmm_batch_set_lanes(h, 0)
    assert lib.nadmm_batch_get_lanes(h) == 0
    lib.nadmm_batch_set_lanes(h, 3)
    assert lib.nadmm_batch_get_lanes(h) == 3
    lib.nadmm_destroy(h)
    taped = lib.nadmm_create_batched(
        lib.make_config(dims[0], flags=lib.NADMM_FLAG_SAVE_FOR_BACKWARD), dims)
    assert lib.nadmm_batch_get_lanes(taped) == 2
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_batch_set_lanes(taped, 0)
    assert e.value.status == lib.NADMM_ERR_INVALID_ARG
    lib.nadmm_destroy(taped)


def test_batched_create_rejects_bad_pair(lib):
    dims = [(32, 32, 24), (10, 8, 8)]
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_create_batched(lib.make_config(dims[0]), dims)
    assert e.value.status == lib.NADMM_ERR_UNSUPPORTED_SIZE
    assert "pair 1" in str(e.value)
    with pytest.raises(lib.NadmmError):
        lib.nadmm_create_batched(lib.make_config(dims[0]), [])


def test_batched_handle_only_takes_batched_calls(lib):
    h = lib.nadmm_create_batched(lib.make_config((32, 32, 24)), [(32, 32, 24), (16, 16, 8)])
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_register(h, 16, 16, 16)
    assert e.value.status == lib.NADMM_ERR_INVALID_ARG
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_register_batched(h, [16, 16], [16, 16], [16, 16])
    assert e.value.status == lib.NADMM_ERR_NO_WORKSPACE
    lib.nadmm_destroy(h)
    single = lib.nadmm_create(lib.make_config((32, 32, 24)))
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_batch_set_lanes(single, 2)
    assert e.value.status == lib.NADMM_ERR_INVALID_ARG
    lib.nadmm_destroy(single)


def test_pyramid_create_checks(lib):
    cfg = lib.make_config((128, 128, 96))
    h = lib.nadmm_create_pyramid(cfg, (10, 10, 5), (10, 5, 5))
    ws = lib.nadmm_workspace_size(h)
    assert ws >= _ws_parts((128, 128, 96))  # the shared state region is the finest level's
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_register(h, 16, 16, 16)
    assert e.value.status == lib.NADMM_ERR_INVALID_ARG
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_register_pyramid(h, 16, 16, 16)
    assert e.value.status == lib.NADMM_ERR_NO_WORKSPACE
    lib.nadmm_destroy(h)
    with pytest.raises(lib.NadmmError) as e:  # 96 / 4 = 24 but 20 / 4 = 5 is odd -> ny check
        lib.nadmm_create_pyramid(lib.make_config((128, 20, 96)), (1, 1, 1), (1, 1, 1))
    assert e.value.status == lib.NADMM_ERR_UNSUPPORTED_SIZE
    with pytest.raises(lib.NadmmError) as e:  # coarsest 32/8 = 4 -> nx % 4 ok, 24 / 8 = 3 < 4
        lib.nadmm_create_pyramid(lib.make_config((32, 32, 24)), (1,) * 4, (1,) * 4)
    assert e.value.status == lib.NADMM_ERR_UNSUPPORTED_SIZE
    assert "level 3" in str(e.value)


def test_plan_flags_and_autotune_sizes(lib):
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_create(lib.make_config((32, 32, 24),
                                         flags=lib.NADMM_FLAG_LANE8(1) | lib.NADMM_FLAG_LANE16(1)))
    assert e.value.status == lib.NADMM_ERR_INVALID_ARG
    for ax in range(3):  # either choice creates a handle for 96 x 96 x 64 (12.8 / 6.16 splits)
        for f in (lib.NADMM_FLAG_LANE8(ax), lib.NADMM_FLAG_LANE16(ax)):
            lib.nadmm_destroy(lib.nadmm_create(lib.make_config((96, 96, 64), flags=f)))
    cfg = lib.make_config((128, 128, 96))
    need = lib.nadmm_autotune_workspace_size(cfg)
    h = lib.nadmm_create(cfg)
    assert need >= lib.nadmm_workspace_size(h)
    lib.nadmm_destroy(h)
    b = lib.nadmm_create_batched(cfg, [(128, 128, 96), (96, 96, 64)])
    lib.nadmm_batch_set_pair_plan(b, 1, lib.NADMM_FLAG_LANE16(2))
    with pytest.raises(lib.NadmmError):
        lib.nadmm_batch_set_pair_plan(b, 2, 0)
    with pytest.raises(lib.NadmmError):
        lib.nadmm_batch_set_pair_plan(b, 0, lib.NADMM_FLAG_NO_GRAPH)
    lib.nadmm_destroy(b)


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library every entry point raises: there is no
    fallback implementation (fresh interpreter, library path redirected)."""
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_2109_12688_gb300 import nadmm\n"
        "nadmm.LIB_PATH = %r\n"
        "try:\n"
        "    nadmm.make_config((32, 32, 24)); nadmm.nadmm_create(nadmm.make_config((32, 32, 24)))\n"
        "except ImportError as e:\n"
        "    print('raised', 'no fallback' in str(e))\n"
        "else:\n"
        "    print('no error')\n" % (ROOT, str(tmp_path / "libnadmm.so")))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert out.stdout.strip() == "raised True", out.stdout + out.stderr


def test_high_level_calls_reject_host_tensors(lib):
    """The Registration classes check their tensors before any device work:
    a host tensor never reaches a kernel as a device pointer."""
    torch = pytest.importorskip("torch")
    reg = object.__new__(lib.Registration)      # no device workspace needed
    reg.dims, reg.handle = (8, 8, 8), None
    host = torch.zeros((8, 8, 8))
    with pytest.raises(ValueError, match="CUDA tensor"):
        reg.register(host, host)
    with pytest.raises(ValueError, match="CUDA tensor"):
        reg.backward(host, host, torch.zeros((3, 8, 8, 8)))
    b = object.__new__(lib.BatchedRegistration)
    b.dims_list, b.handle = [(8, 8, 8), (4, 4, 4)], None
    with pytest.raises(ValueError, match="2 tensors expected"):
        b.register([host], [host])
    with pytest.raises(ValueError, match="CUDA tensor"):
        b.register([host, torch.zeros((4, 4, 4))], [host, torch.zeros((4, 4, 4))])


@pytest.mark.parametrize("dims,why", [((22, 12, 14), "factors in {2,3,5,7}"),
                                      ((44, 26, 23), "factors in {2,3,5,7}"),
                                      ((64, 64, 320), "nz must be <= 256"),
                                      ((160, 160, 112), "24 MiB"),
                                      ((10, 8, 8), "nx a multiple of 4")])
def test_noalloc_limits_are_checked_before_device_work(lib, dims, why):
    """The no-allocation solve takes a narrower set of grids than
    nadmm_create (factors 2, 3, 5, 7 only; nz <= 256; 24 MiB of static
    scratch) and rejects the rest on the host, before any device call; the
    pointers here are aligned stand-ins that are never dereferenced."""
    nx, ny, nz = dims
    if dims[0] % 4 == 0 and dims != (64, 64, 320):  # nadmm_create plans these grids
        lib.nadmm_destroy(lib.nadmm_create(lib.make_config(dims)))
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_spectral_solve_noalloc(nx, ny, nz, 2, 10.0, 0.1, 4096, 8192)
    assert e.value.status == lib.NADMM_ERR_UNSUPPORTED_SIZE
    assert why in str(e.value)


def test_noalloc_argument_checks_before_device_work(lib):
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_spectral_solve_noalloc(32, 32, 24, 0, 10.0, 0.1, 4096, 8192)
    assert e.value.status == lib.NADMM_ERR_INVALID_ARG
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_spectral_solve_noalloc(32, 32, 24, 2, 10.0, 0.1, 4100, 8192)
    assert e.value.status == lib.NADMM_ERR_ALIGNMENT
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_spectral_solve_noalloc(32, 32, 24, 2, 10.0, 0.1, None, 8192)
    assert e.value.status == lib.NADMM_ERR_INVALID_ARG


def test_restart_configuration_checks(lib):
    """Adaptive restart (restart_eta >= 0) needs the slab path, fixed
    iteration counts and no reverse mode; NaN is rejected (host only)."""
    lib.nadmm_destroy(lib.nadmm_create(lib.make_config((128, 128, 96), restart_eta=0.999)))
    lib.nadmm_destroy(lib.nadmm_create(lib.make_config((32, 32, 24), restart_eta=math.inf)))
    for kw, status in (({"restart_eta": float("nan")}, lib.NADMM_ERR_INVALID_ARG),
                       ({"restart_eta": 0.9, "flags": lib.NADMM_FLAG_SAVE_FOR_BACKWARD},
                        lib.NADMM_ERR_INVALID_ARG),
                       ({"restart_eta": 0.9, "admm_tol": 0.01}, lib.NADMM_ERR_INVALID_ARG),
                       ({"restart_eta": 0.9, "flags": lib.NADMM_FLAG_FOUR_PASS},
                        lib.NADMM_ERR_UNSUPPORTED_SIZE)):
        with pytest.raises(lib.NadmmError) as e:
            lib.nadmm_create(lib.make_config((32, 32, 24), **kw))
        assert e.value.status == status
    with pytest.raises(lib.NadmmError) as e:
        lib.nadmm_create(lib.make_config((20, 12, 14), restart_eta=0.999))
    assert e.value.status == lib.NADMM_ERR_UNSUPPORTED_SIZE
    assert "slab path" in str(e.value)
