"""The three-level pyramid (nadmm_register_pyramid) against the FP64
oracle's pyramid (oracle/nadmm_oracle_pyramid.py): max |du| <= 1e-3 voxel on
the finest grid, on small grids and on 128x128x96 with the paper's first
schedule (ADMM 10/5/5, warpings 10/10/5, coarsest first)."""
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


def run(lib, dims, pair, outer, inner, **kw):
    reg = lib.PyramidRegistration(dims, outer=outer, inner=inner, device=DEV, **kw)
    u = reg.register(dev(pair["fixed"]), dev(pair["moving"]))
    assert lib.nadmm_get_status(reg.handle, torch.cuda.current_stream()) == lib.NADMM_OK
    return u.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_pyramid_32x32x24(lib, n):
    dims = (32, 32, 24)
    p = synth.make_pair(dims, seed=20 + n)
    u = run(lib, dims, p, (3, 2, 2), (4, 3, 2), order_n=n)
    ref = O.register_pyramid(p["fixed"], p["moving"], outer=(3, 2, 2), inner=(4, 3, 2),
                             lam=10.0, theta=0.1, n=n)
    assert np.abs(u - ref).max() <= 1e-3


def test_one_level_pyramid_equals_single_registration(lib):
    dims = (32, 32, 24)
    p = synth.make_pair(dims, seed=5)
    u = run(lib, dims, p, (3,), (4,))
    reg = lib.Registration(dims, device=DEV, outer=3, inner=4)
    ref = reg.register(dev(p["fixed"]), dev(p["moving"])).cpu().numpy()
    assert np.array_equal(u, ref.astype(np.float64))


def test_pyramid_graph_and_direct_agree(lib):
    dims = (32, 32, 24)
    p = synth.make_pair(dims, seed=6)
    a = run(lib, dims, p, (2, 2), (3, 3))
    b = run(lib, dims, p, (2, 2), (3, 3), flags=lib.NADMM_FLAG_NO_GRAPH)
    assert np.array_equal(a, b)


def test_pyramid_128x128x96_paper_schedule(lib):
    """The paper's first hyper-parameter version on a 128x128x96 pair:
    oracle parity, no folds, better label overlap than before registration."""
    dims = (128, 128, 96)
    p = synth.make_pair(dims, seed=0)
    u = run(lib, dims, p, (10, 10, 5), (10, 5, 5), order_n=2)
    ref = O.register_pyramid(p["fixed"], p["moving"], lam=10.0, theta=0.1, n=2)
    assert np.abs(u - ref).max() <= 1e-3
    assert O.nonpositive_jacobian_percent(u) == 0.0
    warped = O.warp_labels(p["labels_moving"], u)
    d0 = np.mean([O.dice(p["labels_moving"], p["labels_fixed"], k) for k in (1, 2, 3)])
    d1 = np.mean([O.dice(warped, p["labels_fixed"], k) for k in (1, 2, 3)])
    assert d1 > d0
