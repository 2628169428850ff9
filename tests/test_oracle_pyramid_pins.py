"""Pins of the pyramid (oracle/nadmm_oracle_pyramid.py): block averages by
hand and by invariants, the displacement upsampling on constant and linear
fields, and the reduction of the pyramid to the single-level method."""
import numpy as np

import oracle as O


def test_downsample2_hand_and_invariants():
    f = np.arange(2 * 2 * 4, dtype=float).reshape(2, 2, 4)
    # block (x 0-1): (0 + 1 + 4 + 5 + 8 + 9 + 12 + 13) / 8 = 6.5; next block + 2
    np.testing.assert_allclose(O.downsample2(f), [[[6.5, 8.5]]])
    g = np.random.default_rng(0).random((6, 8, 10))
    assert abs(O.downsample2(g).mean() - g.mean()) < 1e-14
    assert np.all(O.downsample2(np.full((4, 4, 4), 3.25)) == 3.25)


def test_upsample_displacement_constant_and_linear():
    uc = np.zeros((3, 4, 5, 6))
    uc[0] = 0.3
    uc[2] = -0.7
    uf = O.upsample_displacement(uc, (8, 10, 12))
    np.testing.assert_allclose(uf[0], 0.6)
    np.testing.assert_allclose(uf[1], 0.0)
    np.testing.assert_allclose(uf[2], -1.4)
    # a linear coarse field a * xc is reproduced as 2 a (x - 1/2) / 2 inside
    xc = np.arange(6, dtype=float)
    uc = np.zeros((3, 4, 5, 6))
    uc[0] = 0.1 * xc[None, None, :]
    uf = O.upsample_displacement(uc, (8, 10, 12))
    x = np.arange(12, dtype=float)
    inside = (x >= 1) & (x <= 10)
    expect = np.broadcast_to(0.1 * (x[inside] - 0.5), (8, 10, int(inside.sum())))
    np.testing.assert_allclose(uf[0][:, :, inside], expect, atol=1e-12)
    # the same along y and z (grid sides differ, so a swapped axis shows)
    yc, zc = np.arange(5, dtype=float), np.arange(4, dtype=float)
    uc = np.zeros((3, 4, 5, 6))
    uc[1] = 0.2 * yc[None, :, None]
    uc[2] = -0.3 * zc[:, None, None]
    uf = O.upsample_displacement(uc, (8, 10, 12))
    y, z = np.arange(10, dtype=float), np.arange(8, dtype=float)
    iy, iz = (y >= 1) & (y <= 8), (z >= 1) & (z <= 6)
    np.testing.assert_allclose(uf[1][:, iy, :], np.broadcast_to(
        0.2 * (y[iy] - 0.5)[None, :, None], (8, int(iy.sum()), 12)), atol=1e-12)
    np.testing.assert_allclose(uf[2][iz, :, :], np.broadcast_to(
        -0.3 * (z[iz] - 0.5)[:, None, None], (int(iz.sum()), 10, 12)), atol=1e-12)


def test_two_levels_with_no_fine_steps_is_the_upsampled_coarse_result():
    """Level 0 registers the 2 x 2 x 2 block averages of both images; a fine
    level with no warps returns the coarse displacement resampled and doubled
    (reading R18)."""
    from paper_2109_12688_gb300 import synth
    p = synth.make_pair((16, 12, 8), seed=7)
    kw = dict(lam=10.0, theta=0.1, n=2)
    u = O.register_pyramid(p["fixed"], p["moving"], outer=(2, 0), inner=(3, 3), **kw)
    uc = O.register(O.downsample2(p["fixed"]), O.downsample2(p["moving"]), outer=2, inner=3, **kw)
    np.testing.assert_array_equal(u, O.upsample_displacement(uc, (8, 12, 16)))
    assert np.abs(uc).max() > 0.05  # the coarse level did move


def test_one_level_pyramid_is_the_method_and_u0_continues():
    from paper_2109_12688_gb300 import synth
    p = synth.make_pair((16, 16, 12), seed=3)
    kw = dict(lam=10.0, theta=0.1, n=2)
    u1 = O.register_pyramid(p["fixed"], p["moving"], outer=(3,), inner=(4,), **kw)
    np.testing.assert_array_equal(u1, O.register(p["fixed"], p["moving"], outer=3, inner=4, **kw))
    # starting from u after two steps and running one more = three steps
    u2 = O.register(p["fixed"], p["moving"], outer=2, inner=4, **kw)
    u3 = O.register(p["fixed"], p["moving"], outer=1, inner=4, u0=u2, **kw)
    np.testing.assert_allclose(u3, u1, atol=1e-12)


def test_three_level_pyramid_improves_on_the_fine_level_alone():
    from paper_2109_12688_gb300 import synth
    p = synth.make_pair((32, 32, 24), seed=1)
    kw = dict(lam=10.0, theta=0.1, n=2)
    u = O.register_pyramid(p["fixed"], p["moving"], outer=(4, 3, 2), inner=(6, 4, 4), **kw)
    ssd = lambda v: float(((O.warp(p["moving"], v) - p["fixed"]) ** 2).sum())
    assert ssd(u) < ssd(np.zeros_like(u))
    assert O.jacobian_determinant(u).min() > 0
