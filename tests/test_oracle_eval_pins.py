"""Pins of the evaluation measures (oracle/nadmm_oracle_eval.py) by hand
examples and brute force."""
import itertools

import numpy as np

import oracle as O


def test_dice_hand_examples():
    a = np.zeros((1, 2, 5), np.uint8)
    b = np.zeros((1, 2, 5), np.uint8)
    a[0, 0, :4] = 1          # 4 voxels
    b[0, 0, 1:5] = 1         # 4 voxels, 3 shared
    b[0, 1, :2] = 1          # 6 voxels
    assert O.dice(a, b, 1) == 2 * 3 / 10
    assert O.dice(a, a, 1) == 1.0
    assert O.dice(a, np.zeros_like(a), 1) == 0.0
    assert O.dice(np.zeros_like(a), np.zeros_like(a), 2) == 1.0


def brute_hd(A, B):
    pa = np.argwhere(A)
    pb = np.argwhere(B)
    d = np.sqrt(((pa[:, None, :] - pb[None, :, :]) ** 2).sum(-1))
    return max(d.min(axis=1).max(), d.min(axis=0).max())


def test_hausdorff_per_slice():
    a = np.zeros((3, 12, 12), np.uint8)
    b = np.zeros_like(a)
    a[0, 2, 2] = 1
    b[0, 5, 6] = 1                    # one pixel each, 3-4-5 triangle
    a[1, 2:6, 2:6] = 1
    b[1, 2:6, 4:8] = 1                # square shifted by 2 pixels
    a[2, 3, 3] = 1                    # slice 2: label absent from b -> skipped
    hd = O.hausdorff_per_slice(a, b, 1, spacing=1.2)
    assert abs(hd - (5.0 + 2.0) / 2 * 1.2) < 1e-12
    # the default spacing is the data's 1.2 mm isotropic voxel (Sec. 4)
    assert O.hausdorff_per_slice(a, b, 1) == hd
    rng = np.random.default_rng(0)
    for _ in range(5):
        A = rng.random((1, 9, 11)) < 0.1
        B = rng.random((1, 9, 11)) < 0.1
        A[0, 0, 0] = B[0, 8, 10] = True
        got = O.hausdorff_per_slice(A.astype(np.uint8), B.astype(np.uint8), 1, spacing=1.0)
        assert abs(got - brute_hd(A[0], B[0])) < 1e-12


def test_warp_labels_integer_shift_and_clamp():
    lab = np.arange(4 * 5 * 6).reshape(4, 5, 6)
    u = np.zeros((3, 4, 5, 6))
    u[0] = 1.0   # sample at x + 1
    u[2] = -0.4  # rounds back to z
    got = O.warp_labels(lab, u)
    for z, y, x in itertools.product(range(4), range(5), range(6)):
        assert got[z, y, x] == lab[z, y, min(x + 1, 5)]


def test_nonpositive_jacobian_percent():
    u = np.zeros((3, 4, 4, 4))
    assert O.nonpositive_jacobian_percent(u) == 0.0
    x = np.arange(4, dtype=float)
    u[0] = -2.0 * x[None, None, :]     # d u_x / dx = -2 inside -> det = -1
    pct = O.nonpositive_jacobian_percent(u)
    # interior x (central difference -2) and borders (one-sided halves -1 -> det 0)
    assert pct == 100.0
