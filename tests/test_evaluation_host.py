"""The package's host-side scoring (paper_2109_12688_gb300/evaluation.py,
Sec. 4 measures used by bench.py) against the oracle's evaluation functions
on the synthetic label maps: same carried labels, Dice and per-slice
Hausdorff distance."""
import numpy as np
import pytest

import oracle as O
from paper_2109_12688_gb300 import evaluation as E
from paper_2109_12688_gb300 import synth


@pytest.mark.parametrize("seed", [0, 3])
def test_scoring_matches_oracle_measures(seed):
    dims = (32, 32, 24)
    pair = synth.make_pair(dims, seed)
    rng = np.random.default_rng(seed)
    u = (rng.normal(size=(3,) + dims[::-1]) * 1.3).astype(np.float32)
    warped = E.carry_labels(pair["labels_moving"], u)
    assert np.array_equal(warped, O.warp_labels(pair["labels_moving"], u))
    for cls in (1, 2, 3):
        assert E.dice_overlap(warped, pair["labels_fixed"], cls) == pytest.approx(
            O.dice(warped, pair["labels_fixed"], cls), abs=1e-15)
        a = E.slice_hausdorff_mm(warped, pair["labels_fixed"], cls)
        b = O.hausdorff_per_slice(warped, pair["labels_fixed"], cls)
        assert a == pytest.approx(b, abs=1e-12) or (np.isnan(a) and np.isnan(b))
    s = E.score(pair["labels_fixed"], pair["labels_moving"], np.zeros_like(u))
    for cls, name in E.CLASSES.items():
        assert s[name]["dice"] == s[name]["dice_unregistered"]
