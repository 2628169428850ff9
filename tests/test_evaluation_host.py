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


def test_bench_scores_of_many_pairs_are_means_of_the_per_pair_scores():
    """bench.py's quality_seeds_0_19: the worker scores a registration with
    evaluation.score, and the summary averages each class over the pairs
    (NaN Hausdorff values, where a class is missing, are left out) and
    keeps the largest share of det <= 0."""
    import bench
    dims = (16, 16, 12)
    pairs = [synth.make_pair(dims, seed=s) for s in (0, 1)]
    u0 = np.zeros((3,) + dims[::-1], dtype=np.float32)
    scores = [bench._score_job((p["labels_fixed"], p["labels_moving"], u0)) for p in pairs]
    for p, sc in zip(pairs, scores):
        assert sc == E.score(p["labels_fixed"], p["labels_moving"], u0)
    scores[1]["RV"]["hausdorff_mm"] = float("nan")
    out = bench.summarize_scores(scores, [0.0, 0.5])
    assert out["pairs"] == 2 and out["nonpositive_jacobian_percent_max"] == 0.5
    for c in ("LV", "LVM", "RV"):
        assert out["dice_mean"][c] == round((scores[0][c]["dice"] + scores[1][c]["dice"]) / 2, 4)
    assert out["hausdorff_mm_mean"]["RV"] == round(scores[0]["RV"]["hausdorff_mm"], 4)
