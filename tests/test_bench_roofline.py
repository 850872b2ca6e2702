"""bench.py's choice of the roofline kernel (host logic, no GPU).

The per-phase pass times the explicit apply (one launch) and the solve chain
(the rest of the step's launches) as two phases; the roofline names the
kernel with the longest launches, so the chain's phase time is divided by
its launch count before the two are compared."""
import pytest

import bench


def _st(variant, launches):
    return {"explicit_variant": bench.EXPLICIT_VARIANTS.index(variant), "launches_per_step": launches}


def test_phase_launches_plain_and_split():
    assert bench.phase_launches(_st("tiles_large", 4)) == {"k_explicit2d": 1, "k_walk+k_top": 3}
    # the split explicit launch adds its far tiles' launch to the step, not to the chain
    assert bench.phase_launches(_st("tiles_small_split4", 5)) == {"k_explicit2d": 1, "k_walk+k_top": 3}
    assert bench.phase_launches(_st("sweep", 1)) == {"k_explicit2d": 1, "k_walk+k_top": 1}


@pytest.mark.parametrize("chain_ms,expect", [(0.0399, "k_explicit2d"), (0.0414, "k_explicit2d"),
                                             (0.120, "k_explicit2d"), (0.130, "k_walk+k_top")])
def test_dominant_kernel_compares_mean_launches(chain_ms, expect):
    # 256x128 plate: explicit 40.9 us in one launch, the chain in three launches
    per_step = {"k_explicit2d": 0.0409, "k_walk+k_top": chain_ms}
    assert bench.dominant_kernel(per_step, bench.phase_launches(_st("tiles_large", 4))) == expect
