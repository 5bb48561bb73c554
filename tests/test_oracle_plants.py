"""Each planted mistake in the oracle must be caught by at least one pin.

The oracle is rebuilt with a -DPLANT_* define that introduces one plausible
error (dropped term, wrong comparison, wrong log base, missing centring, ...);
the named pin must then fail. This shows the pins constrain the oracle.
"""
import pytest

import oracle
import pins

PLANTS = [
    ("PLANT_PEARSON_MEAN", pins.pin_pearson_affine),
    ("PLANT_RANK_TIES", pins.pin_spearman_scipy),
    ("PLANT_BINS_FLIP", pins.pin_bins_edges),
    ("PLANT_HIST_LOG2", pins.pin_hist_mi_sklearn),
    ("PLANT_KSG_LE", pins.pin_ksg_tiny),
    ("PLANT_KSG_LE", pins.pin_ksg_sklearn),
    ("PLANT_KSG_DROP_Y", pins.pin_ksg_tiny),
    ("PLANT_KSG_DROP_Y", pins.pin_ksg_sklearn),
    ("PLANT_PHILOX_9", pins.pin_philox_numpy),
]


@pytest.mark.parametrize("define,pin", PLANTS, ids=lambda v: v if isinstance(v, str) else v.__name__)
def test_plant_is_caught(define, pin):
    o = oracle.Oracle(defines=(define,))
    with pytest.raises(AssertionError):
        pin(o)
