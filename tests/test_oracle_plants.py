"""Each planted mistake in the oracle must be caught by at least one pin.

The oracle is rebuilt with a -DPLANT_* define that introduces one plausible
error (dropped term, wrong comparison, wrong log base, missing centring, ...);
the named pin must then fail. This shows the pins constrain the oracle.
"""
import math

import numpy as np
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


# Planted variants of the python oracles' readings: each is the oracle
# function with one plausible mistake, and its pin must fail on it.
def _fix_no_wrap(v, ext):
    v = np.array(v, np.int64)
    if tuple(v[:3]) == tuple(v[3:]):
        ex, ey, ez = ext
        l = v[3] + ex * (v[4] + ey * v[5]) + 1  # planted: no wrap at the last point
        v[3], v[4], v[5] = l % ex, (l // ex) % ey, l // (ex * ey)
    return v


def _fix_moves_first(v, ext):
    v = np.array(v, np.int64)
    if tuple(v[:3]) == tuple(v[3:]):
        ex, ey, ez = ext
        l = (v[0] + ex * (v[1] + ey * v[2]) + 1) % (ex * ey * ez)
        v[0], v[1], v[2] = l % ex, (l // ex) % ey, l // (ex * ey)  # planted: first voxel
    return v


def _fix_backwards(v, ext):
    v = np.array(v, np.int64)
    if tuple(v[:3]) == tuple(v[3:]):
        ex, ey, ez = ext
        l = (v[3] + ex * (v[4] + ey * v[5]) - 1) % (ex * ey * ez)  # planted: previous point
        v[3], v[4], v[5] = l % ex, (l // ex) % ey, l // (ex * ey)
    return v


def _fix_y_fastest(v, ext):
    v = np.array(v, np.int64)
    if tuple(v[:3]) == tuple(v[3:]):
        ex, ey, ez = ext
        l = (v[4] + ey * (v[3] + ex * v[5]) + 1) % (ex * ey * ez)  # planted: y fastest
        v[4], v[3], v[5] = l % ey, (l // ey) % ex, l // (ex * ey)
    return v


def _pos(X, Y, Z, p):
    p = np.asarray(p, np.int64)
    return np.stack([p % X, (p // X) % Y, p // (X * Y)], 1).astype(np.float64)


def _off_sign(X, Y, Z, pi, pj):
    return (_pos(X, Y, Z, pi) - _pos(X, Y, Z, pj)) / np.array([X, Y, Z], np.float64)


def _off_extent_minus_one(X, Y, Z, pi, pj):
    return (_pos(X, Y, Z, pj) - _pos(X, Y, Z, pi)) / np.array([X - 1, Y - 1, Z - 1], np.float64)


def _off_yx_swapped(X, Y, Z, pi, pj):
    def pos(p):
        p = np.asarray(p, np.int64)
        return np.stack([(p // Y) % X, p % Y, p // (X * Y)], 1).astype(np.float64)
    return (pos(pj) - pos(pi)) / np.array([X, Y, Z], np.float64)


PY_PLANTS = [
    (pins.pyo_self_pair_fix, _fix_no_wrap),
    (pins.pyo_self_pair_fix, _fix_moves_first),
    (pins.pyo_self_pair_fix, _fix_backwards),
    (pins.pyo_self_pair_fix, _fix_y_fastest),
    (pins.pyo_mlp_offsets, _off_sign),
    (pins.pyo_mlp_offsets, _off_extent_minus_one),
    (pins.pyo_mlp_offsets, _off_yx_swapped),
]


def _bm_no_plus_one(words):
    w = np.asarray(words, np.uint64)
    top = (w >> np.uint64(40)).astype(np.float64)
    z = np.empty(6)
    for i in range(3):
        u1 = max(top[2 * i], 1.0) * 2.0 ** -24  # planted: u1 without the + 1
        u2 = top[2 * i + 1] * 2.0 ** -24
        rad = math.sqrt(-2.0 * math.log(u1))
        z[2 * i], z[2 * i + 1] = rad * math.cos(2 * math.pi * u2), rad * math.sin(2 * math.pi * u2)
    return z


def _bm_no_two(words):
    w = np.asarray(words, np.uint64)
    top = (w >> np.uint64(40)).astype(np.float64)
    z = np.empty(6)
    for i in range(3):
        u1 = (top[2 * i] + 1.0) * 2.0 ** -24
        u2 = top[2 * i + 1] * 2.0 ** -24
        rad = math.sqrt(-math.log(u1))  # planted: missing factor 2
        z[2 * i], z[2 * i + 1] = rad * math.cos(2 * math.pi * u2), rad * math.sin(2 * math.pi * u2)
    return z


def _bm_swapped(words):
    w = np.asarray(words, np.uint64)
    top = (w >> np.uint64(40)).astype(np.float64)
    z = np.empty(6)
    for i in range(3):
        u1 = (top[2 * i] + 1.0) * 2.0 ** -24
        u2 = top[2 * i + 1] * 2.0 ** -24
        rad = math.sqrt(-2.0 * math.log(u1))
        z[2 * i], z[2 * i + 1] = rad * math.sin(2 * math.pi * u2), rad * math.cos(2 * math.pi * u2)
    return z


def _inc_later_on_ties(thetas, values, count=2):
    return sorted(range(len(values)), key=lambda i: (-values[i], -i))[:count]


def _inc_smallest(thetas, values, count=2):
    return sorted(range(len(values)), key=lambda i: (values[i], i))[:count]


PY_PLANTS += [
    (pins.pyo_box_muller, _bm_no_plus_one),
    (pins.pyo_box_muller, _bm_no_two),
    (pins.pyo_box_muller, _bm_swapped),
    (pins.pyo_incumbents, _inc_later_on_ties),
    (pins.pyo_incumbents, _inc_smallest),
]


def _lt_relative_to_box_origin(orc, seed, rp, rnd, j, theta_inc, ext, scale):
    from oracle import gp
    w = np.concatenate([orc.philox([j, rp, 2 + rnd, 2], [seed, gp.ROUND_KEY]),
                        orc.philox([j, rp, 2 + rnd, 3], [seed, gp.ROUND_KEY])])
    ext = np.asarray(ext, np.float64)
    return np.clip(scale * ext * gp.box_muller(w), 0.0, ext - 1.0)  # planted: incumbent dropped


def _lt_unit_spread(orc, seed, rp, rnd, j, theta_inc, ext, scale):
    from oracle import gp
    w = np.concatenate([orc.philox([j, rp, 2 + rnd, 2], [seed, gp.ROUND_KEY]),
                        orc.philox([j, rp, 2 + rnd, 3], [seed, gp.ROUND_KEY])])
    ext = np.asarray(ext, np.float64)
    return np.clip(np.asarray(theta_inc) + scale * gp.box_muller(w), 0.0, ext - 1.0)  # planted


@pytest.mark.parametrize("planted", [_lt_relative_to_box_origin, _lt_unit_spread],
                         ids=lambda v: v.__name__)
def test_local_theta_plant_is_caught(orc, planted):
    with pytest.raises(AssertionError):
        pins.pyo_local_theta(planted, orc)


@pytest.mark.parametrize("pin,planted", PY_PLANTS, ids=lambda v: v.__name__)
def test_python_plant_is_caught(pin, planted):
    with pytest.raises(AssertionError):
        pin(planted)
