"""Pins of the CPU oracle to facts fixed by the paper's definitions and by
mathematics -- never by the oracle itself and never by the CUDA path.

Definitions pinned (Ezhov et al. 2022, Section 2.3): thresholding of the
simulated concentration at u_T1Gd and u_FLAIR, the Dice coefficient, the
additive combination of the two Dice values (reported as their mean), and
the ranking of the database by that score.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(12345)


def _f32(hexstr):
    return np.array(int(hexstr, 16), dtype=np.uint32).view(np.float32)


def _load_golden():
    with open(os.path.join(GOLDEN, "dice_2x2x2.json")) as fh:
        return json.load(fh)


def _rn_sum_half(d1: float, d2: float) -> float:
    """(d1 + d2) * 0.5 with one round-to-nearest on the sum, modelled with
    exact rationals (float(Fraction) is correctly rounded)."""
    return float(Fraction(d1) + Fraction(d2)) * 0.5


# ------------------------------------------------------------------ golden
def test_golden_2x2x2_counts_dice_score_order():
    g = _load_golden()
    t1, t2 = _f32(g["t1"]), _f32(g["t2"])
    patient = np.array([_f32(h) for h in g["patient"]], dtype=np.float32)
    db = np.array([[_f32(h) for h in e["values"]] for e in g["database"]], dtype=np.float32)
    res = oracle.query(db.reshape(len(db), 2, 2, 2), patient.reshape(2, 2, 2), t1, t2,
                       k=len(db))
    assert list(res["pcount"]) == [g["P1"], g["P2"]]
    for e, ent in enumerate(g["database"]):
        assert list(res["all_counts"][e]) == [ent["I1"], ent["I2"], ent["E1"], ent["E2"]], e
        d1 = oracle.dice(ent["I1"], g["P1"], ent["E1"])
        d2 = oracle.dice(ent["I2"], g["P2"], ent["E2"])
        # one correctly rounded division each
        assert d1 == float(Fraction(ent["D1"])), e
        assert d2 == float(Fraction(ent["D2"])), e
        s = res["all_scores"][e]
        assert s == _rn_sum_half(d1, d2), e
        exact = Fraction(ent["S"])
        assert abs(Fraction(s) - exact) <= Fraction(math.ulp(1.0)), e
    assert list(res["index"]) == g["order"]


# ------------------------------------------------------------------ Dice invariants
def _random_volumes(n, shape=(8, 8, 8), p_zero=0.3):
    v = rng.random((n,) + shape, dtype=np.float32)
    v[rng.random(v.shape) < p_zero] = 0.0
    return v


def test_dice_self_is_one_and_disjoint_is_zero():
    vols = _random_volumes(6)
    for v in vols:
        res = oracle.query(v[None], v, 0.6, 0.25, 1)
        assert res["score"][0] == 1.0
    a = np.zeros((8, 8, 8), np.float32)
    b = np.zeros((8, 8, 8), np.float32)
    a[:4] = 0.9
    b[4:] = 0.9
    res = oracle.query(b[None], a, 0.6, 0.25, 1)
    assert res["score"][0] == 0.0
    assert list(res["all_counts"][0][:2]) == [0, 0]


def test_dice_empty_conventions():
    assert oracle.dice(0, 0, 0) == 1.0           # both empty: identical
    assert oracle.dice(0, 5, 0) == 0.0           # one empty
    assert oracle.dice(0, 0, 7) == 0.0
    z = np.zeros((2, 2, 2), np.float32)
    assert oracle.query(z[None], z, 0.6, 0.25, 1)["score"][0] == 1.0


def test_dice_symmetry():
    vols = _random_volumes(10)
    for i in range(0, 10, 2):
        a, b = vols[i], vols[i + 1]
        ab = oracle.query(b[None], a, 0.6, 0.25, 1)["score"][0]
        ba = oracle.query(a[None], b, 0.6, 0.25, 1)["score"][0]
        assert ab == ba


def test_jaccard_identity_through_sets():
    """D = 2J / (1 + J) with J = |A n B| / |A u B| computed on Python sets of
    voxel coordinates -- an independent route to the same rational."""
    vols = _random_volumes(12, shape=(8, 8, 8))
    patient = vols[0]
    res = oracle.query(vols[1:], patient, 0.6, 0.25, 11)
    for k, t in enumerate((np.float32(0.6), np.float32(0.25))):
        pa = {tuple(c) for c in np.argwhere(patient >= t)}
        for e in range(11):
            ea = {tuple(c) for c in np.argwhere(vols[1 + e] >= t)}
            union = len(pa | ea)
            if union == 0:
                expect = Fraction(1)
            else:
                j = Fraction(len(pa & ea), union)
                expect = 2 * j / (1 + j)
            c = res["all_counts"][e]
            got = oracle.dice(int(c[k]), int(res["pcount"][k]), int(c[2 + k]))
            assert got == float(expect), (k, e)


def test_brute_force_second_formula_8cube():
    """Dice = 2TP / (2TP + FP + FN) on exhaustive 8^3 comparisons, with TP, FP,
    FN counted by numpy boolean algebra (a different formula for the same
    quantity)."""
    vols = _random_volumes(20)
    patient = vols[-1]
    res = oracle.query(vols, patient, 0.6, 0.25, 20)
    for e in range(20):
        ds = []
        for t in (np.float32(0.6), np.float32(0.25)):
            a = patient >= t
            b = vols[e] >= t
            tp = int(np.sum(a & b))
            fp = int(np.sum(~a & b))
            fn = int(np.sum(a & ~b))
            den = 2 * tp + fp + fn
            ds.append(1.0 if den == 0 else float(Fraction(2 * tp, den)))
        assert res["all_scores"][e] == _rn_sum_half(*ds), e
    assert res["all_scores"][19] == 1.0


# ------------------------------------------------------------------ thresholds
def test_threshold_boundary_values():
    for t in (np.float32(0.6), np.float32(0.25), np.float32(0.2)):
        below = np.nextafter(t, np.float32(0))
        above = np.nextafter(t, np.float32(1))
        vol = np.array([t, below, above, 0.0, 1.0, -0.0, np.inf, np.nan], dtype=np.float32)
        m = oracle.threshold(vol, t, t)
        assert list(m[0]) == [1, 0, 1, 0, 1, 0, 1, 0]
        assert list(m[1]) == list(m[0])


def test_threshold_monotone_subset():
    v = _random_volumes(1)[0]
    m = oracle.threshold(v, 0.6, 0.25)
    assert np.all(m[0] <= m[1])               # t1 > t2: T1Gd mask inside FLAIR mask


# ------------------------------------------------------------------ ranking
def test_planted_duplicates_lowest_index_wins():
    vols = _random_volumes(30)
    patient = _random_volumes(1)[0]
    vols[17] = patient
    vols[23] = patient
    res = oracle.query(vols, patient, 0.6, 0.25, 3)
    assert list(res["index"][:2]) == [17, 23]
    assert res["score"][0] == 1.0 and res["score"][1] == 1.0
    assert res["score"][2] < 1.0


def test_all_equal_entries_rank_by_index():
    v = _random_volumes(1)[0]
    db = np.repeat(v[None], 9, axis=0)
    res = oracle.query(db, _random_volumes(1)[0], 0.6, 0.25, 9)
    assert list(res["index"]) == list(range(9))


def test_permutation_equivariance():
    vols = _random_volumes(25)
    patient = vols[3].copy()
    perm = rng.permutation(25)
    a = oracle.query(vols, patient, 0.6, 0.25, 25)
    b = oracle.query(vols[perm], patient, 0.6, 0.25, 25)
    np.testing.assert_array_equal(b["all_scores"], a["all_scores"][perm])
    # same multiset of top scores; the order among equal scores follows the indices
    np.testing.assert_array_equal(np.sort(a["score"]), np.sort(b["score"]))


def test_rank_matches_exact_rational_order():
    """The fp64 ranking agrees with the ranking by exact rational scores
    except where two different rationals round to the same double."""
    vols = _random_volumes(40, shape=(8, 8, 8), p_zero=0.5)
    patient = vols[0]
    res = oracle.query(vols[1:], patient, 0.6, 0.25, 39)
    p1, p2 = (int(x) for x in res["pcount"])
    exact = []
    for e, c in enumerate(res["all_counts"]):
        i1, i2, e1, e2 = (int(x) for x in c)
        d1 = Fraction(1) if p1 + e1 == 0 else Fraction(2 * i1, p1 + e1)
        d2 = Fraction(1) if p2 + e2 == 0 else Fraction(2 * i2, p2 + e2)
        exact.append(((d1 + d2) / 2, e))
    order = [e for _, e in sorted(exact, key=lambda t: (-t[0], t[1]))]
    got = list(res["index"])
    for pos, (a, b) in enumerate(zip(order, got)):
        if a != b:
            assert res["all_scores"][a] == res["all_scores"][b], pos


def test_rank_rejects_k_above_n():
    with pytest.raises(ValueError):
        oracle.rank(np.zeros(3), 4)


# ------------------------------------------------------------------ binary16
def test_f16_decoder_all_patterns_against_numpy():
    bits = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    ref = bits.view(np.float16).astype(np.float64)
    got = np.array([oracle.f16_to_f64(int(b)) for b in bits])
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], ref[~nan])
    assert np.array_equal(np.signbit(got[~nan]), np.signbit(ref[~nan]))


def test_f16_threshold_equals_monotone_bit_compare():
    """Non-negative binary16 patterns order like unsigned integers, so
    h >= t  <=>  bits(h) >= bits(smallest binary16 >= t) for 0 <= bits <= 0x7C00."""
    bits = np.arange(0, 0x7C01, dtype=np.uint16)
    vals = bits.view(np.float16).astype(np.float64)
    for t in (np.float32(0.6), np.float32(0.25), np.float32(0.5004883), np.float32(0.15),
              np.float32(0.35), np.float32(1.0), np.float32(6e-8)):
        first = int(np.argmax(vals >= float(t)))
        m = oracle.threshold(bits, t, t)[0]
        assert np.array_equal(m.astype(bool), bits >= first), float(t)
    # negative, -0 and NaN patterns are never in a mask for t > 0
    neg = np.array([0x8000, 0x8001, 0xBC00, 0xFC00, 0x7E00, 0xFE00], dtype=np.uint16)
    assert not oracle.threshold(neg, 0.25, 0.25)[0].any()


def test_f16_counts_match_f32_of_same_values():
    v16 = _random_volumes(5).astype(np.float16)
    p16 = _random_volumes(1)[0].astype(np.float16)
    pm = oracle.threshold(p16, 0.55, 0.3)
    a, _ = oracle.counts(v16, pm, 0.55, 0.3)
    b, _ = oracle.counts(v16.astype(np.float32), pm, 0.55, 0.3)
    np.testing.assert_array_equal(a, b)


# ------------------------------------------------------------------ layouts
def test_unpack_planes_layout():
    v = 9 * 10 * 11
    words = (v + 31) // 32
    for vox in (0, 1, 31, 32, 33, 500, v - 1):
        planes = np.zeros((2, words), np.uint32)
        planes[1, vox // 32] = np.uint32(1) << np.uint32(vox % 32)
        m = oracle.unpack_planes(planes, v)
        assert m[0].sum() == 0
        assert m[1].sum() == 1 and m[1][vox] == 1


def test_block_mean_single_voxel_and_full():
    nx, ny, nz, f = 32, 16, 24, 8
    for (x, y, z) in [(0, 0, 0), (31, 15, 23), (9, 3, 17), (8, 8, 8)]:
        m = np.zeros(nx * ny * nz, np.uint8)
        m[x + nx * (y + ny * z)] = 1
        out = oracle.block_mean(m, nx, ny, nz, f)
        j = (x // f) + (nx // f) * ((y // f) + (ny // f) * (z // f))
        assert out[j] == 1.0 / 512 and out.sum() == 1.0 / 512
    assert np.all(oracle.block_mean(np.ones(nx * ny * nz, np.uint8), nx, ny, nz, f) == 1.0)


def test_l2_closed_forms():
    assert oracle.l2(np.array([0.0, 0.0]), np.array([3.0, 4.0])) == 5.0
    a = rng.random(4096)
    assert oracle.l2(a, a) == 0.0
    b = a + 0.5
    assert math.isclose(oracle.l2(a, b), 0.5 * 64.0, rel_tol=1e-15)


def test_downsample_nearest_neighbour_layout():
    nx = ny = nz = 16
    for f in (2, 4):
        for (x, y, z) in [(0, 0, 0), (1, 2, 3), (3, 3, 3)]:
            m = np.zeros(nx * ny * nz, np.uint8)
            m[f * x + nx * (f * y + ny * f * z)] = 1
            m[f * x + 1 + nx * (f * y + ny * f * z)] = 1   # a voxel the sampling skips
            out = oracle.downsample_nn(m, nx, ny, nz, f)
            o = nx // f
            assert out.sum() == 1 and out[x + o * (y + o * z)] == 1


# ------------------------------------------------------------------ counts from masks
def test_counts_masks_golden_2x2x2_hand_worked():
    """The hand-worked golden query, with every segmentation written out as
    the set of voxels the golden file lists, not derived by any oracle
    call: patient T1Gd {0,1,4}, FLAIR {0,1,2,4,5,7}; the entries' sets
    follow from their values by reading them against 0.6 and 0.25."""
    g = _load_golden()
    v = 8
    sets = [  # (T1Gd voxels, FLAIR voxels) of each golden entry, by hand
        ({0, 1, 4}, {0, 1, 2, 4, 5, 7}),       # identical to the patient
        (set(), set()),                         # all zero
        ({0}, {0}),                             # 0.6 at voxel 0 only
        ({2, 3, 6}, {2, 3, 6, 7}),              # 0.1 0.1 0.9 0.9 0.1 0.1 0.9 0.3
        (set(range(8)), set(range(8))),         # all one
        ({0}, {0}),                             # same as entry 2
        (set(), {0, 1}),                        # values just below / at the thresholds
    ]
    db = np.zeros((len(sets), 2, v), np.uint8)
    for e, (a, b) in enumerate(sets):
        db[e, 0, sorted(a)] = 1
        db[e, 1, sorted(b)] = 1
    pm = np.zeros((2, v), np.uint8)
    pm[0, [0, 1, 4]] = 1
    pm[1, [0, 1, 2, 4, 5, 7]] = 1
    cnt, pc = oracle.counts_masks(db, pm)
    assert list(pc) == [g["P1"], g["P2"]]
    for e, ent in enumerate(g["database"]):
        assert list(cnt[e]) == [ent["I1"], ent["I2"], ent["E1"], ent["E2"]], e


def test_counts_masks_sets_on_irregular_grid():
    """Counts of random byte masks against Python set sizes, per plane, on a
    grid whose voxel count is not a multiple of anything the GPU uses."""
    v = 7 * 5 * 3
    db = (rng.random((9, 2, v)) < 0.4).astype(np.uint8)
    pm = (rng.random((2, v)) < 0.5).astype(np.uint8)
    cnt, pc = oracle.counts_masks(db, pm)
    psets = [set(np.flatnonzero(pm[k]).tolist()) for k in range(2)]
    assert list(pc) == [len(psets[0]), len(psets[1])]
    for e in range(9):
        esets = [set(np.flatnonzero(db[e, k]).tolist()) for k in range(2)]
        assert list(cnt[e]) == [len(psets[0] & esets[0]), len(psets[1] & esets[1]),
                                len(esets[0]), len(esets[1])], e


def test_counts_masks_equals_counts_of_thresholded_volumes():
    """counts_masks(threshold(vols), threshold(patient)) == counts(vols, patient):
    carries the pins of the volume counts over to the mask counts, with the
    two planes thresholded at different values so that a swapped plane or
    a dropped plane offset shows."""
    vols = _random_volumes(15, shape=(6, 9, 11))
    patient = _random_volumes(1, shape=(6, 9, 11))[0]
    vols[4] = patient
    t1, t2 = 0.6, 0.25
    pm = oracle.threshold(patient, t1, t2)
    want, wpc = oracle.counts(vols, pm, t1, t2)
    dbm = np.stack([oracle.threshold(x, t1, t2) for x in vols])
    got, gpc = oracle.counts_masks(dbm, pm)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(gpc, wpc)
    assert np.any(want[:, 0] != want[:, 1]) and np.any(want[:, 2] != want[:, 3])


def test_counts_masks_rejects_non_binary_bytes():
    db = np.zeros((2, 2, 16), np.uint8)
    pm = np.zeros((2, 16), np.uint8)
    oracle.counts_masks(db, pm)
    db[1, 1, 5] = 2
    with pytest.raises(ValueError):
        oracle.counts_masks(db, pm)
    db[1, 1, 5] = 1
    pm[0, 3] = 255
    with pytest.raises(ValueError):
        oracle.counts_masks(db, pm)
