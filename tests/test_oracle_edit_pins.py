"""Pins of the editing oracle (Eq. 25, Eq. 26, the thresholding of Sec. 3.1.4 /
Sec. 3.2.3 and the boundary-preserving offset of Sec. 2.3.2) against facts that
do not come from the oracle itself: hand-worked values, closed forms,
invariants and least-squares solutions from a library routine."""
import math

import numpy as np
import pytest

import oracle
from paper_1902_00176_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---- field statistics and Eq. 25 ---------------------------------------------------

def test_field_stats_small_hand_values():
    # [1, 2, 3, 4, 5, 6]: mean 3.5, population variance 35/12
    m, s = oracle.field_stats(np.arange(1, 7, dtype=np.float64).reshape(2, 3))
    assert m == pytest.approx(3.5, abs=1e-15)
    assert s == pytest.approx(math.sqrt(35.0 / 12.0), abs=1e-15)


def test_color_correct_hand_example():
    # Ic = [0, 2] (mean 1, std 1); I = [1, 3] (mean 2, std 1): shift by +1
    out = oracle.color_correct(np.array([[0.0, 2.0]]), np.array([[1.0, 3.0]]))
    np.testing.assert_allclose(out, [[1.0, 3.0]], atol=1e-15)
    # Ic = [0, 1] (std 1/2); I = [10, 14] (mean 12, std 2): scale 4 about the mean
    out = oracle.color_correct(np.array([[0.0, 1.0]]), np.array([[10.0, 14.0]]))
    np.testing.assert_allclose(out, [[10.0, 14.0]], atol=1e-14)


def test_color_correct_matches_library_moments():
    rng = np.random.default_rng(7)
    Ic = rng.normal(3.0, 0.2, (37, 53))
    I = rng.uniform(0.0, 1.0, (37, 53))
    out = oracle.color_correct(Ic, I)
    assert np.mean(out) == pytest.approx(np.mean(I), abs=1e-12)
    assert np.std(out) == pytest.approx(np.std(I), rel=1e-12)
    # an affine map with a positive scale keeps the order of the pixels
    assert np.array_equal(np.argsort(out, axis=None), np.argsort(Ic, axis=None))


def test_color_correct_undoes_positive_affine_map():
    # Sec. 3.2.2: any constant may be added to Ic, and the std ratio undoes a
    # change of contrast, so a * I + b maps back onto I exactly
    rng = np.random.default_rng(8)
    I = rng.uniform(0.0, 1.0, (19, 31))
    for a, b in ((1.0, 0.0), (0.3, -2.0), (7.5, 11.0)):
        np.testing.assert_allclose(oracle.color_correct(a * I + b, I), I, atol=1e-12)


def test_color_correct_constant_and_per_channel():
    # a constant solved field has no contrast: it maps to the original's mean
    out = oracle.color_correct(np.full((4, 5), 2.5), np.array([[0.0, 1.0, 2.0, 3.0, 4.0]] * 4))
    np.testing.assert_allclose(out, 2.0, atol=1e-15)
    # statistics are per channel: channels with different ranges each land on their own
    rng = np.random.default_rng(9)
    I = np.stack([rng.uniform(0, 1, (16, 16)), rng.uniform(5, 9, (16, 16)), rng.uniform(-3, -1, (16, 16))])
    Ic = np.stack([rng.normal(0, 1, (16, 16)) for _ in range(3)])
    out = oracle.color_correct_batch(Ic[None], I[None])[0]
    for c in range(3):
        assert np.mean(out[c]) == pytest.approx(np.mean(I[c]), abs=1e-12)
        assert np.std(out[c]) == pytest.approx(np.std(I[c]), rel=1e-12)


def test_color_correct_is_near_identity_without_edits():
    # Sec. 3.2.2: with an unedited gradient Ic ~ I up to a constant, so the
    # correction only restores that constant
    # (a constant border makes the zero-extended forward gradient conservative)
    rng = np.random.default_rng(10)
    img, _ = synth.constant_border_image(rng, 24, 32)
    gx, gy = synth.forward_gradient(img)
    M, N = 32, 40
    Ic = oracle.solve_from_gradient(gx, gy, M, N, 4)
    np.testing.assert_allclose(oracle.color_correct(Ic, img), img, atol=1e-10)


# ---- thresholding -----------------------------------------------------------------

def test_threshold_hand_example():
    # magnitudes 5, 0.1, 0.2, 1 (exact squares: 25, 0.01, 0.04, 1 up to FP32 rounding)
    gx = np.array([[3.0, 0.1], [0.0, 1.0]], dtype=np.float32)
    gy = np.array([[4.0, 0.0], [0.2, 0.0]], dtype=np.float32)
    ox, oy, keep = oracle.gradient_threshold(gx, gy, 0.1)  # drops |E| < 0.5
    assert keep.tolist() == [[True, False], [False, True]]
    np.testing.assert_array_equal(ox, [[3.0, 0.0], [0.0, 1.0]])
    np.testing.assert_array_equal(oy, [[4.0, 0.0], [0.0, 0.0]])
    # threshold exactly 1.0 (fl(0.2f * 5) = 1): a magnitude equal to it is kept
    _, _, keep = oracle.gradient_threshold(gx, gy, 0.2)
    assert keep.tolist() == [[True, False], [False, True]]
    _, _, keep = oracle.gradient_threshold(gx, gy, 0.25)
    assert keep.tolist() == [[True, False], [False, False]]


def test_threshold_absolute_reference():
    # the "highest possible gradient" of an image in [0, 1] is 1: 30% drops |E| < 0.3
    gx = np.array([[0.29, 0.31, 0.0, -0.5]], dtype=np.float32)
    gy = np.zeros_like(gx)
    _, _, keep = oracle.gradient_threshold(gx, gy, 0.3, ref=1.0)
    assert keep.tolist() == [[False, True, False, True]]


def test_threshold_brute_force_and_monotone():
    rng = np.random.default_rng(11)
    gx = rng.normal(0, 1, (12, 9)).astype(np.float32)
    gy = rng.normal(0, 1, (12, 9)).astype(np.float32)
    mags = np.hypot(gx.astype(np.float64), gy.astype(np.float64))
    prev = None
    for frac in (0.0, 0.1, 0.3, 0.5, 0.9):
        ox, oy, keep = oracle.gradient_threshold(gx, gy, frac)
        # brute force in FP64, away from the boundary where FP32 could decide otherwise
        t = frac * mags.max()
        clear = np.abs(mags - t) > 1e-5
        assert np.array_equal(keep[clear], (mags >= t)[clear])
        # kept values are copied bit for bit, dropped ones are 0
        assert np.array_equal(ox[keep], gx[keep]) and np.array_equal(oy[keep], gy[keep])
        assert not ox[~keep].any() and not oy[~keep].any()
        if prev is not None:
            assert not (keep & ~prev).any()  # a higher threshold never brings a pixel back
        prev = keep
    assert oracle.gradient_threshold(gx, gy, 0.0)[2].all()


# ---- gradient-domain merging, Eq. 26 ------------------------------------------------

def test_merge_hand_example():
    # E = (3, 4), C = 4, alpha = 1/2: |Ep| = sqrt(5) * 2, direction (0.6, 0.8)
    ox, oy = oracle.gradient_merge(np.array([[3.0]]), np.array([[4.0]]), np.array([[4.0]]), 0.5)
    assert ox[0, 0] == pytest.approx(2.683281572999748, abs=1e-14)
    assert oy[0, 0] == pytest.approx(3.577708763999664, abs=1e-14)


def test_merge_limits_and_orientation():
    rng = np.random.default_rng(12)
    gx, gy = rng.normal(0, 1, (2, 8, 8))
    C = rng.uniform(0, 1, (8, 8))
    ox, oy = oracle.gradient_merge(gx, gy, C, 0.0)  # alpha 0: the gradient itself
    np.testing.assert_allclose(ox, gx, rtol=1e-14)
    np.testing.assert_allclose(oy, gy, rtol=1e-14)
    ox, oy = oracle.gradient_merge(gx, gy, C, 1.0)  # alpha 1: the edge map as magnitude
    np.testing.assert_allclose(np.hypot(ox, oy), C, rtol=1e-13)
    for a in (0.25, 0.5, 0.8):
        ox, oy = oracle.gradient_merge(gx, gy, C, a)
        # orientation kept: parallel (zero cross product) and same sense (positive dot product)
        np.testing.assert_allclose(ox * gy - oy * gx, 0.0, atol=1e-13)
        assert (ox * gx + oy * gy > 0).all()
        # the magnitude is the weighted geometric mean of |E| and C
        g = np.exp((1 - a) * np.log(np.hypot(gx, gy)) + a * np.log(C))
        np.testing.assert_allclose(np.hypot(ox, oy), g, rtol=1e-12)


def test_merge_zero_cases():
    ox, oy = oracle.gradient_merge(np.array([[0.0, 1.0]]), np.array([[0.0, 0.0]]), np.array([[0.7, 0.0]]), 0.5)
    np.testing.assert_array_equal(ox, [[0.0, 0.0]])
    np.testing.assert_array_equal(oy, [[0.0, 0.0]])


# ---- boundary-preserving offset (Sec. 2.3.2) -----------------------------------------

def test_ring_mask_counts():
    m = oracle.ring_mask(10, 12, 3)
    assert m.sum() == 10 * 12 - 4 * 6
    assert m[:3].all() and m[-3:].all() and m[:, :3].all() and m[:, -3:].all()
    assert not m[3:-3, 3:-3].any()


def test_boundary_offset_hand_example():
    u = np.arange(16, dtype=np.float64).reshape(4, 4)
    # ring of width 1: every value except 5, 6, 9, 10; their mean is 90/12 = 7.5
    np.testing.assert_allclose(oracle.boundary_offset(u, 1), [[5 - 7.5, 6 - 7.5], [9 - 7.5, 10 - 7.5]])


def test_boundary_offset_is_least_squares_constant():
    rng = np.random.default_rng(13)
    u = rng.normal(0, 1, (14, 17))
    m = oracle.ring_mask(14, 17, 3)
    # argmin_c sum_ring (u + c)^2 from a least-squares solver
    c = np.linalg.lstsq(np.ones((m.sum(), 1)), -u[m], rcond=None)[0][0]
    np.testing.assert_allclose(oracle.boundary_offset(u, 3), (u + c)[3:-3, 3:-3], atol=1e-13)


def test_boundary_offset_recovers_padded_image():
    # a conservative field of a zero-ringed image: the solve plus this offset returns the image
    img, gx, gy = synth.ring_padded_batch(1, 1, 26, 30, ring=3, seed=14)
    Ht, Wt = 26, 30
    gx0, gy0 = synth.forward_gradient(img[0, 0])
    u = oracle.solve_from_gradient(gx0, gy0, Ht + 8, Wt + 8, 4)
    np.testing.assert_allclose(oracle.boundary_offset(u, 3), img[0, 0, 3:-3, 3:-3], atol=1e-10)
    # an edited field: the ring of the offset solution has zero mean
    u = oracle.solve_from_gradient(gx[0, 0].astype(np.float64), gy[0, 0].astype(np.float64), Ht + 8, Wt + 8, 4)
    m = oracle.ring_mask(Ht, Wt, 3)
    c = -u[m].mean()
    assert abs((u + c)[m].mean()) < 1e-12
