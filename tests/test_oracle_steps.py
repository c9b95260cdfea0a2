"""Pins of the oracle's single steps (arXiv 1802.00036, Section IV) against
library routines (scipy.ndimage), closed forms and brute force on tiny maps.

Each step of the oracle is written as direct loops in C; here every step is
recomputed by an independent route, so that a dropped term, a wrong border,
a transposed index or a flipped comparison in the C code fails a test.
"""
import itertools

import numpy as np
import pytest
from scipy import ndimage

import oracle
from paper_1802_00036_gb300 import synth

INF = np.float32(np.inf)

# footprints of Fig. 4 / Table 2 as boolean masks (row = dy, col = dx)
def footprint(shape):
    if shape == "diamond5":
        return np.array([[abs(y) + abs(x) <= 2 for x in range(-2, 3)] for y in range(-2, 3)])
    if shape == "cross5":
        return np.array([[y == 0 or x == 0 for x in range(-2, 3)] for y in range(-2, 3)])
    if shape == "circle5":
        return np.array([[y * y + x * x <= 5 for x in range(-2, 3)] for y in range(-2, 3)])
    k = {"full3": 3, "full5": 5, "full7": 7}[shape]
    return np.ones((k, k), dtype=bool)


SIZES = [(1, 1), (1, 9), (9, 1), (2, 3), (5, 5), (17, 23), (40, 31)]


def sparse(H, W, seed, density=0.15):
    return synth.random_sparse(H, W, density, seed)


def inverted(H, W, seed, density=0.15):
    return oracle.invert(sparse(H, W, seed, density))


# ---- step 1 ---------------------------------------------------------------

def test_invert_closed_form():
    d = np.array([[0.0, 0.05, 0.0999999, 0.1, 2.5, 80.0, 99.5, 1e-30]], dtype=np.float32)
    v = oracle.invert(d)
    want = np.where(d >= np.float32(0.1), np.float32(100.0) - d, np.float32(0.0))
    assert v.dtype == np.float32
    np.testing.assert_array_equal(v, want)
    # 0.1 itself is valid; the float just below it is empty
    below = np.nextafter(np.float32(0.1), np.float32(0.0))
    assert oracle.invert(np.array([[below]], np.float32))[0, 0] == 0.0


def test_invert_buffer_between_valid_and_empty():
    # Section IV-1: valid depths <= 80 m map to >= 20, empties stay 0
    d = synth.random_sparse(64, 64, 0.5, 3, d_min=0.1, d_max=80.0)
    v = oracle.invert(d)
    assert np.all(v[d > 0] >= 20.0) and np.all(v[d == 0] == 0.0)


# ---- step 2 / grey morphology ----------------------------------------------

@pytest.mark.parametrize("shape", ["diamond5", "full5", "cross5", "full3", "circle5", "full7"])
@pytest.mark.parametrize("hw", SIZES)
def test_dilate_shape_vs_scipy(shape, hw):
    a = inverted(*hw, seed=hw[0] * 100 + hw[1])
    got = oracle.dilate_shape(a, shape)
    want = ndimage.maximum_filter(a, footprint=footprint(shape), mode="constant", cval=-INF)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("k", [1, 3, 5, 7, 15, 31])
@pytest.mark.parametrize("hw", SIZES)
def test_dilate_erode_square_vs_scipy(k, hw):
    a = inverted(*hw, seed=7 + hw[0] + k)
    np.testing.assert_array_equal(
        oracle.dilate_square(a, k),
        ndimage.maximum_filter(a, size=k, mode="constant", cval=-INF))
    np.testing.assert_array_equal(
        oracle.erode_square(a, k),
        ndimage.minimum_filter(a, size=k, mode="constant", cval=INF))


def test_impulse_gives_the_footprint():
    # one valid pixel in an empty map: dilation paints exactly the element
    for shape in ["diamond5", "full5", "cross5", "full3", "circle5", "full7"]:
        fp = footprint(shape)
        d = np.zeros((11, 11), np.float32)
        d[5, 5] = 30.0
        got = oracle.dilate_shape(oracle.invert(d), shape)
        k = fp.shape[0] // 2
        want = np.zeros((11, 11), np.float32)
        want[5 - k:5 + k + 1, 5 - k:5 + k + 1][fp] = 70.0
        np.testing.assert_array_equal(got, want)
    assert footprint("diamond5").sum() == 13 and footprint("cross5").sum() == 9
    assert footprint("circle5").sum() == 21


def test_diamond_is_cross3_twice():
    # the decomposition the GPU path relies on, exact with ignored borders
    cross3 = np.array([[0, 1, 0], [1, 1, 1], [0, 1, 0]], dtype=bool)
    for seed, hw in enumerate(SIZES):
        a = inverted(*hw, seed=seed + 50)
        twice = ndimage.maximum_filter(
            ndimage.maximum_filter(a, footprint=cross3, mode="constant", cval=-INF),
            footprint=cross3, mode="constant", cval=-INF)
        np.testing.assert_array_equal(oracle.dilate_shape(a, "diamond5"), twice)


def test_square_is_rows_then_columns():
    for seed, hw in enumerate(SIZES):
        a = inverted(*hw, seed=seed + 90)
        for k in (5, 7, 31):
            sep = ndimage.maximum_filter1d(
                ndimage.maximum_filter1d(a, k, axis=1, mode="constant", cval=-INF),
                k, axis=0, mode="constant", cval=-INF)
            np.testing.assert_array_equal(oracle.dilate_square(a, k), sep)


# ---- step 3 ---------------------------------------------------------------

@pytest.mark.parametrize("hw", SIZES)
def test_close_vs_scipy_and_idempotent(hw):
    a = oracle.dilate_shape(inverted(*hw, seed=11 * hw[0] + hw[1]), "diamond5")
    c = oracle.close_square(a, 5)
    want = ndimage.minimum_filter(
        ndimage.maximum_filter(a, size=5, mode="constant", cval=-INF),
        size=5, mode="constant", cval=INF)
    np.testing.assert_array_equal(c, want)
    # closing is extensive and idempotent
    assert np.all(c >= a)
    np.testing.assert_array_equal(oracle.close_square(c, 5), c)


def test_close_fills_a_one_pixel_gap_but_not_a_wide_one():
    # two plateaus 1 px apart are joined by a 5x5 close; 6 px apart they stay apart
    v = np.zeros((9, 20), np.float32)
    v[:, 0:8] = 40.0
    v[:, 9:20] = 40.0
    c = oracle.close_square(v, 5)
    assert np.all(c[:, 8] == 40.0)
    w = np.zeros((9, 20), np.float32)
    w[:, 0:7] = 40.0
    w[:, 13:20] = 40.0
    np.testing.assert_array_equal(oracle.close_square(w, 5), w)


# ---- steps 4 and 6 ----------------------------------------------------------

@pytest.mark.parametrize("k", [7, 15, 31, 51])
@pytest.mark.parametrize("hw", SIZES)
def test_fill_vs_scipy(k, hw):
    a = inverted(*hw, seed=hw[0] * 3 + hw[1] + k, density=0.05)
    got = oracle.fill_square(a, k)
    dil = ndimage.maximum_filter(a, size=k, mode="constant", cval=-INF)
    want = np.where(a < np.float32(0.1), dil, a)
    np.testing.assert_array_equal(got, want)
    # never moves a non-empty pixel
    ne = a >= np.float32(0.1)
    np.testing.assert_array_equal(got[ne], a[ne])


def test_fill_reaches_exactly_chebyshev_radius():
    a = np.zeros((41, 41), np.float32)
    a[20, 20] = 55.0
    f = oracle.fill_square(a, 31)
    yy, xx = np.mgrid[-20:21, -20:21]
    inside = np.maximum(abs(yy), abs(xx)) <= 15
    assert np.all(f[inside] == 55.0) and np.all(f[~inside] == 0.0)


# ---- step 5 ---------------------------------------------------------------

def brute_extend(c, max_rows=-1):
    H, W = c.shape
    e = c.copy()
    for col in range(W):
        rows = [r for r in range(H) if c[r, col] >= np.float32(0.1)]
        if not rows:
            continue
        top = rows[0]
        lo = 0 if max_rows < 0 else max(0, top - max_rows)
        for r in range(lo, top):
            e[r, col] = c[top, col]
    return e


@pytest.mark.parametrize("hw", SIZES)
@pytest.mark.parametrize("max_rows", [-1, 0, 3])
def test_extend_brute_force(hw, max_rows):
    c = inverted(*hw, seed=5 * hw[0] + hw[1], density=0.2)
    np.testing.assert_array_equal(oracle.extend_top(c, max_rows), brute_extend(c, max_rows))


def test_extend_property_column_dense_down_to_top():
    c = inverted(60, 40, seed=4, density=0.02)
    e = oracle.extend_top(c)
    for col in range(40):
        ne = np.nonzero(c[:, col] >= np.float32(0.1))[0]
        if len(ne) == 0:
            np.testing.assert_array_equal(e[:, col], c[:, col])
        else:
            assert np.all(e[: ne[0] + 1, col] == c[ne[0], col])
            np.testing.assert_array_equal(e[ne[0]:, col], c[ne[0]:, col])


# ---- step 7: median -----------------------------------------------------------

@pytest.mark.parametrize("hw", SIZES)
def test_median_vs_scipy(hw):
    f = inverted(*hw, seed=hw[0] + 13 * hw[1], density=0.6)
    np.testing.assert_array_equal(oracle.median5(f),
                                  ndimage.median_filter(f, size=5, mode="nearest"))


def test_median_explicit_windows():
    f = inverted(12, 15, seed=21, density=0.7)
    m = oracle.median5(f)
    H, W = f.shape
    for r, c in itertools.product(range(H), range(W)):
        win = [f[min(max(r + dy, 0), H - 1), min(max(c + dx, 0), W - 1)]
               for dy in range(-2, 3) for dx in range(-2, 3)]
        assert m[r, c] == np.sort(np.array(win, np.float32))[12]


# ---- step 7: Gaussian -----------------------------------------------------------

BINOM = np.array([1.0, 4.0, 6.0, 4.0, 1.0])


@pytest.mark.parametrize("hw", [(3, 3), (5, 7), (17, 23), (40, 31)])
def test_gauss_vs_scipy_mirror(hw):
    m = inverted(*hw, seed=hw[0] * 7 + hw[1], density=0.8)
    g = oracle.gauss5(m)
    k2 = np.outer(BINOM, BINOM) / 256.0
    ref = ndimage.correlate(m.astype(np.float64), k2, mode="mirror")  # mirror = reflect-101
    want = np.where(m < np.float32(0.1), m.astype(np.float64), ref)
    np.testing.assert_allclose(g, want, rtol=1e-13, atol=1e-12)


def test_gauss_impulse_response_is_binomial_outer_product():
    base, peak = 30.0, 94.0
    m = np.full((9, 9), base, np.float32)
    m[4, 4] = peak
    g = oracle.gauss5(m)
    want = np.full((9, 9), base)
    want[2:7, 2:7] += (peak - base) * np.outer(BINOM, BINOM) / 256.0
    np.testing.assert_allclose(g, want, rtol=0, atol=1e-12)


def test_gauss_preserves_constants_exactly():
    m = np.full((6, 8), 47.125, np.float32)
    assert np.all(oracle.gauss5(m) == 47.125)


def test_gauss_reflect101_at_the_edge():
    # a single bright column at x = 1 next to the left edge: reflect-101
    # mirrors it onto x = -1, so pixel x = 0 sees it with weight (4 + 4)/16
    # and pixel x = 1 with weight (6 + 1)/16 (itself, and its mirror at -1)
    m = np.full((5, 6), 10.0, np.float32)
    m[:, 1] = 42.0
    g = oracle.gauss5(m)
    assert g[2, 0] == pytest.approx(10.0 + 32.0 * 8.0 / 16.0, abs=1e-12)
    assert g[2, 1] == pytest.approx(10.0 + 32.0 * 7.0 / 16.0, abs=1e-12)
    assert g[2, 3] == pytest.approx(10.0 + 32.0 * 1.0 / 16.0, abs=1e-12)


# ---- step 7: bilateral ------------------------------------------------------------

DISK = [(dy, dx) for dy in range(-2, 3) for dx in range(-2, 3) if dy * dy + dx * dx <= 4]


def test_bilateral_has_13_taps():
    assert len(DISK) == 13


def test_bilateral_wide_range_sigma_is_normalised_spatial_gaussian():
    m = inverted(17, 19, seed=31, density=0.9)
    g = oracle.bilateral5(m, 1.5, 1e9)
    k = np.zeros((5, 5))
    for dy, dx in DISK:
        k[dy + 2, dx + 2] = np.exp(-(dy * dy + dx * dx) / (2 * 1.5 ** 2))
    k /= k.sum()
    ref = ndimage.correlate(m.astype(np.float64), k, mode="mirror")
    want = np.where(m < np.float32(0.1), m.astype(np.float64), ref)
    np.testing.assert_allclose(g, want, rtol=1e-12, atol=1e-10)


def test_bilateral_single_neighbour_closed_form():
    a, b = 50.0, 50.75
    m = np.full((7, 7), a, np.float32)
    m[3, 4] = b                              # right neighbour of the centre
    g = oracle.bilateral5(m, 1.5, 0.5)
    ws = {o: np.exp(-(o[0] ** 2 + o[1] ** 2) / (2 * 1.5 ** 2)) for o in DISK}
    wc = np.exp(-((b - a) ** 2) / (2 * 0.5 ** 2))
    num = sum(a * w for o, w in ws.items() if o != (0, 1)) + b * ws[(0, 1)] * wc
    den = sum(w for o, w in ws.items() if o != (0, 1)) + ws[(0, 1)] * wc
    assert g[3, 3] == pytest.approx(num / den, rel=1e-14)


def test_bilateral_keeps_a_step_edge_sharp():
    m = np.full((8, 10), 30.0, np.float32)
    m[:, 5:] = 60.0
    g = oracle.bilateral5(m, 1.5, 0.5)
    np.testing.assert_allclose(g, m.astype(np.float64), rtol=0, atol=1e-12)
    # while the Gaussian blurs it
    assert oracle.gauss5(m)[4, 4] > 30.5


def test_blurs_leave_empty_pixels_alone():
    m = inverted(20, 20, seed=41, density=0.5)
    e = m < np.float32(0.1)
    assert np.all(oracle.gauss5(m)[e] == m[e]) and np.all(oracle.bilateral5(m)[e] == m[e])
