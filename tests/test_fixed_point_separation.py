"""The mixed form's separations on explicit positions, restated on the CPU:
positions as fixed-point fractions of the box, u = rint(x 2^32 / L) mod
2^32 per axis, and a pair's separation as the signed 32-bit difference of
two words times the float L 2^-32, all in float32 after the integer
subtraction.  The minimum image is exact by construction, so the error is
the quantisation (L 2^-33 per word) plus three float roundings, whatever
the box; rounding the FP64 difference to float before the image shift (the
form this replaced) leaves up to L 2^-24 on pairs across a face."""
import numpy as np
import pytest

TWO32 = 4294967296.0


def words(x, L):
    return (np.rint(x * (TWO32 / L)).astype(np.int64) % (1 << 32)).astype(np.uint32)


def fix_diff(uj, ui, L):
    d = (uj - ui).view(np.int32)  # wrap-around of the subtraction is the periodic image
    return d.astype(np.float32) * np.float32(L * 2.0 ** -32)


def exact_min_image(xj, xi, L):
    d = xj - xi
    return d - L * np.rint(d / L)


@pytest.mark.parametrize("L", [20.0, 170.0, 250.0, 249.44845826116753, 1000.0])
def test_separation_error_does_not_grow_with_the_box(L):
    rng = np.random.default_rng(int(L))
    n = 200_000
    xi = rng.uniform(0.0, L, n)
    d = rng.uniform(-5.3, 5.3, n)
    xi[: n // 4] = rng.uniform(0.0, 5.3, n // 4)  # a quarter across the x = 0 face
    xj = np.mod(xi + d, L)
    got = fix_diff(words(xj, L), words(xi, L), L).astype(np.float64)
    want = exact_min_image(xj, xi, L)
    bound = 3 * 2.0 ** -24 * np.abs(want) * 1.0001 + L * 2.0 ** -32 + 2.0 ** -149
    assert np.all(np.abs(got - want) <= bound)
    assert np.abs(got - want).max() < 1e-6  # A, for every box here


def test_word_reduction_wraps_negative_and_full_box_positions():
    L = 250.0
    x = np.array([0.0, L * (1 - 2.0 ** -40), -1e-6, L, 2 * L + 1.0, -L + 1.0])
    u = words(x, L)
    assert u[0] == 0 and u[1] == 0 and u[3] == 0  # 2^32 reduces to 0
    assert u[2] == np.uint32((1 << 32) - 17)      # -1e-6 A is 17.2 units below 0
    assert u[4] == words(np.array([1.0]), L)[0] and u[5] == words(np.array([1.0]), L)[0]


def test_float_difference_before_the_shift_loses_l_2_to_the_minus_24():
    """The replaced form: (float)(x_j - x_i), then the shift in float."""
    L = 250.0
    xi = np.array([0.3, 249.9])
    xj = np.array([249.7, 0.1])
    dd = (xj - xi).astype(np.float32)
    old = dd - np.float32(L) * np.rint(dd * np.float32(1.0 / L))
    want = exact_min_image(xj, xi, L)
    new = fix_diff(words(xj, L), words(xi, L), L)
    assert np.abs(old - want).max() > 1e-6
    assert np.abs(new - want).max() < 1e-6
