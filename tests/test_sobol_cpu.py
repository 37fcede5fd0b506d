"""Sobol' directions of the library (QS_DIR_SOBOL; Sec. 4.1, "QMC Sequences").

Host code, no GPU.  Pins: coordinates 0 and 1 of every Sobol' sequence are
fixed by the construction (van der Corput, and the degree-1 polynomial x + 1
with m_1 = 1), so the unshifted points match SciPy's unscrambled Sobol'
there bit for bit; the first 2^m points of every coordinate fall one into
each dyadic interval of length 2^-m, and coordinates 0 and 1 form a
(0, m, 2)-net, with or without the digital shift; the directions are the
normalised inverse-normal images of the points (SciPy's ndtri as reference).
"""
import numpy as np
import pytest

from paper_2410_01316_gb300 import _lib, directions, sobol_points


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def test_first_two_coordinates_match_scipy_unscrambled():
    qmc = pytest.importorskip("scipy.stats.qmc")
    P, d = 1024, 10
    u = sobol_points(d, P, seed=0)
    ref = qmc.Sobol(d, scramble=False).random(P)
    # the library's points are (x + 1/2) / 2^32 with 32-bit integers x
    x = np.floor(u * 2.0 ** 32)
    xr = np.round(ref * 2.0 ** 32)
    assert np.array_equal(x[:, :2], xr[:, :2])


@pytest.mark.parametrize("seed", [0, 12345])
@pytest.mark.parametrize("m", [4, 7, 10])
def test_every_coordinate_is_stratified(seed, m):
    d, P = 40, 2 ** m
    u = sobol_points(d, P, seed=seed)
    assert np.all((u > 0) & (u < 1))
    cells = np.floor(u * P).astype(np.int64)
    for j in range(d):
        assert np.array_equal(np.sort(cells[:, j]), np.arange(P)), j


@pytest.mark.parametrize("seed", [0, 99])
def test_first_two_coordinates_form_a_0m2_net(seed):
    m = 8
    u = sobol_points(2, 2 ** m, seed=seed)
    for a in range(m + 1):          # elementary boxes 2^-a x 2^-(m - a)
        i = np.floor(u[:, 0] * 2 ** a).astype(np.int64)
        k = np.floor(u[:, 1] * 2 ** (m - a)).astype(np.int64)
        counts = np.bincount(i * 2 ** (m - a) + k, minlength=2 ** m)
        assert np.all(counts == 1), a


def test_higher_coordinates_differ_and_shift_changes_points():
    u0 = sobol_points(64, 256, seed=0)
    u1 = sobol_points(64, 256, seed=1)
    assert not np.array_equal(u0, u1)
    # no two coordinates share their direction numbers
    assert len({u0[:, j].tobytes() for j in range(64)}) == 64


def test_directions_are_normalised_inverse_normal_images():
    special = pytest.importorskip("scipy.special")
    d, P, seed = 16, 512, 7
    u = sobol_points(d, P, seed=seed)
    g = special.ndtri(u)
    ref = g / np.linalg.norm(g, axis=1, keepdims=True)
    xi = directions("sobol", d, P, seed=seed)
    assert np.max(np.abs(xi - ref)) < 2e-7


def test_sobol_argument_errors(lib):
    out = np.empty(8, dtype=np.float64)
    assert lib.qs_sobol_points(0, 4, 0, out.ctypes.data) == 1
    assert lib.qs_sobol_points(5000, 1, 0, out.ctypes.data) == 1
    assert lib.qs_sobol_points(2, 4, 0, None) == 1
