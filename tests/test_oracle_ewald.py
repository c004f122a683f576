"""Pins of the oracle's Ewald/Harris W~ (Sec. 2.1 split into a real-space erfc
part and a reciprocal-lattice part, for layers a height z apart): independence
of the splitting width, the closed-form lattice sum, agreement with the image
sum plus continuum tail (z = 0) and with a brute-force numpy image sum of the
full 3 x 3 tensor (z != 0), symmetries and the far-field limit."""
import numpy as np
import pytest
from scipy.special import zeta

from oracle import oracle as orc


def beta_32():
    # Dirichlet beta(3/2) = 4^-3/2 (zeta(3/2, 1/4) - zeta(3/2, 3/4))
    return 4 ** -1.5 * (zeta(1.5, 0.25) - zeta(1.5, 0.75))


@pytest.mark.parametrize("L,z", [(5, 0.0), (8, 0.0), (8, 0.7), (12, 2.5)])
def test_independent_of_the_splitting_width(L, z):
    Ws = [orc.wtilde_ewald(L, z, eta) for eta in (L / 3.0, L / 4.0, L / 7.0)]
    scale = np.abs(Ws[0]).max()
    for W in Ws[1:]:
        assert np.abs(W - Ws[0]).max() <= 1e-12 * scale


@pytest.mark.parametrize("L", [4, 7, 16])
def test_lattice_sum_closed_form(L):
    """sum over the cell of W~_zz = sum over all lattice points != 0 of 1/r^3 =
    4 zeta(3/2) beta(3/2); xx and yy carry -1/2 of it, xy none."""
    W = orc.wtilde_ewald(L)
    s = 4 * zeta(1.5) * beta_32()
    assert W[3].sum() == pytest.approx(s, rel=1e-12)
    assert W[0].sum() == pytest.approx(-0.5 * s, rel=1e-12)
    assert W[2].sum() == pytest.approx(-0.5 * s, rel=1e-12)
    assert abs(W[1].sum()) < 1e-12
    assert np.abs(W[4:]).max() == 0.0          # no xz, yz coupling within the plane


@pytest.mark.parametrize("L", [6, 16])
def test_matches_image_sum_with_tail(L):
    We = orc.wtilde_ewald(L)[:4]
    Wi = orc.wtilde(L, 64, True)
    assert np.abs(We - Wi).max() <= 1e-7 * np.abs(Wi).max()


def brute_force_layer(L, z, A):
    """numpy image sum of the 3 x 3 dipole tensor between two layers, |a|, |b| <= A,
    plus the continuum tail beyond the square of half-width (A + 1/2) L."""
    a = np.arange(-A, A + 1, dtype=np.float64) * L
    out = np.zeros((6, L, L))
    tail = 4 * np.sqrt(2) / ((A + 0.5) * L * L * L)
    for y in range(L):
        for x in range(L):
            dx = (x + a)[None, :]
            dy = (y + a)[:, None]
            r2 = dx * dx + dy * dy + z * z
            r = np.sqrt(r2)
            ir3, ir5 = 1 / (r2 * r), 3 / (r2 * r2 * r)
            out[0, y, x] = (ir3 - ir5 * dx * dx).sum()
            out[1, y, x] = (-ir5 * dx * dy).sum()
            out[2, y, x] = (ir3 - ir5 * dy * dy).sum()
            out[3, y, x] = (ir3 - ir5 * z * z).sum()
            out[4, y, x] = (-ir5 * dx * z).sum()
            out[5, y, x] = (-ir5 * dy * z).sum()
    out[3] += tail
    out[0] -= 0.5 * tail
    out[2] -= 0.5 * tail
    return out


@pytest.mark.parametrize("z", [0.7, 1.5])
def test_layers_match_brute_force(z):
    L = 4
    We = orc.wtilde_ewald(L, z)
    Wb = brute_force_layer(L, z, 400)
    assert np.abs(We - Wb).max() <= 2e-7 * np.abs(Wb).max(), np.abs(We - Wb).max()


def test_layer_symmetries_and_far_field():
    L, z = 8, 1.3
    W = orc.wtilde_ewald(L, z)
    Wm = orc.wtilde_ewald(L, -z)
    flip_x = lambda a: np.roll(a[:, ::-1], 1, axis=1)      # rho_x -> -rho_x (mod L)  # noqa: E731
    flip_y = lambda a: np.roll(a[::-1, :], 1, axis=0)      # noqa: E731
    tol = 1e-13 * np.abs(W).max()
    for c, sx, sy in [(0, 1, 1), (1, -1, -1), (2, 1, 1), (3, 1, 1), (4, -1, 1), (5, 1, -1)]:
        assert np.abs(flip_x(W[c]) - sx * W[c]).max() <= tol
        assert np.abs(flip_y(W[c]) - sy * W[c]).max() <= tol
    assert np.abs(Wm[:4] - W[:4]).max() <= tol and np.abs(Wm[4:] + W[4:]).max() <= tol
    # a layer far away sees a uniform sheet: every component decays like exp(-2 pi z / L)
    Wfar = orc.wtilde_ewald(L, 3.0 * L)
    assert np.abs(Wfar).max() < 1e-6
