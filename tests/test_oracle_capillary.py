"""Pins of the interface-height definition and the height spectrum used for
the capillary fluctuations of Sec. VI B: exact recovery of the dividing
surface of symmetric profiles (shifted, tilted and wavy), independence of the
window choice, periodic windows, and the spectrum of a single mode."""
import numpy as np
import pytest

import oracle


def _stripe(nx, ny, h1, h2, rl=2.3, rg=0.06, width=3.0):
    x = np.arange(nx)[None, :]
    left = 0.5 * (1 + np.tanh((x - h1[:, None]) / width))
    right = 0.5 * (1 - np.tanh((x - h2[:, None]) / width))
    return rg + (rl - rg) * left * right


def test_symmetric_profiles_give_their_midpoints():
    """tanh walls are odd about their midpoint, so the liquid fraction places
    the dividing surface exactly there (to the overlap of the two walls)."""
    ny, nx = 16, 100
    y = np.arange(ny)
    h1 = 25.3 + 1.7 * np.sin(2 * np.pi * y / ny)
    h2 = 75.6 - 0.9 * np.cos(4 * np.pi * y / ny)
    r = _stripe(nx, ny, h1, h2, width=2.0)
    g1, g2 = oracle.interface_heights(r, 50, 0)
    # what is left is the walls' tails beyond the windows and at the bulk
    # columns, ~exp(-2 * 25 / width): ~3e-8 for width 2
    assert np.max(np.abs(g1 - h1)) < 1e-6
    assert np.max(np.abs(g2 - h2)) < 1e-6
    # other bulk columns, same surfaces
    g1b, g2b = oracle.interface_heights(r, 48, 97)
    assert np.max(np.abs(g1b - g1)) < 1e-6 and np.max(np.abs(g2b - g2)) < 1e-6


def test_windows_wrap_periodically():
    """A stripe across the periodic edge (liquid around x = 0)."""
    ny, nx = 8, 128
    r = np.roll(_stripe(nx, ny, np.full(ny, 40.0), np.full(ny, 88.0)), -64, axis=1)
    g1, g2 = oracle.interface_heights(r, 0, 64)
    assert np.allclose(g1, 40.0 - 64, atol=1e-5)
    assert np.allclose(g2, 88.0 - 64, atol=1e-5)


@pytest.mark.parametrize("m", [1, 5, 16])
def test_spectrum_of_one_mode(m):
    """h = h0 + A cos(k_m y): |h_hat(k_m)|^2 / n = n A^2 / 4 at k_m, zero elsewhere."""
    ny, A, phase = 32, 0.37, 0.3
    y = np.arange(ny)
    s = oracle.height_spectrum(12.0 + A * np.cos(2 * np.pi * m * y / ny + phase))
    want = np.zeros(ny // 2)
    # below the Nyquist mode the wave splits evenly between +k and -k; at the
    # Nyquist mode only its cosine part survives on the integer sites
    want[m - 1] = ny * A ** 2 / 4 if m < ny // 2 else ny * (A * np.cos(phase)) ** 2
    assert np.allclose(s, want, atol=1e-12)


@pytest.mark.parametrize("center", [50.0, 13.0, 91.5])
def test_tracking_finds_the_stripe(center):
    """A stripe of half the box width centred anywhere (across the periodic
    edge too): the liquid column is its middle, the gas column half a box away."""
    ny, nx = 8, 100
    x = np.arange(nx)
    d = (x - center + nx / 2) % nx - nx / 2  # signed periodic distance to the centre
    phi = 0.5 * (1 - np.tanh((np.abs(d) - 25.0) / 2.0))
    r = np.tile(0.06 + 2.24 * phi, (ny, 1))
    xl, xg = oracle.track_stripe(r)
    assert abs(((xl - center + nx / 2) % nx) - nx / 2) <= 1.0
    assert xg == (xl + 50) % nx
