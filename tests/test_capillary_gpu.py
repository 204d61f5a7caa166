"""Capillary fluctuations of a flat interface on the GPU (flbm_cap_*, Sec. VI
B): interface heights and their spectrum against the oracle's definition on
the same state, snapshot averaging, argument checks, and the spectrum of a
fluctuating stripe against the surface tension of a Laplace test (the fitted
values go to capillary.json in FLBM_REPORT_DIR when that variable is set)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1410_5584_gb300 import D2Q9, D3Q19, FlbmError, Lattice

pytestmark = pytest.mark.gpu

RL, RG = 2.3, 0.06


def _stripe_state(nx, ny, seed, shift=0):
    rng = np.random.default_rng(seed)
    y = np.arange(ny)
    h1 = 25.0 + 0.8 * np.sin(2 * np.pi * 3 * y / ny) + 0.3 * rng.standard_normal(ny)
    h2 = 75.0 - 0.5 * np.cos(2 * np.pi * 5 * y / ny) + 0.3 * rng.standard_normal(ny)
    x = np.arange(nx)[None, :]
    phi = 0.25 * (1 + np.tanh((x - h1[:, None]) / 2.0)) * (1 - np.tanh((x - h2[:, None]) / 2.0))
    ra = RG + (RL - RG) * phi + 1e-3 * rng.standard_normal((ny, nx))
    rb = RG + (RL - RG) * (1 - phi) + 1e-3 * rng.standard_normal((ny, nx))
    return np.roll(ra, shift, axis=1), np.roll(rb, shift, axis=1)


@pytest.mark.parametrize("nx,ny,xl,xg,shift", [(100, 64, 50, 0, 0), (100, 37, 48, 97, 0), (100, 64, 10, 60, -40)])
def test_heights_and_spectrum_match_oracle(nx, ny, xl, xg, shift):
    """One snapshot of a rough stripe (also across the periodic edge and with
    an odd number of rows), against the oracle's heights and spectrum of the
    densities the oracle computes from the same populations."""
    ra, rb = _stripe_state(nx, ny, seed=ny + shift, shift=shift)
    g = Lattice(D2Q9, nx, ny, 1, 1.0, 1.0, 1e-5, 1.5, 3, rho0_a=1.18, rho0_b=1.18)
    g.init(ra.ravel(), rb.ravel())
    f = g.get_populations()
    g.cap_sample(xl, xg)
    s, hm, n = g.cap_spectrum()
    assert n == 1
    o = oracle.Oracle(D2Q9, nx, ny, 1, 1.0, 1.0, 1e-5, 1.5, 3)
    o.set_f(f)
    oa, ob, u, cons = o.moments()
    h1, h2 = oracle.interface_heights(oa[0], xl, xg)
    want = 0.5 * (oracle.height_spectrum(h1) + oracle.height_spectrum(h2))
    # the GPU sums the deviations of each site in float (error ~1e-7 per site,
    # ~1e-6 on a height); the spectrum carries that relative to its largest mode
    assert np.max(np.abs(s - want)) <= 1e-4 * want.max()
    assert abs(hm[0] - h1.mean()) < 1e-5 and abs(hm[1] - h2.mean()) < 1e-5


def test_tracked_columns_match_oracle():
    """Columns found on the device (x_liquid = x_gas = -1) for a stripe moved
    across the periodic edge: the same columns, heights and spectrum as the
    oracle's tracking rule."""
    nx, ny = 100, 64
    ra, rb = _stripe_state(nx, ny, seed=21, shift=-38)
    g = Lattice(D2Q9, nx, ny, 1, 1.0, 1.0, 1e-5, 1.5, 3, rho0_a=1.18, rho0_b=1.18)
    g.init(ra.ravel(), rb.ravel())
    f = g.get_populations()
    g.cap_sample(-1, -1)
    s, hm, n = g.cap_spectrum()
    o = oracle.Oracle(D2Q9, nx, ny, 1, 1.0, 1.0, 1e-5, 1.5, 3)
    o.set_f(f)
    oa = o.moments()[0][0]
    xl, xg = oracle.track_stripe(oa)
    h1, h2 = oracle.interface_heights(oa, xl, xg)
    want = 0.5 * (oracle.height_spectrum(h1) + oracle.height_spectrum(h2))
    assert np.max(np.abs(s - want)) <= 1e-4 * want.max()
    assert abs(hm[0] - h1.mean()) < 1e-5 and abs(hm[1] - h2.mean()) < 1e-5


def test_snapshots_average_and_arguments_are_checked():
    ra, rb = _stripe_state(100, 32, seed=5)
    g = Lattice(D2Q9, 100, 32, 1, 1.0, 1.0, 1e-5, 1.5, 3, rho0_a=1.18, rho0_b=1.18)
    g.init(ra.ravel(), rb.ravel())
    g.cap_sample(50, 0)
    first = g.cap_spectrum()[0]
    g.step(5)
    g.cap_sample(50, 0)
    both, hm, n = g.cap_spectrum()
    g.cap_reset()
    g.cap_sample(50, 0)
    second = g.cap_spectrum()[0]
    assert n == 2
    assert np.allclose(both, 0.5 * (first + second), rtol=1e-12, atol=1e-18)
    with pytest.raises(FlbmError):
        g.cap_sample(49, 0)  # other columns while snapshots are accumulated
    with pytest.raises(FlbmError):
        g.cap_sample(50, 50)
    with pytest.raises(FlbmError):
        g.cap_spectrum(nk=17)
    h = Lattice(D3Q19, 8, 8, 8, 1.0, 1.0, 0.0, 0.0, 1)
    h.init()
    with pytest.raises(FlbmError):
        h.cap_sample(4, 0)


def _droplet_pressure_jump(R, n=128, steps=20000, G=1.5):
    """A droplet of radius R relaxed without noise: (effective radius from its
    area, Laplace pressure jump with the Shan-Chen mixture pressure
    p = c_s^2 (rho + rho' + G rho rho'))."""
    y, x = np.mgrid[0:n, 0:n]
    phi = 0.5 * (1 - np.tanh((np.hypot(x - n / 2 + 0.5, y - n / 2 + 0.5) - R) / 2.0))
    g = Lattice(D2Q9, n, n, 1, 1.0, 1.0, 0.0, G, 1, rho0_a=1.18, rho0_b=1.18)
    g.init((RG + (RL - RG) * phi).ravel(), (RG + (RL - RG) * (1 - phi)).ravel())
    g.step(steps)
    fa, fb, u, cons = g.moments()
    fa, fb = fa.reshape(n, n), fb.reshape(n, n)
    c = n // 2
    ina, inb = fa[c - 3:c + 3, c - 3:c + 3].mean(), fb[c - 3:c + 3, c - 3:c + 3].mean()
    outa, outb = fa[:6, :6].mean(), fb[:6, :6].mean()
    p = lambda a, b: (a + b + G * a * b) / 3.0
    return np.sqrt(np.sum((fa - outa) / (ina - outa)) / np.pi), p(ina, inb) - p(outa, outb)


def test_capillary_spectrum_matches_the_laplace_surface_tension():
    """Sec. VI B: the height spectrum of a thermally fluctuating stripe
    (100 x 512, G = 1.5, kT = 1e-5, all rates 1) follows kT / (gamma k^2) with
    the surface tension gamma of an independent Laplace test (droplets of five
    radii).  At larger k the liquid fractions also carry the bulk density
    noise of the windows, a white floor; so S_h = kT / (gamma_c k^2) + c is
    fitted over 0.02 < k < 0.3 and gamma_c is compared with the Laplace value.
    The bound is 25 %: a circular droplet averages the tension over all
    orientations, while the spectrum of an interface along a lattice axis
    measures its stiffness there (measured: gamma_c / gamma_l = 1.14)."""
    jumps = np.array([_droplet_pressure_jump(R) for R in (14, 18, 24, 30, 36)])
    A = np.stack([1.0 / jumps[:, 0], np.ones(len(jumps))], axis=1)
    (gamma_l, offset), *_ = np.linalg.lstsq(A, jumps[:, 1], rcond=None)
    assert 0.12 < gamma_l < 0.20  # the paper reports 0.174 for its variant of the model
    assert abs(offset) < 0.05 * gamma_l / 14
    nx, ny, kT = 100, 512, 1e-5
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    phi = 0.25 * (1 + np.tanh((x - 25) / 2.0)) * (1 - np.tanh((x - 75) / 2.0))
    g = Lattice(D2Q9, nx, ny, 1, 1.0, 1.0, kT, 1.5, 7, rho0_a=1.18, rho0_b=1.18)
    g.init((RG + (RL - RG) * phi).ravel(), (RG + (RL - RG) * (1 - phi)).ravel())
    g.step(20000)
    for _ in range(1000):
        g.step(1000)
        g.cap_sample(-1, -1)
    s, hm, n = g.cap_spectrum()
    assert n == 1000
    k = 2 * np.pi * np.arange(1, ny // 2 + 1) / ny
    fit = (k > 0.02) & (k < 0.3)
    B = np.stack([kT / k[fit] ** 2, np.ones(fit.sum())], axis=1)
    (inv_gamma_c, floor), *_ = np.linalg.lstsq(B, s[fit], rcond=None)
    gamma_c = 1.0 / inv_gamma_c
    report = {"gamma_laplace": gamma_l, "laplace_offset": offset, "gamma_capillary": gamma_c, "white_floor": floor,
              "ratio_m1_12": list(s[:12] * gamma_l * k[:12] ** 2 / kT), "snapshots": n}
    if os.environ.get("FLBM_REPORT_DIR"):
        with open(os.path.join(os.environ["FLBM_REPORT_DIR"], "capillary.json"), "w") as f:
            json.dump(report, f, indent=1)
    assert abs(gamma_c / gamma_l - 1) < 0.25, (gamma_c, gamma_l)
    low = slice(1, 8)  # m = 2 .. 8, k < 0.1, where the floor is < 10 % of the spectrum
    assert abs(np.mean(s[low] * gamma_l * k[low] ** 2 / kT) - 1) < 0.2
    assert 0 < floor < 1e-3
