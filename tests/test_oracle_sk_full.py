"""Pins of the full-wavevector structure factors and the structure functions
of Eq. structurefunctions (Sec. IV A) in the oracle: a brute-force DFT, the
Parseval identity, agreement with the oracle's own axis structure factor on
the same state, and the linear combinations checked against spectra of the
linearised total-density and concentration fields formed directly."""
import numpy as np

import oracle
from paper_1410_5584_gb300 import inputs


def _brute(a, b):
    nz, ny, nx = a.shape
    n = a.size
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    da, db = a - a.mean(), b - b.mean()
    out = np.zeros((3,) + a.shape)
    for mz in range(nz):
        for my in range(ny):
            for mx in range(nx):
                ph = np.exp(-2j * np.pi * (mz * z / nz + my * y / ny + mx * x / nx))
                fa, fb = np.sum(da * ph), np.sum(db * ph)
                out[:, mz, my, mx] = (abs(fa) ** 2 / n, (fa * np.conj(fb)).real / n, abs(fb) ** 2 / n)
    return out


def test_full_structure_factor_is_the_dft_definition():
    rng = np.random.default_rng(4)
    a = 1.0 + 0.01 * rng.standard_normal((3, 4, 5))
    b = 0.8 + 0.01 * rng.standard_normal((3, 4, 5))
    got = np.stack(oracle.structure_factor_full(a, b))
    assert np.allclose(got, _brute(a, b), rtol=1e-12, atol=1e-18)
    assert np.all(np.abs(got[:, 0, 0, 0]) <= 1e-12 * got.max())  # the conserved k = 0 mode (rounding only)


def test_parseval():
    rng = np.random.default_rng(5)
    a = 1.0 + 0.02 * rng.standard_normal((6, 8, 10))
    b = 0.5 * a[::-1]
    s_aa, s_ab, s_bb = oracle.structure_factor_full(a, b)
    da, db = a - a.mean(), b - b.mean()
    assert abs(s_aa.sum() - np.sum(da ** 2)) <= 1e-12 * s_aa.sum()
    assert abs(s_ab.sum() - np.sum(da * db)) <= 1e-12 * s_aa.sum()


def test_axis_wavevectors_equal_the_oracle_axis_structure_factor():
    """The axis structure factor (profile along x, then its DFT) is the full
    structure factor at k = (k_x, 0, 0): checked on one oracle state."""
    c, w, T, N = oracle.tables(oracle.D3Q19)
    shape = (4, 5, 12)
    f = inputs.random_populations(np.stack([w * 1.0, w * 0.7]), shape, 0.03, seed=2)
    o = oracle.Oracle(oracle.D3Q19, 12, 5, 4, 1.0, 1.0, 1e-4, 0.3, 1)
    o.set_f(f)
    ra, rb, u, cons = o.moments()
    o.sf_sample(axis=0)
    s_aa, s_ab, s_bb, _, n = o.structure_factor()
    full = oracle.structure_factor_full(ra, rb)
    m = np.arange(1, 7)
    assert n == 1
    assert np.allclose(full[0][0, 0, m], s_aa, rtol=1e-10)
    assert np.allclose(full[1][0, 0, m], s_ab, rtol=1e-10, atol=1e-14 * s_aa.max())
    assert np.allclose(full[2][0, 0, m], s_bb, rtol=1e-10)


def test_structure_functions_match_the_linearised_fields():
    rng = np.random.default_rng(6)
    r0a, r0b = 1.3, 0.6
    da = 0.01 * rng.standard_normal((1, 16, 12))
    db = 0.01 * rng.standard_normal((1, 16, 12))
    s = oracle.structure_factor_full(r0a + da, r0b + db)
    s_tt, s_cc, s_tc = oracle.structure_functions(*s, r0a, r0b)
    rt = r0a + r0b
    dt = da + db
    dc = (r0b * da - r0a * db) / rt ** 2
    f_t, f_c = np.fft.fftn(dt - dt.mean()), np.fft.fftn(dc - dc.mean())
    n = da.size
    assert np.allclose(s_tt, np.abs(f_t) ** 2 / n, rtol=1e-10, atol=1e-20)
    assert np.allclose(s_cc, np.abs(f_c) ** 2 / n, rtol=1e-10, atol=1e-24)
    assert np.allclose(s_tc, (f_t * np.conj(f_c)).real / n, rtol=1e-9, atol=1e-22)
    # special cases: fluctuations at fixed concentration have S_CC = 0, at
    # fixed total density S_tt = 0
    s_fixed_c = oracle.structure_factor_full(r0a + da, r0b + da * r0b / r0a)
    assert np.max(np.abs(oracle.structure_functions(*s_fixed_c, r0a, r0b)[1])) <= 1e-12 * np.max(s_fixed_c[0])
    s_fixed_t = oracle.structure_factor_full(r0a + da, r0b - da)
    assert np.max(np.abs(oracle.structure_functions(*s_fixed_t, r0a, r0b)[0])) <= 1e-12 * np.max(s_fixed_t[0])
