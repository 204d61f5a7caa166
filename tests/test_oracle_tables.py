"""Pins of the oracle's lattice tables, equilibrium/forcing moments and noise
generator against what the paper and the mathematics fix (CPU only)."""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import sympy

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac_w(w):
    return [Fraction(x).limit_denominator(1000) for x in w]


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_basis_orthogonal_and_complete_exact(lat):
    """Eq. V-orthog-compl-discrete: sum_i w_i T_ai T_bi = N_a delta_ab and
    w_i sum_a T_ai T_aj / N_a = delta_ij, checked in exact rationals."""
    c, w, T, N = oracle.tables(lat)
    Q = len(w)
    wf = _frac_w(w)
    assert sum(wf) == 1
    Ti = [[int(round(T[a, i])) for i in range(Q)] for a in range(Q)]
    assert np.array_equal(np.array(Ti, dtype=float), T), "basis entries are integers"
    Nf = []
    for a in range(Q):
        for b in range(Q):
            s = sum(wf[i] * Ti[a][i] * Ti[b][i] for i in range(Q))
            if a == b:
                Nf.append(s)
            else:
                assert s == 0, (a, b)
    assert [float(x) for x in Nf] == pytest.approx(list(N), rel=0, abs=1e-15)
    for i in range(Q):
        for j in range(Q):
            s = wf[i] * sum(Fraction(Ti[a][i] * Ti[a][j]) / Nf[a] for a in range(Q))
            assert s == (1 if i == j else 0), (i, j)


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_isotropy_relations(lat):
    """Eq. w-rel: sum w = 1, sum w c c = c_T^2 I, sum w cccc = c_T^4 (3 delta delta
    symmetrised), with c_T^2 = 1/3 (Sec. V B); odd moments vanish."""
    c, w, T, N = oracle.tables(lat)
    D = 2 if lat == oracle.D2Q9 else 3
    wf = _frac_w(w)
    cs2 = Fraction(1, 3)
    d = lambda a, b: 1 if a == b else 0
    for a in range(D):
        assert sum(wf[i] * c[i, a] for i in range(len(w))) == 0
        for b in range(D):
            assert sum(wf[i] * c[i, a] * c[i, b] for i in range(len(w))) == cs2 * d(a, b)
            for g in range(D):
                assert sum(wf[i] * c[i, a] * c[i, b] * c[i, g] for i in range(len(w))) == 0
                for h in range(D):
                    s = sum(wf[i] * c[i, a] * c[i, b] * c[i, g] * c[i, h] for i in range(len(w)))
                    assert s == cs2 ** 2 * (d(a, b) * d(g, h) + d(a, g) * d(b, h) + d(a, h) * d(b, g))


def test_d2q9_matches_table_one():
    """The oracle's D2Q9 rows, norms and m^eq column equal Table I."""
    spec = json.load(open(os.path.join(GOLDEN, "table1_d2q9.json")))
    c, w, T, N = oracle.tables(oracle.D2Q9)
    cx, cy, c2, rho, vx, vy = sympy.symbols("cx cy c2 rho vx vy")
    rng = np.random.default_rng(5)
    samples = [(1.0 + 0.3 * rng.random(), *(0.05 * rng.standard_normal(2))) for _ in range(5)]
    meqs = [oracle.meq(oracle.D2Q9, r, [ux, uy]) for r, ux, uy in samples]
    for row in spec["rows"]:
        a = row["a"]
        Tf = sympy.sympify(row["T"])
        for i in range(9):
            val = Tf.subs({cx: int(c[i, 0]), cy: int(c[i, 1]), c2: int(c[i, 0] ** 2 + c[i, 1] ** 2)})
            assert float(val) == T[a, i], (a, i)
        assert N[a] == pytest.approx(float(sympy.Rational(row["N"])), rel=1e-15)
        mf = sympy.sympify(row["meq"])
        for (r, ux, uy), m in zip(samples, meqs):
            assert m[a] == pytest.approx(float(mf.subs({rho: r, vx: ux, vy: uy})), rel=1e-13, abs=1e-15)


def _hermite2(c, D):
    """H_ab(c) = c_a c_b - c_T^2 delta_ab (Eq. setofT), one row per (a <= b)."""
    rows = []
    for a in range(D):
        for b in range(a, D):
            rows.append(c[:, a] * c[:, b] - (1.0 / 3.0 if a == b else 0.0))
    return rows


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q19])
def test_equilibrium_and_forcing_moments(lat):
    """m^eq and Phi from the second-order Hermite expansions (Eqs. hermite-feq,
    hermite-for): the Hermite projections are rho, rho u, rho u_a u_b and 0, rho a,
    rho (a_a v_b + v_a a_b); ghost projections vanish (Sec. V B remark on the
    truncation)."""
    c, w, T, N = oracle.tables(lat)
    D = 2 if lat == oracle.D2Q9 else 3
    Q = len(w)
    rng = np.random.default_rng(11)
    Tinv = np.linalg.inv(T)
    for _ in range(5):
        rho = 0.5 + rng.random()
        u = 0.05 * rng.standard_normal(D)
        acc = 1e-3 * rng.standard_normal(D)
        v = 0.05 * rng.standard_normal(D)
        meq = oracle.meq(lat, rho, u)
        phi = oracle.phi(lat, rho, acc, v)
        # back to populations, then project on the Hermite polynomials directly
        feq = Tinv @ meq
        fph = Tinv @ phi
        H = _hermite2(c.astype(float), D)
        assert feq.sum() == pytest.approx(rho, rel=1e-14)
        assert fph.sum() == pytest.approx(0.0, abs=1e-15)
        for a in range(D):
            assert c[:, a] @ feq == pytest.approx(rho * u[a], rel=1e-12)
            assert c[:, a] @ fph == pytest.approx(rho * acc[a], rel=1e-12)
        k = 0
        for a in range(D):
            for b in range(a, D):
                assert H[k] @ feq == pytest.approx(rho * u[a] * u[b], rel=1e-10, abs=1e-16)
                assert H[k] @ fph == pytest.approx(rho * (acc[a] * v[b] + v[a] * acc[b]), rel=1e-10, abs=1e-18)
                k += 1
        nhyd = 1 + D + D * (D + 1) // 2
        assert np.allclose(meq[nhyd:], 0.0, atol=1e-15)
        assert np.allclose(phi[nhyd:], 0.0, atol=1e-17)


def test_philox_known_answers():
    """Philox4x32-10 against its published known-answer values."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_gaussians_are_standard_normal():
    """Box-Muller over Philox output (Sec. VI A): a large sample is N(0, 1), with
    independent positions within a block (the third pair is built from the
    words' low bits) and no correlation between neighbouring counters."""
    scipy_stats = pytest.importorskip("scipy.stats")
    n = 30000
    g = np.array([[oracle.gaussian(1234, s, 7, 0, a) for a in range(1, 7)] for s in range(n)])
    flat = g.ravel()
    assert abs(flat.mean()) < 4.0 / np.sqrt(flat.size)
    assert abs(flat.var() - 1.0) < 4.0 * np.sqrt(2.0 / flat.size)
    assert scipy_stats.kstest(flat, "norm").pvalue > 1e-3
    for col in range(6):
        assert scipy_stats.kstest(g[:, col], "norm").pvalue > 1e-4, col
    cc = np.corrcoef(g.T)
    assert np.all(np.abs(cc - np.eye(6)) < 4.0 / np.sqrt(n))
    # the squared radius of a pair is -2 ln u1: exponential with mean 2
    r2 = g[:, 4] ** 2 + g[:, 5] ** 2
    assert scipy_stats.kstest(r2 / 2.0, "expon").pvalue > 1e-3
    lag = np.corrcoef(g[:-1, 0], g[1:, 0])[0, 1]
    assert abs(lag) < 4.0 / np.sqrt(n)


def _uniforms(x):
    """The six 21-bit uniforms of a Philox block, as the noise definition cuts
    them: the top 21 bits of each word, then two from the low bits."""
    return [w >> 11 for w in x] + [((x[0] & 0x7FF) << 10) | (x[1] & 0x3FF),
                                   ((x[2] & 0x7FF) << 10) | (x[3] & 0x3FF)]


def test_gaussian_counter_layout():
    """Mode a >= 1 is Gaussian n = a - 1 of its species: modes a and a + 6 use
    different Philox counters (site, step, species, n / 6); species, step,
    site and seed enter the key or counter; the three Box-Muller pairs of one
    block share their words as stated, radius from the first uniform of the
    pair and angle from the second (cosine for even n, sine for odd n)."""
    base = oracle.gaussian(9, 3, 5, 0, 1)
    assert base != oracle.gaussian(9, 3, 5, 0, 7)
    assert base != oracle.gaussian(9, 3, 5, 1, 1)
    assert base != oracle.gaussian(9, 3, 6, 0, 1)
    assert base != oracle.gaussian(9, 4, 5, 0, 1)
    assert base != oracle.gaussian(10, 3, 5, 0, 1)
    assert np.isnan(oracle.gaussian(9, 3, 5, 0, 0))
    for blk, a0 in ((0, 1), (1, 7), (2, 13)):
        x = oracle.philox4x32_10([3, 5, 1, blk], [9, 0])
        U = _uniforms(x)
        for q in range(3):
            g0 = oracle.gaussian(9, 3, 5, 1, a0 + 2 * q)
            g1 = oracle.gaussian(9, 3, 5, 1, a0 + 2 * q + 1)
            u1, u2 = (U[2 * q] + 1) * 2.0 ** -21, U[2 * q + 1] * 2.0 ** -21
            r = np.sqrt(-2.0 * np.log(u1))
            assert g0 == pytest.approx(r * np.cos(2 * np.pi * u2), rel=1e-12, abs=1e-14), (blk, q)
            assert g1 == pytest.approx(r * np.sin(2 * np.pi * u2), rel=1e-12, abs=1e-14), (blk, q)
