"""Pins of the N-species oracle (App. C-D): exact conservation, the momentum
noise covariance (2 lb_d - lb_d^2) kT (rho^s delta - rho^s rho^t / rho_t) and
its zero sum, the per-species ghost-noise variances of Eq. new-noise, and the
structure factors of ideal and interacting three-species mixtures against
S = mu R (1 + alpha G R)^-1 (reducing to Eq. str-bin-hom for two species)."""
import numpy as np
import pytest

import oracle
import theory
from paper_1410_5584_gb300 import inputs


def _random_multi_state(lat, ns, shape, rhos, seed):
    c, w, T, N = oracle.tables(lat)
    base = np.stack([w * r for r in rhos])
    return inputs.random_populations(base, shape, 0.02, seed=seed)


@pytest.mark.parametrize("lat,ns", [(oracle.D2Q9, 3), (oracle.D2Q9, 4), (oracle.D3Q19, 3)])
def test_masses_and_total_momentum_are_conserved(lat, ns):
    shape = (1, 9, 11) if lat == oracle.D2Q9 else (4, 5, 6)
    rhos = [1.0, 0.8, 0.6, 0.9][:ns]
    rng = np.random.default_rng(ns)
    G = rng.uniform(0.1, 0.5, (ns, ns))
    G = 0.5 * (G + G.T)
    o = oracle.MultiOracle(lat, ns, shape[2], shape[1], shape[0], np.linspace(0.8, 1.2, ns), 1e-4, G, 3)
    o.set_f(_random_multi_state(lat, ns, shape, rhos, 4))
    _, _, c0 = o.moments()
    o.step(20)
    _, _, c1 = o.moments()
    assert np.allclose(c1[:ns], c0[:ns], rtol=1e-12)
    assert np.all(np.abs(c1[ns:] - c0[ns:]) <= 1e-12 * c0[0])


def _one_site_noise(lat, rhos, tau, kT, trials):
    """Noise terms of single steps from rest on a one-site box: streaming maps
    the site to itself and, at rest with G = 0, R = xi, so the change of each
    mode is its noise."""
    c, w, T, N = oracle.tables(lat)
    ns = len(rhos)
    o = oracle.MultiOracle(lat, ns, 1, 1, 1, tau, kT, np.zeros((ns, ns)), 11)
    rest = np.stack([w * r for r in rhos]).reshape(ns, len(w), 1, 1, 1)
    out = []
    for t in range(trials):
        o.set_f(rest, step=t)
        o.step(1)
        f = o.get_f().reshape(ns, len(w))
        out.append(f @ T.T)  # moments after the step, [s][a]
    return np.array(out), N


def test_momentum_noise_covariance_and_zero_sum():
    rhos, tau, kT = np.array([1.0, 0.7, 0.4]), [1.0, 0.8, 1.25], 1e-4
    m, N = _one_site_noise(oracle.D2Q9, rhos, tau, kT, 3000)
    lam_d = 3 / sum(tau)
    xi = m[:, :, 1:3]                        # [trial][s][alpha]
    assert np.max(np.abs(xi.sum(axis=1))) < 1e-15
    samples = np.concatenate([xi[:, :, 0], xi[:, :, 1]])
    cov = samples.T @ samples / len(samples)
    want = (2 * lam_d - lam_d ** 2) * kT * (np.diag(rhos) - np.outer(rhos, rhos) / rhos.sum())
    # the estimate of a covariance from n Gaussian samples has relative error ~ sqrt(2/n)
    err = np.sqrt(2.0 / len(samples)) * np.sqrt(np.outer(np.diag(want), np.diag(want)))
    assert np.all(np.abs(cov - want) < 4 * err), (cov, want)


def test_ghost_noise_variances_per_species():
    rhos, tau, kT = np.array([1.0, 0.7, 0.4]), [1.0, 0.8, 1.25], 1e-4
    m, N = _one_site_noise(oracle.D2Q9, rhos, tau, kT, 2000)
    for s in range(3):
        lam = 1.0 / tau[s]
        for a in (6, 7, 8):  # ghost modes: no equilibrium, no force moment
            want = (2 * lam - lam ** 2) * N[a] * 3 * kT * rhos[s]
            var = np.mean(m[:, s, a] ** 2)
            assert abs(var / want - 1) < 4 * np.sqrt(2.0 / len(m)), (s, a, var, want)
    # species are independent on these modes
    c = np.corrcoef(m[:, 0, 6], m[:, 1, 6])[0, 1]
    assert abs(c) < 4 / np.sqrt(len(m))


def test_multi_formula_reduces_to_the_binary_one():
    for G, alpha, ra, rb in ((0.4, 0.9, 1.0, 1.0), (0.9, 0.5, 1.3, 0.7)):
        S = theory.multi_sk(1e-5, [ra, rb], [[0, G], [G, 0]], alpha)
        a = G * alpha
        assert np.isclose(S[0, 0], theory.s_rho_rho(1e-5, ra, rb, a), rtol=1e-12)
        assert np.isclose(S[0, 1], theory.s_rho_rhop(1e-5, ra, rb, a), rtol=1e-12)


def _axis_sk_batches(o, nbatch, nsnap, every, burn):
    """Axis structure factors S_{s s'}(k_x, 0, 0) of the density profiles
    (Sec. IV A), in nbatch consecutive batches of nsnap snapshots."""
    o.step(burn)
    out = []
    for _ in range(nbatch):
        acc = np.zeros((o.ns, o.ns, o.nx // 2))
        for _ in range(nsnap):
            o.step(every)
            rho, u, cons = o.moments()
            prof = rho.sum(axis=(1, 2))  # k along x with k_y = k_z = 0
            f = np.fft.fft(prof - prof.mean(axis=1, keepdims=True), axis=1)[:, 1:o.nx // 2 + 1]
            acc += np.einsum("sk,tk->stk", f, np.conj(f)).real
        out.append(acc / (nsnap * o.N))
    return np.array(out)


def test_lattice_theory_reduces_to_binary_and_continuum():
    """The N-species linearised-lattice covariance equals the binary one for two
    species and tends to S = mu R (1 + alpha G R)^-1 as k -> 0."""
    c, w, T, N = oracle.tables(oracle.D2Q9)
    for k in (0.3, 1.0, 2.5):
        Sm = theory.multi_lattice_linear_sk(c, w, T, N, (k, 0), [[0, 0.4], [0.4, 0]], [1.0, 0.8], [1.0, 1.0], 1e-4)
        Sb = theory.lattice_linear_sk(c, w, T, N, (k, 0), 0.4, rho=(1.0, 0.8), kT=1e-4)
        assert np.allclose([Sm[0, 0], Sm[0, 1], Sm[1, 1]], Sb[:3], rtol=1e-10)
    G, rhos = 0.25 * (1 - np.eye(3)), [1.0, 0.8, 0.6]
    for k in (0.02, 0.1):
        Sm = theory.multi_lattice_linear_sk(c, w, T, N, (k, 0), G, rhos, [1.0, 0.8, 1.25], 1e-4)
        Sc = theory.multi_sk(1e-4, rhos, G, np.sinc(k / np.pi))
        assert np.max(np.abs(Sm - Sc)) < 0.05 * k ** 2 * 3e-4


@pytest.mark.slow
@pytest.mark.filterwarnings("ignore:An ill-conditioned matrix")  # k = pi: sin k = 0, a near-unit eigenvalue pair
@pytest.mark.parametrize("g", [0.0, 0.25])
def test_three_species_structure_factors(g):
    """64 x 4 box, rho = (1, 0.8, 0.6), tau = (1, 0.8, 1.25), kT = 1e-4: every
    S_{s s'} at every axis wavevector against the linearised-lattice covariance
    (flat 3 kT rho_s delta at G = 0), and the k < 0.5 band against the
    continuum S = mu R (1 + alpha G R)^-1, alpha = G sin(k)/k."""
    rhos, tau, kT = np.array([1.0, 0.8, 0.6]), [1.0, 0.8, 1.25], 1e-4
    nx, ny = 64, 4
    c, w, T, N = oracle.tables(oracle.D2Q9)
    k = 2 * np.pi * np.arange(1, nx // 2 + 1) / nx
    G = g * (1 - np.eye(3))
    o = oracle.MultiOracle(oracle.D2Q9, 3, nx, ny, 1, tau, kT, G, 5)
    o.init(np.repeat(rhos, nx * ny))
    B = _axis_sk_batches(o, 20, 80, 10, 2000)
    lat = np.array([theory.multi_lattice_linear_sk(c, w, T, N, (kk, 0), G, rhos, tau, kT) for kk in k])
    bands = [k < 0.5, (k >= 0.5) & (k < 1.5), (k >= 1.5) & (k < 2.5), k >= 2.5]
    for s in range(3):
        for t in range(3):
            scale = 3 * kT * np.sqrt(rhos[s] * rhos[t])
            for band in bands:
                got = B[:, s, t, band].mean(axis=1)
                m, se = got.mean(), got.std(ddof=1) / np.sqrt(len(got))
                pred = lat[band, s, t].mean()
                assert abs(m - pred) < 4 * se + 0.01 * scale, (g, s, t, m, pred, se)
            low = k < 0.5
            cont = np.array([theory.multi_sk(kT, rhos, G, np.sinc(kk / np.pi))[s, t] for kk in k[low]]).mean()
            got = B[:, s, t, low].mean(axis=1)
            assert abs(got.mean() - cont) < 4 * got.std(ddof=1) / np.sqrt(len(got)) + 0.02 * scale


@pytest.mark.parametrize("lat,shape", [(oracle.D2Q9, (1, 5, 7)), (oracle.D3Q19, (4, 5, 6))])
def test_block_with_rng_origin_reproduces_the_large_box(lat, shape):
    """A 3^D block updated with the noise indices of its place in a larger
    box gives, for the block's centre site, exactly the large box's
    post-collision values f_i(r + c_i)."""
    nz, ny, nx = shape
    ns = 3
    c, w, T, N = oracle.tables(lat)
    Q, D = len(w), (2 if lat == oracle.D2Q9 else 3)
    G = np.array([[0, 0.3, 0.5], [0.3, 0, 0.2], [0.5, 0.2, 0]])
    tau = [1.0, 0.8, 1.25]
    f0 = _random_multi_state(lat, ns, shape, [1.0, 0.8, 0.6], 9)
    big = oracle.MultiOracle(lat, ns, nx, ny, nz, tau, 1e-4, G, 5)
    big.set_f(f0, step=17)
    big.step(1)
    fb_all = big.get_f()
    z, y, x = (nz // 2 if D == 3 else 0), 2, 3
    bz = 3 if D == 3 else 1
    fb = np.zeros((ns, Q, bz, 3, 3))
    for dz in (range(-1, 2) if D == 3 else (0,)):
        for dy in range(-1, 2):
            for dx in range(-1, 2):
                fb[:, :, dz + 1 if D == 3 else 0, dy + 1, dx + 1] = f0[:, :, (z + dz) % nz, (y + dy) % ny, (x + dx) % nx]
    blk = oracle.MultiOracle(lat, ns, 3, 3, bz, tau, 1e-4, G, 5)
    blk.set_rng_origin(shape, ((z - 1) % nz if D == 3 else 0, (y - 1) % ny, (x - 1) % nx))
    blk.set_f(fb, step=17)
    blk.step(1)
    fo = blk.get_f()
    cz = 1 if D == 3 else 0
    for i in range(Q):
        got = fo[:, i, (cz + c[i, 2]) % bz, 1 + c[i, 1], 1 + c[i, 0]]
        want = fb_all[:, i, (z + c[i, 2]) % nz, (y + c[i, 1]) % ny, (x + c[i, 0]) % nx]
        assert np.array_equal(got, want), i
