"""Closed-form predictions of arXiv 1410.5584 used to pin the oracle.

Lattice units: Delta t = Delta r = 1, c_T^2 = 1/3, k_B = 1 (Sec. V B, VI A).
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0


def alpha_lattice(G: float, k):
    """alpha(k) of the lattice mean-field force along a lattice axis:
    G sin(k)/k, i.e. 6 (1 - sin k / k) in place of k^2 in Eq. alpha:lb
    (Sec. VI A)."""
    k = np.asarray(k, dtype=float)
    return G * np.sinc(k / np.pi)


def s_rho_rho(kT, rho0, rho0p, alpha):
    """S_{rho,rho}(k), Eq. str-bin-hom (Sec. IV A)."""
    return kT / CS2 * rho0 / (1.0 - rho0 * rho0p * alpha ** 2)


def s_rho_rhop(kT, rho0, rho0p, alpha):
    """S_{rho,rho'}(k), Eq. str-bin-hom (Sec. IV A)."""
    return -kT / CS2 * rho0 * rho0p * alpha / (1.0 - rho0 * rho0p * alpha ** 2)


def s_vb(kT, rho_t0):
    """Baricentric-velocity structure factor per component, Eq. str-bin-hom-vel."""
    return kT / rho_t0


def structure_functions(kT, rho_t0, C0, alpha):
    """(S_tt, S_CC, S_tC): Eq. structurefunctions (Sec. IV A)."""
    x = C0 * (1.0 - C0)
    den = 1.0 - x * rho_t0 ** 2 * alpha ** 2
    s_tt = rho_t0 * kT / CS2 * (1.0 - 2.0 * x * rho_t0 * alpha) / den
    s_cc = kT * x / (CS2 * rho_t0) * (1.0 + 2.0 * x * rho_t0 * alpha) / den
    s_tc = -kT * x / CS2 * (1.0 - 2.0 * C0) * rho_t0 * alpha / den
    return s_tt, s_cc, s_tc


def hydro_k0(kT, rho_t0, C0, G):
    """k -> 0 structure factors from the Shan-Chen thermodynamics of App. E
    (Eqs. SC:1 - SC:4 and the three results after them), built from mu_C,
    beta and c_s^2 rather than from Eq. structurefunctions."""
    x = C0 * (1.0 - C0)
    beta_rt = -G * rho_t0 ** 2 * (1.0 - 2.0 * C0) / (1.0 + 2.0 * G * rho_t0 * x)  # rho_t0 * beta
    beta = beta_rt / rho_t0
    mu_c = CS2 / x - 2.0 * CS2 * G * rho_t0 + CS2 * G * (1.0 - 2.0 * C0) * beta_rt
    cs2 = CS2 * (1.0 + 2.0 * G * rho_t0 * x)
    s_tt = rho_t0 * kT * (1.0 / cs2 + beta ** 2 / mu_c)
    s_cc = kT / (rho_t0 * mu_c)
    s_tc = beta * kT / mu_c
    return s_tt, s_cc, s_tc


def shear_viscosity(lam_s):
    """Kinematic shear viscosity of the lattice scheme, c_s^2 (1/lambdabar - 1/2)
    (standard Chapman-Enskog result for Eq. lattice-freq rates)."""
    return CS2 * (1.0 / lam_s - 0.5)


def diffusivity(lam_d):
    """Mutual diffusivity of the ideal mixture, c_s^2 (1/lambdabar_d - 1/2); the
    paper cites the Chapman-Enskog analysis for it (Sec. VI) without printing it."""
    return CS2 * (1.0 / lam_d - 0.5)


def batch_means(x, nbatch=20):
    """Mean and standard error of a correlated series by batch means."""
    x = np.asarray(x, dtype=float)
    n = (len(x) // nbatch) * nbatch
    b = x[:n].reshape(nbatch, -1, *x.shape[1:]).mean(axis=1)
    return b.mean(axis=0), b.std(axis=0, ddof=1) / np.sqrt(nbatch)


def family_sigma(ncomp, nbatch=20, level=0.0027):
    """Multiplier of the batch-means standard error for ``ncomp`` simultaneous
    comparisons held to the false-alarm rate of one 3-standard-error check
    (level 0.27 %, two-sided) as a family: each comparison gets the Sidak
    share 1 - (1 - level)^(1/ncomp), and since the standard error is itself
    estimated from ``nbatch`` batch means, (mean - prediction)/SE follows
    Student's t with nbatch - 1 degrees of freedom.  One comparison with 20
    batches gives 3.45; twenty give 4.76."""
    from scipy import stats

    p = 1.0 - (1.0 - level) ** (1.0 / ncomp)
    return float(stats.t.ppf(1.0 - p / 2.0, nbatch - 1))


def lattice_linear_sk(c, w, T, N, k_vec, G, rho=(1.0, 1.0), lam=(1.0, 1.0), lam_d=1.0,
                      kT=1e-5, sdf=True):
    """Exact stationary structure factors of the *linearised lattice* update at
    one wavevector: the lattice algorithm (Eqs. algorithm, lattice finalstep)
    linearised about a uniform rest state, written in Fourier space as
    x_{n+1} = A x_n + B xi_n, and solved for the stationary covariance with the
    discrete Lyapunov equation P = A P A^H + B Xi B^H.

    This is a second formulation of the same update (population space, Fourier
    modes, a linear solve instead of a stochastic run); it contains the lattice
    corrections that the continuum result Eq. str-bin-hom lacks at large k.
    Returns (S_aa, S_ab, S_bb, S_uu per component averaged over D)."""
    import scipy.linalg as sl

    c = np.asarray(c, dtype=float)
    Q = len(w)
    D = int(np.count_nonzero(np.abs(c).sum(axis=0)))
    kv = np.zeros(3)
    kv[:len(k_vec)] = k_vec
    ph = np.exp(1j * (c @ kv))           # shift r -> r + c_i
    n = 2 * Q
    rt = rho[0] + rho[1]
    Rm = np.zeros((2 * Q, n), complex)   # R[s, a] as a linear form of f
    acc = []
    for q in range(2):
        qp = 1 - q
        rows = []
        for d in range(D):
            r = np.zeros(n, complex)
            r[qp * Q:(qp + 1) * Q] = -G * np.sum(w * c[:, d] * ph)
            rows.append(r)
        acc.append(rows)
    for s in range(2):
        for d in range(D):
            u = np.zeros(n, complex)
            u[0:Q] += c[:, d] / rt
            u[Q:2 * Q] += c[:, d] / rt
            u += 0.5 * (rho[0] * acc[0][d] + rho[1] * acc[1][d]) / rt
            j = np.zeros(n, complex)
            j[s * Q:(s + 1) * Q] = c[:, d]
            Rm[s * Q + 1 + d] = lam_d * (rho[s] * u - j) + (1 - lam_d / 2) * rho[s] * acc[s][d]
        for a in range(D + 1, Q):
            Rm[s * Q + a, s * Q:(s + 1) * Q] = -lam[s] * T[a]
    Bm = np.zeros((n, 2 * Q))
    for s in range(2):
        for i in range(Q):
            for a in range(Q):
                Bm[s * Q + i, s * Q + a] = w[i] * T[a, i] / N[a]
    S = np.diag(np.concatenate([np.exp(-1j * (c @ kv))] * 2))
    A = S @ (np.eye(n) + Bm @ Rm)
    Xi = np.zeros((2 * Q, 2 * Q))
    vj = (2 * lam_d - lam_d ** 2) * kT * rho[0] * rho[1] / rt if sdf else 0.0
    for d in range(D):
        a = 1 + d
        Xi[a, a] = Xi[Q + a, Q + a] = vj
        Xi[a, Q + a] = Xi[Q + a, a] = -vj
    for s in range(2):
        for a in range(D + 1, Q):
            Xi[s * Q + a, s * Q + a] = (2 * lam[s] - lam[s] ** 2) * N[a] * 3 * kT * rho[s]
    Qn = S @ Bm @ Xi @ Bm.T @ S.conj().T
    P = sl.solve_discrete_lyapunov(A, Qn, method="direct")
    eA = np.zeros(n)
    eA[:Q] = 1
    eB = np.zeros(n)
    eB[Q:] = 1
    suu = 0.0
    for d in range(D):
        # u_b = (jbar_t + F_t/2)/rho_t, linear in f
        e = np.zeros(n, complex)
        e[0:Q] += c[:, d] / rt
        e[Q:2 * Q] += c[:, d] / rt
        e += 0.5 * (rho[0] * acc[0][d] + rho[1] * acc[1][d]) / rt
        # the Fourier velocity is the form e^T x, so its variance is e^T P conj(e)
        # (P = <x x^H>); the force part of e is complex, so the order matters
        suu += (e @ P @ e.conj()).real / D
    return (eA @ P @ eA).real, (eA @ P @ eB).real, (eB @ P @ eB).real, suu


def multi_sk(kT, rho, G, alpha):
    """S_{s s'}(k) of an N-species mixture (App. D): the self-consistency
    condition mu alpha^{st} + sum_k rho^k gamma^{sk} alpha^{tk} + gamma^{st} = 0
    with alpha^{st} = G_{st} alpha(k) gives gamma = -mu A (1 + R A)^-1 and
    S = mu R + R gamma R = mu R (1 + A R)^-1, R = diag(rho), A = alpha G."""
    R = np.diag(np.asarray(rho, dtype=float))
    A = alpha * np.asarray(G, dtype=float)
    return kT / CS2 * R @ np.linalg.inv(np.eye(len(rho)) + A @ R)


def multi_lattice_linear_sk(c, w, T, N, k_vec, G, rho, tau, kT):
    """Exact stationary structure factors S_{s s'}(k) of the N-species lattice
    update (App. C-D) linearised about a uniform rest state: the same Fourier
    state-space model as lattice_linear_sk with ns species, per-species rates
    1/tau_s on the non-conserved modes, the common momentum rate
    ns / sum tau_s, forces between different species only and the projected
    momentum noise (2 lb_d - lb_d^2) kT (rho^s delta - rho^s rho^t / rho_t)."""
    import scipy.linalg as sl

    c = np.asarray(c, dtype=float)
    rho = np.asarray(rho, dtype=float)
    G = np.asarray(G, dtype=float) * (1 - np.eye(len(rho)))
    ns, Q = len(rho), len(w)
    D = int(np.count_nonzero(np.abs(c).sum(axis=0)))
    lam = 1.0 / np.asarray(tau, dtype=float)
    lam_d = ns / np.sum(tau)
    kv = np.zeros(3)
    kv[:len(k_vec)] = k_vec
    ph = np.exp(1j * (c @ kv))
    n = ns * Q
    rt = rho.sum()
    # acc[s][d]: the acceleration of species s as a linear form of f
    acc = np.zeros((ns, D, n), complex)
    for s in range(ns):
        for t in range(ns):
            for d in range(D):
                acc[s, d, t * Q:(t + 1) * Q] += -G[s, t] * np.sum(w * c[:, d] * ph)
    ub = np.zeros((D, n), complex)
    for d in range(D):
        for s in range(ns):
            ub[d, s * Q:(s + 1) * Q] += c[:, d] / rt
            ub[d] += 0.5 * rho[s] * acc[s, d] / rt
    Rm = np.zeros((n, n), complex)
    for s in range(ns):
        for d in range(D):
            j = np.zeros(n, complex)
            j[s * Q:(s + 1) * Q] = c[:, d]
            Rm[s * Q + 1 + d] = lam_d * (rho[s] * ub[d] - j) + (1 - lam_d / 2) * rho[s] * acc[s, d]
        for a in range(D + 1, Q):
            Rm[s * Q + a, s * Q:(s + 1) * Q] = -lam[s] * T[a]
    Bm = np.zeros((n, n))
    for s in range(ns):
        Bm[s * Q:(s + 1) * Q, s * Q:(s + 1) * Q] = (np.asarray(w)[:, None] * np.asarray(T).T) / np.asarray(N)[None, :]
    S = np.diag(np.concatenate([np.exp(-1j * (c @ kv))] * ns))
    A = S @ (np.eye(n) + Bm @ Rm)
    Xi = np.zeros((n, n))
    cov_d = (2 * lam_d - lam_d ** 2) * kT * (np.diag(rho) - np.outer(rho, rho) / rt)
    for d in range(D):
        a = 1 + d
        for s in range(ns):
            for t in range(ns):
                Xi[s * Q + a, t * Q + a] = cov_d[s, t]
    for s in range(ns):
        for a in range(D + 1, Q):
            Xi[s * Q + a, s * Q + a] = (2 * lam[s] - lam[s] ** 2) * N[a] * 3 * kT * rho[s]
    P = sl.solve_discrete_lyapunov(A, S @ Bm @ Xi @ Bm.T @ S.conj().T, method="direct")
    E = np.zeros((ns, n))
    for s in range(ns):
        E[s, s * Q:(s + 1) * Q] = 1
    return (E @ P @ E.T).real
