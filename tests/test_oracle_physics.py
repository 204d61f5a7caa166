"""Pins of the oracle's lattice update against conservation laws, textbook
special cases, exact distributions and the paper's statistical predictions
(CPU only; the statistical runs take a few seconds each)."""
import numpy as np
import pytest

import oracle
import theory
from paper_1410_5584_gb300 import inputs

DIMS = {oracle.D2Q9: (2, 9), oracle.D3Q19: (3, 19)}


def _base(lat, rho_a, rho_b):
    c, w, T, N = oracle.tables(lat)
    return np.stack([w * rho_a, w * rho_b])


def _unstream(f, c):
    """Undo one push-streaming step: fstar_i(r) = f_i(r + c_i)."""
    out = np.empty_like(f)
    for i in range(f.shape[1]):
        out[:, i] = np.roll(f[:, i], shift=(-c[i, 2], -c[i, 1], -c[i, 0]), axis=(1, 2, 3))
    return out


@pytest.mark.parametrize("lat,shape", [(oracle.D2Q9, (1, 16, 32)), (oracle.D3Q19, (6, 8, 8))])
def test_mass_and_total_momentum_are_invariant(lat, shape):
    """R_0 = 0 conserves each species' mass; the common momentum rate and
    xibar' = -xibar make sum_s R_alpha = F_t,alpha (Sec. III, Eq. diffusionrelaxation;
    Sec. IV A), and the lattice force sums to zero over a periodic box, so the
    totals of rho^A, rho^B and jbar_t + F_t/2 are invariant (FP64: ~1e-13)."""
    nz, ny, nx = shape
    o = oracle.Oracle(lat, nx, ny, nz, 0.8, 1.0, 1e-4, 0.9, 42)
    f0 = inputs.random_populations(_base(lat, 1.0, 1.0), shape, 0.02, seed=3)
    o.set_f(f0)
    _, _, _, c0 = o.moments()
    o.step(60)
    _, _, _, c1 = o.moments()
    assert abs(c1[0] - c0[0]) / c0[0] < 1e-13
    assert abs(c1[1] - c0[1]) / c0[1] < 1e-13
    assert np.all(np.abs(c1[2:] - c0[2:]) < 1e-13 * c0[0])
    # the lattice force itself sums to zero: F_t = 2 (cons - sum jbar_t)
    c, w, T, N = oracle.tables(lat)
    f = o.get_f()
    jt = np.einsum("sixyz,id->d", f.reshape(2, len(w), -1, 1, 1), c.astype(float))
    D = DIMS[lat][0]
    assert np.all(np.abs(2.0 * (c1[2:2 + D] - jt[:D])) < 1e-12 * c0[0])


@pytest.mark.parametrize("lat,shape", [(oracle.D2Q9, (1, 64, 64)), (oracle.D3Q19, (16, 16, 16))])
@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_one_step_moment_variances(lat, shape, tau):
    """From a uniform rest state the post-collision non-conserved moments are
    exactly the noise (m^eq = Phi = mbar = 0 there), so their variances over sites
    are those of Eq. new-noise: (2 lb - lb^2) N_a (kT/c_T^2) rho for a > D and
    (2 lb_d - lb_d^2) kT rho rho'/rho_t for the momenta, with xibar' = -xibar
    exactly (Sec. IV A, Sec. V A)."""
    nz, ny, nx = shape
    D, Q = DIMS[lat]
    kT, ra, rb = 1e-4, 0.7, 1.3
    o = oracle.Oracle(lat, nx, ny, nz, tau, tau, kT, 0.3, 7)
    o.init(np.full(nx * ny * nz, ra), np.full(nx * ny * nz, rb))
    o.step(1)
    c, w, T, N = oracle.tables(lat)
    fs = _unstream(o.get_f(), c)
    m = np.einsum("ai,sixyz->saxyz", T, fs).reshape(2, Q, -1)
    base = np.einsum("ai,si->sa", T, _base(lat, ra, rb))
    dm = m - base[:, :, None]
    lb = 1.0 / tau
    nsite = dm.shape[2]
    tol = 5.0 * np.sqrt(2.0 / nsite)
    for s, rho in enumerate((ra, rb)):
        assert np.all(np.abs(dm[s, 0]) < 1e-14)
        for a in range(D + 1, Q):
            var = (2 * lb - lb * lb) * N[a] * 3 * kT * rho
            assert abs(dm[s, a].var() / var - 1.0) < tol, (s, a)
            assert abs(dm[s, a].mean()) < 5.0 * np.sqrt(var / nsite)
    vj = (2 * lb - lb * lb) * kT * ra * rb / (ra + rb)
    for a in range(1, D + 1):
        assert abs(dm[0, a].var() / vj - 1.0) < tol
        assert np.all(np.abs(dm[0, a] + dm[1, a]) < 1e-15)
    # transport/ghost noises of the two species are independent
    for a in range(D + 1, Q):
        assert abs(np.corrcoef(dm[0, a], dm[1, a])[0, 1]) < 5.0 / np.sqrt(nsite)


def test_uniform_state_is_a_fixed_point_without_noise():
    """kT = 0: a uniform rest state has zero force and stays exactly uniform."""
    o = oracle.Oracle(oracle.D3Q19, 6, 5, 4, 0.8, 1.1, 0.0, 0.9, 1)
    o.init(np.full(120, 1.0), np.full(120, 0.7))
    f0 = o.get_f()
    o.step(20)
    assert np.max(np.abs(o.get_f() - f0)) < 1e-15


def _wave_rate(o, amp, n1, n2):
    o.step(n1)
    a1 = amp()
    o.step(n2 - n1)
    a2 = amp()
    return -np.log(a2 / a1) / (n2 - n1)


@pytest.mark.parametrize("lat,nx,tau", [(oracle.D2Q9, 128, 1.0), (oracle.D2Q9, 128, 0.7),
                                        (oracle.D3Q19, 64, 1.0)])
def test_shear_wave_decays_at_lattice_viscosity(lat, nx, tau):
    """kT = 0, G = 0: a transverse velocity wave decays as exp(-nu k^2 t) with
    nu = c_s^2 (1/lambdabar_s - 1/2) (Eq. lattice-freq; Chapman-Enskog)."""
    ny, nz = (4, 1) if lat == oracle.D2Q9 else (2, 2)
    o = oracle.Oracle(lat, nx, ny, nz, tau, tau, 0.0, 0.0, 1)
    c, w, T, N = oracle.tables(lat)
    k = 2 * np.pi / nx
    prof = np.sin(k * np.arange(nx))
    uy = 1e-4 * prof
    f = np.zeros((2, len(w), nz, ny, nx))
    for s in range(2):
        for i in range(len(w)):
            cu = c[i, 1] * uy
            f[s, i] = w[i] * 0.5 * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uy * uy)
    o.set_f(f)

    def amp():
        return 2 * (o.moments()[2][1].mean(axis=(0, 1)) * prof).mean()

    rate = _wave_rate(o, amp, 200, 800)
    assert rate == pytest.approx(theory.shear_viscosity(1.0 / tau) * k * k, rel=2e-3)


@pytest.mark.parametrize("lat,nx,taus", [(oracle.D2Q9, 128, (1.0, 1.0)), (oracle.D2Q9, 128, (0.8, 1.0)),
                                         (oracle.D3Q19, 64, (1.0, 1.0))])
def test_concentration_wave_decays_at_mutual_diffusivity(lat, nx, taus):
    """kT = 0, G = 0: an interdiffusion wave (rho_t uniform) decays as
    exp(-D k^2 t), D = c_s^2 (1/lambdabar_d - 1/2), lambdabar_d the common
    momentum rate (Sec. III; the Chapman-Enskog result the paper cites in Sec. VI)."""
    ny, nz = (4, 1) if lat == oracle.D2Q9 else (2, 2)
    o = oracle.Oracle(lat, nx, ny, nz, taus[0], taus[1], 0.0, 0.0, 1)
    k = 2 * np.pi / nx
    prof = np.sin(k * np.arange(nx))
    ra = np.broadcast_to(0.5 * (1 + 1e-3 * prof), (nz, ny, nx))
    rb = np.broadcast_to(0.5 * (1 - 1e-3 * prof), (nz, ny, nx))
    o.init(ra, rb)

    def amp():
        a, b, u, cons = o.moments()
        return 2 * ((a - b).mean(axis=(0, 1)) * prof).mean()

    lam_d = 1.0 / taus[0] if taus[0] == taus[1] else 2.0 / sum(taus)
    rate = _wave_rate(o, amp, 200, 800)
    assert rate == pytest.approx(theory.diffusivity(lam_d) * k * k, rel=2e-3)


def test_structure_factor_transform_of_a_planted_wave():
    """S(k_m) = |sum_r drho e^{-i k_m x}|^2 / N: a planted cosine of amplitude eps
    at m0 gives (eps nx ny / 2)^2 / N at m0 and zero elsewhere."""
    nx, ny, m0, eps = 32, 4, 3, 1e-3
    o = oracle.Oracle(oracle.D2Q9, nx, ny, 1, 1.0, 1.0, 0.0, 0.0, 1)
    x = np.arange(nx)
    ra = np.broadcast_to(1.0 + eps * np.cos(2 * np.pi * m0 * x / nx), (1, ny, nx))
    rb = np.broadcast_to(1.0 - 2 * eps * np.cos(2 * np.pi * m0 * x / nx), (1, ny, nx))
    o.init(ra, rb)
    o.sf_sample(axis=0)
    saa, sab, sbb, suu, n = o.structure_factor()
    assert n == 1
    expect = (eps * nx * ny / 2) ** 2 / (nx * ny)
    assert saa[m0 - 1] == pytest.approx(expect, rel=1e-9)
    assert sbb[m0 - 1] == pytest.approx(4 * expect, rel=1e-9)
    assert sab[m0 - 1] == pytest.approx(-2 * expect, rel=1e-9)
    others = np.delete(np.arange(nx // 2), m0 - 1)
    assert np.all(np.abs(saa[others]) < 1e-20) and np.all(np.abs(suu) < 1e-20)


def test_theory_structure_functions_reduce_to_appendix_e():
    """Eq. structurefunctions at k -> 0 (alpha = G) equals the Shan-Chen
    thermodynamic results of App. E."""
    for rho_t0, C0, G in [(2.0, 0.5, 0.4), (2.0, 0.3, 0.2), (1.5, 0.7, 0.6)]:
        a = theory.structure_functions(1e-5, rho_t0, C0, G)
        b = theory.hydro_k0(1e-5, rho_t0, C0, G)
        assert np.allclose(a, b, rtol=1e-12)


# --------------------------------------------------------------------------
# second formulation: the update written in population space (Sec. V B)
# --------------------------------------------------------------------------

def _population_space_step(f, lat, tau, kT, G, seed, step, sdf=True, noise_rho0=None,
                           force_velocity=False, lambda_d=None, mode_rates=None, ghost_noise=False):
    """One step of the FLBE written with the MRT matrix
    Lambda_ij = w_i sum_a lambdabar_a T_ai T_aj / N_a (Sec. V B) acting on f^eq
    and (I - Lambda/2) acting on the Hermite forcing Phi_i, plus the noise mapped
    to populations, then np.roll streaming.  Shares only the tables and the noise
    draws with the oracle.

    Options, each the population-space statement of one oracle option:
    sdf=False drops the shared momentum noise (the no-sdf control of Sec. VI A);
    noise_rho0=(rA, rB) puts fixed reference densities in the amplitudes of
    Eq. new-noise instead of the local ones; force_velocity=True takes the
    species velocity inside Phi as v = jbar/rho + a/2 instead of
    rho v = jbar + R_j/2 (Eq. 2system); lambda_d overrides the common momentum
    rate (Sec. III); mode_rates {(s, a): lambdabar} overrides single modes;
    ghost_noise=True draws the non-conserved noise as one Gaussian per
    population, of variance mu w_i rho(r + c_i) (the density where the
    population lands), mapped to the non-conserved modes."""
    c, w, T, N = oracle.tables(lat)
    D, Q = DIMS[lat]
    cf = c.astype(float)
    lam = np.zeros((2, Q))
    lam_d = 1.0 / tau[0] if tau[0] == tau[1] else 2.0 / (tau[0] + tau[1])
    if lambda_d is not None:
        lam_d = lambda_d
    for s in range(2):
        lam[s, 1:] = 1.0 / tau[s]
        lam[s, 1:D + 1] = lam_d
    for (s, a), lb in (mode_rates or {}).items():
        lam[s, a] = lb
    Lam = [np.einsum("i,a,ai,aj->ij", w, lam[s] / N, T, T) for s in range(2)]
    nz, ny, nx = f.shape[2:]
    rho = f.sum(axis=1)
    acc = np.zeros((2, 3, nz, ny, nx))
    for s in range(2):
        for i in range(Q):
            nb = np.roll(rho[1 - s], shift=(-c[i, 2], -c[i, 1], -c[i, 0]), axis=(0, 1, 2))
            acc[s] += -G * w[i] * nb[None] * cf[i][:, None, None, None]
    j = np.einsum("sixyz,id->sdxyz", f, cf)
    rt = rho[0] + rho[1]
    u = (j[0] + j[1]) / rt + 0.5 * (rho[0] * acc[0] + rho[1] * acc[1]) / rt

    def feq(r, uu):
        cu = np.einsum("id,dxyz->ixyz", cf, uu)
        usq = (uu * uu).sum(axis=0)
        return w[:, None, None, None] * r * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * usq)

    def force(r, a, v):
        ca = np.einsum("id,dxyz->ixyz", cf, a)
        cv = np.einsum("id,dxyz->ixyz", cf, v)
        av = (a * v).sum(axis=0)
        return w[:, None, None, None] * r * (3 * ca + 9 * (ca * cv - av / 3))

    xi = np.zeros((2, Q, nz, ny, nx))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                site = (z * ny + y) * nx + x
                nr = (rho[0, z, y, x], rho[1, z, y, x]) if noise_rho0 is None else noise_rho0
                vj = (2 * lam_d - lam_d ** 2) * kT * nr[0] * nr[1] / (nr[0] + nr[1])
                for a in range(1, D + 1):
                    g = oracle.gaussian(seed, site, step, 0, a)
                    xi[0, a, z, y, x] = (np.sqrt(vj) if sdf else 0.0) * g
                    xi[1, a, z, y, x] = -xi[0, a, z, y, x]
                for s in range(2):
                    if ghost_noise:
                        eta = np.array([oracle.gaussian(seed, site, step, s + 2, i + 1) for i in range(Q)])
                        dest = np.array([rho[s, (z + c[i, 2]) % nz, (y + c[i, 1]) % ny, (x + c[i, 0]) % nx]
                                         if noise_rho0 is None else noise_rho0[s] for i in range(Q)])
                        xs = np.sqrt(3 * kT * w * dest) * eta
                    for a in range(D + 1, Q):
                        if ghost_noise:
                            xi[s, a, z, y, x] = np.sqrt(2 * lam[s, a] - lam[s, a] ** 2) * (T[a] @ xs)
                            continue
                        var = (2 * lam[s, a] - lam[s, a] ** 2) * N[a] * 3 * kT * nr[s]
                        xi[s, a, z, y, x] = np.sqrt(var) * oracle.gaussian(seed, site, step, s, a)
    out = np.empty_like(f)
    I = np.eye(Q)
    for s in range(2):
        noise = np.einsum("i,ai,axyz->ixyz", w, T / N[:, None], xi[s])
        zero = np.zeros_like(u)
        d1 = (np.einsum("ij,jxyz->ixyz", Lam[s], feq(rho[s], u) - f[s])
              + np.einsum("ij,jxyz->ixyz", I - Lam[s] / 2, force(rho[s], acc[s], zero)) + noise)
        Rj = np.einsum("ixyz,id->dxyz", d1, cf)
        v = j[s] / rho[s] + 0.5 * acc[s] if force_velocity else (j[s] + 0.5 * Rj) / rho[s]
        d = (np.einsum("ij,jxyz->ixyz", Lam[s], feq(rho[s], u) - f[s])
             + np.einsum("ij,jxyz->ixyz", I - Lam[s] / 2, force(rho[s], acc[s], v)) + noise)
        post = f[s] + d
        for i in range(Q):
            out[s, i] = np.roll(post[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2))
    return out


# One entry per oracle option branch: (oracle options, mode-rate overrides,
# keyword arguments of the population-space form).  The reference densities
# (1.4, 0.5) differ from the state's local ones (about 1.0 and 0.8), so that a
# wrong density in the noise amplitude shows.
_OPTION_CASES = {
    "default": ({}, {}, {}),
    "no_sdf": ({"sdf": 0}, {}, {"sdf": False}),
    "noise_rho_reference": ({"noise_rho": 1, "rho0_a": 1.4, "rho0_b": 0.5}, {},
                            {"noise_rho0": (1.4, 0.5)}),
    "force_velocity": ({"force_velocity": 1}, {}, {"force_velocity": True}),
    "lambda_d": ({"lambda_d": 1.3}, {}, {"lambda_d": 1.3}),
    "mode_rates": ({}, {(0, 4): 1.5, (1, 5): 0.6, (0, 8): 1.9, (1, 8): 0.3}, {}),
    "ghost_noise": ({"ghost_noise": 1}, {(0, 4): 1.5, (1, 8): 0.6}, {"ghost_noise": True}),
    "all": ({"noise_rho": 1, "rho0_a": 1.4, "rho0_b": 0.5, "force_velocity": 1, "lambda_d": 0.9},
            {(0, 6): 1.2, (1, 7): 1.7},
            {"noise_rho0": (1.4, 0.5), "force_velocity": True, "lambda_d": 0.9}),
}


@pytest.mark.parametrize("lat,shape", [(oracle.D2Q9, (1, 4, 5)), (oracle.D3Q19, (3, 3, 4))])
@pytest.mark.parametrize("case", sorted(_OPTION_CASES))
def test_moment_space_update_equals_population_space_form(lat, shape, case):
    """The oracle's moment-space update equals the population-space MRT form of
    Sec. V B (Lambda_ij, Hermite f^eq and Phi, noise mapped to populations) on a
    random non-uniform state with G != 0, tau_A != tau_B, over three steps, for
    the default update and for every option branch of the oracle: no shared
    momentum noise (Sec. VI A), reference densities in Eq. new-noise, the
    alternative species velocity inside Phi (Eq. 2system), an overridden
    common momentum rate (Sec. III) and single-mode rates."""
    tau, kT, G, seed = (0.8, 1.1), 1e-3, 0.7, 99
    opts, rates, kw = _OPTION_CASES[case]
    f = inputs.random_populations(_base(lat, 1.0, 0.8), shape, 0.05, seed=5)
    o = oracle.Oracle(lat, shape[2], shape[1], shape[0], tau[0], tau[1], kT, G, seed, **opts)
    for (s, a), lb in rates.items():
        o.set_mode_rate(s, a, lb)
    o.set_f(f, step=10)
    ref = f.copy()
    for n in range(3):
        ref = _population_space_step(ref, lat, tau, kT, G, seed, 10 + n, mode_rates=rates, **kw)
    o.step(3)
    assert np.max(np.abs(o.get_f() - ref)) < 1e-13


@pytest.mark.parametrize("lat,shape", [(oracle.D2Q9, (1, 64, 64)), (oracle.D3Q19, (12, 12, 12))])
@pytest.mark.parametrize("noise_rho", [0, 1])
def test_one_step_variances_follow_the_density_option(lat, shape, noise_rho):
    """Eq. new-noise on a non-uniform state: with every rate 1 the
    post-collision ghost moments are exactly the noise (m^eq = Phi = 0 on the
    ghosts), so ghost_a(r) / sqrt(N_a 3 kT rho(r)) is a standard Gaussian over
    sites when the local densities enter the amplitude, and
    ghost_a(r) / sqrt(N_a 3 kT rho0) when the reference densities do.  The
    densities vary by a factor of three across the box and rho0 sits far from
    them, so the wrong density (or a wrong factor) moves the variance well
    outside the bound."""
    nz, ny, nx = shape
    D, Q = DIMS[lat]
    kT = 1e-4
    rho0 = (2.5, 0.2)
    rng = np.random.Generator(np.random.PCG64(17))
    ra = rng.uniform(0.5, 1.5, size=shape)
    rb = rng.uniform(0.3, 0.9, size=shape)
    o = oracle.Oracle(lat, nx, ny, nz, 1.0, 1.0, kT, 0.0, 23, noise_rho=noise_rho,
                      rho0_a=rho0[0], rho0_b=rho0[1])
    o.init(ra, rb)
    o.step(1)
    c, w, T, N = oracle.tables(lat)
    m = np.einsum("ai,sixyz->saxyz", T, _unstream(o.get_f(), c)).reshape(2, Q, -1)
    nsite = m.shape[2]
    tol = 5.0 * np.sqrt(2.0 / nsite)
    ghosts = range(D + 1 + (3 if lat == oracle.D2Q9 else 6), Q)
    for s, rho in enumerate((ra.ravel(), rb.ravel())):
        amp_rho = np.full(nsite, rho0[s]) if noise_rho else rho
        for a in ghosts:
            z = m[s, a] / np.sqrt(N[a] * 3 * kT * amp_rho)
            assert abs(z.var() - 1.0) < tol, (s, a, z.var())
            assert abs(z.mean()) < 5.0 / np.sqrt(nsite)
    # the shared momentum noise, G = 0 and rest state: R_j = xi exactly
    nr = (np.full(nsite, rho0[0]), np.full(nsite, rho0[1])) if noise_rho else (ra.ravel(), rb.ravel())
    vj = kT * nr[0] * nr[1] / (nr[0] + nr[1])
    for a in range(1, D + 1):
        z = m[0, a] / np.sqrt(vj)
        assert abs(z.var() - 1.0) < tol
        assert np.all(np.abs(m[0, a] + m[1, a]) < 1e-15)


# --------------------------------------------------------------------------
# statistical predictions (Sec. VI A)
# --------------------------------------------------------------------------

def _sk_run(lat, nx, ny, nz, G, rho0, kT, burn, steps, every, seed=1, sdf=True):
    o = oracle.Oracle(lat, nx, ny, nz, 1.0, 1.0, kT, G, seed, sdf=sdf)
    N = nx * ny * nz
    o.init(np.full(N, rho0), np.full(N, rho0))
    o.step(burn)
    snaps = []
    for _ in range(steps // every):
        o.step(every)
        o.sf_reset()
        o.sf_sample(0)
        snaps.append(np.stack(o.structure_factor()[:4]))
    return np.array(snaps)


@pytest.mark.parametrize("lat,ny,nz,steps", [(oracle.D2Q9, 2, 1, 30000), (oracle.D3Q19, 2, 2, 12000)])
def test_ideal_mixture_structure_factor_is_flat(lat, ny, nz, steps):
    """G = 0 (Sec. VI A, Fig. 1 set-up on a 64-long periodic box): S_rho,rho =
    S_rho',rho' = kT rho0 / c_T^2 at every k, S_rho,rho' = 0 and the baricentric
    velocity structure factor kT/rho_t0 (Eqs. str-bin-hom, str-bin-hom-vel);
    parameters rho0 = 0.5, kT = 1e-4, all lambdabar = 1."""
    nx, rho0, kT = 64, 0.5, 1e-4
    snaps = _sk_run(lat, nx, ny, nz, 0.0, rho0, kT, 2000, steps, 10)
    m, se = theory.batch_means(snaps)
    keep = slice(0, nx // 2 - 1)  # k = pi excluded (a Nyquist mode of the lattice)
    th_rr = 3 * kT * rho0
    for idx in (0, 2):
        er = m[idx, keep] / th_rr
        er_se = se[idx, keep] / th_rr
        assert abs(er.mean() - 1.0) < 3 * np.sqrt((er_se ** 2).sum()) / er.size + 0.01
        assert np.all(np.abs(er - 1.0) < 5 * er_se + 0.02)
    ab = m[1, keep] / kT
    assert np.all(np.abs(ab) < 5 * se[1, keep] / kT + 0.02)
    eru = m[3, keep] / theory.s_vb(kT, 2 * rho0)
    eru_se = se[3, keep] / theory.s_vb(kT, 2 * rho0)
    assert abs(eru.mean() - 1.0) < 3 * np.sqrt((eru_se ** 2).sum()) / eru.size + 0.01


def test_no_sdf_negative_control_is_detected():
    """Without noise on the species momenta ("no-sdf", Sec. VI A, Fig. 1) the
    densities are under-thermalised and S_rho,rho' != 0; the run agrees instead
    with the linearised-lattice prediction for that scheme."""
    nx, rho0, kT = 64, 0.5, 1e-4
    snaps = _sk_run(oracle.D2Q9, nx, 2, 1, 0.0, rho0, kT, 2000, 12000, 10, sdf=False)
    m, se = theory.batch_means(snaps)
    k = 2 * np.pi * np.arange(1, nx // 2 + 1) / nx
    low = k < 1.0
    assert np.all(m[1, low] / kT > 0.3)
    assert np.all(m[0, low] / (3 * kT * rho0) < 0.8)
    c, w, T, N = oracle.tables(oracle.D2Q9)
    for mi in (4, 10, 16):
        pred = theory.lattice_linear_sk(c, w, T, N, [k[mi]], 0.0, rho=(rho0, rho0), kT=kT, sdf=False)
        assert abs(m[0, mi] - pred[0]) < 5 * se[0, mi] + 0.03 * pred[0]
        assert abs(m[1, mi] - pred[1]) < 5 * se[1, mi] + 0.03 * abs(pred[1])


def test_interacting_mixture_structure_factor():
    """G = 0.4, rho0 = rho0' = 1, kT = 1e-5 (Sec. VI A, Figs. 2 and 4): at small k
    the run follows Eq. str-bin-hom with alpha = G sin k / k; at every k it follows
    the exact linearised-lattice prediction, which departs from the continuum
    formula at k >~ 0.5 (lattice corrections the continuum theory omits)."""
    nx, G, rho0, kT = 64, 0.4, 1.0, 1e-5
    snaps = _sk_run(oracle.D2Q9, nx, 2, 1, G, rho0, kT, 2000, 30000, 10)
    m, se = theory.batch_means(snaps)
    k = 2 * np.pi * np.arange(1, nx // 2 + 1) / nx
    al = theory.alpha_lattice(G, k)
    small = k < 0.5
    cont_rr = theory.s_rho_rho(kT, rho0, rho0, al)
    cont_rp = theory.s_rho_rhop(kT, rho0, rho0, al)
    assert np.all(np.abs(m[0, small] - cont_rr[small]) < 3 * se[0, small] + 0.05 * cont_rr[small])
    assert np.all(np.abs(m[1, small] - cont_rp[small]) < 3 * se[1, small] + 0.05 * np.abs(cont_rp[small]))
    c, w, T, N = oracle.tables(oracle.D2Q9)
    for mi in range(0, nx // 2 - 1, 3):
        pred = theory.lattice_linear_sk(c, w, T, N, [k[mi]], G, rho=(rho0, rho0), kT=kT)
        assert abs(m[0, mi] - pred[0]) < 5 * se[0, mi] + 0.02 * pred[0], mi
        assert abs(m[1, mi] - pred[1]) < 5 * se[1, mi] + 0.02 * pred[0], mi
        assert abs(m[3, mi] - pred[3]) < 5 * se[3, mi] + 0.02 * pred[3], mi


@pytest.mark.parametrize("lat,shape", [(oracle.D2Q9, (1, 6, 10)), (oracle.D3Q19, (3, 4, 5))])
def test_full_relaxation_forgets_the_non_conserved_moments(lat, shape):
    """With lambdabar_a = 1 on every non-conserved mode (and lambdabar_d = 1),
    Eq. algorithm gives m*_a = m^eq_a + Phi_a/2 + xi_a: the old m_a drops out,
    so a step depends on each species' populations only through rho^s and
    jbar^s.  Adding to the populations anything orthogonal to the density and
    momentum rows of T (a kernel vector of rows 0 .. D) leaves the state
    after one step unchanged, to FP64 rounding.  At tau = 0.8 the same
    change does alter the result (the check has teeth).  This is the
    property the library's moment-fed collide relies on."""
    nz, ny, nx = shape
    c, w, T, N = oracle.tables(lat)
    D, Q = DIMS[lat]
    f0 = inputs.random_populations(_base(lat, 1.0, 0.8), shape, 0.02, seed=21)
    rng = np.random.default_rng(5)
    # project random vectors onto the complement of rows 0 .. D of T
    C = np.asarray(T[:D + 1], dtype=float)                   # (D + 1) x Q
    P = np.eye(Q) - C.T @ np.linalg.solve(C @ C.T, C)
    delta = np.einsum("ij,sjzyx->sizyx", P, rng.normal(0.0, 3e-3, f0.shape))
    assert np.max(np.abs(np.einsum("aj,sjzyx->sazyx", C, delta))) < 1e-15
    f1 = f0 + delta
    for tau, same in ((1.0, True), (0.8, False)):
        out = []
        for f in (f0, f1):
            o = oracle.Oracle(lat, nx, ny, nz, tau, tau, 1e-4, 0.7, 13)
            o.set_f(f, step=4)
            o.step(1)
            out.append(o.get_f())
            o.close()
        diff = np.max(np.abs(out[0] - out[1]))
        if same:
            assert diff < 1e-15, diff
        else:
            assert diff > 1e-5, diff


@pytest.mark.parametrize("lat,shape", [(oracle.D2Q9, (1, 400, 8)), (oracle.D3Q19, (40, 40, 8))])
@pytest.mark.parametrize("ghost", [0, 1])
def test_non_conserved_noise_covariance_in_a_density_gradient(lat, shape, ghost):
    """The off-diagonal noise of the non-conserved modes (the correction left
    open after Eq. finalstep, Sec. V B and Sec. VII, in the reading of one
    Gaussian per population at the density where it lands): one step from a
    rest state (G = 0, every rate 1, so the post-collision non-conserved
    modes are the noise alone) on a density that varies along x.  For each
    column x the covariance of those modes over the sites of the column is
    mu sum_i T_ai T_bi w_i rho(x + c_ix) with the option, and the diagonal
    mu N_a rho(x) of Eq. new-noise without it; each entry is compared with
    its own sampling error (family-wise 3 standard errors).  A wrong
    neighbour (the source density instead of the destination), a missing
    weight or a diagonal-only draw fails the option case, whose
    off-diagonal correlations between modes reach 0.2 - 0.35 here."""
    nz, ny, nx = shape
    D, Q = DIMS[lat]
    kT, mu = 1e-4, 3e-4
    c, w, T, N = oracle.tables(lat)
    xs = np.arange(nx)
    prof = 1.0 + 0.6 * np.sin(2 * np.pi * xs / nx)
    ra = np.broadcast_to(prof, shape).copy()
    rb = np.broadcast_to(0.7 * prof[::-1], shape).copy()
    o = oracle.Oracle(lat, nx, ny, nz, 1.0, 1.0, kT, 0.0, 31, ghost_noise=ghost)
    o.init(ra, rb)
    o.step(1)
    m = np.einsum("ai,sizyx->sazyx", T, _unstream(o.get_f(), c))  # [s][a][z][y][x]
    nc = list(range(D + 1, Q))
    nsamp = ny * nz
    npairs = len(nc) * (len(nc) + 1) // 2
    zcrit = theory.family_sigma(2 * nx * npairs, nbatch=10 ** 6)  # Gaussian quantile for the whole family
    worst_off = 0.0
    for s, rho in enumerate((prof, 0.7 * prof[::-1])):
        for x in range(nx):
            dest = np.array([rho[(x + c[i, 0]) % nx] for i in range(Q)])
            if ghost:
                pred = mu * np.einsum("ai,bi,i->ab", T[nc], T[nc], w * dest)
            else:
                pred = mu * rho[x] * np.diag(N[nc])
            v = m[s][nc][:, :, :, x].reshape(len(nc), -1)
            cov = v @ v.T / nsamp  # the noise has mean zero
            # standard error of a sample covariance of Gaussians: sqrt((C_aa C_bb + C_ab^2) / n)
            se = np.sqrt((np.outer(np.diag(pred), np.diag(pred)) + pred ** 2) / nsamp)
            assert np.all(np.abs(cov - pred) < zcrit * se), (s, x)
            sd = np.sqrt(np.diag(pred))
            worst_off = max(worst_off, np.max(np.abs(pred - np.diag(np.diag(pred))) / np.outer(sd, sd)))
    if ghost:
        assert worst_off > 0.1
