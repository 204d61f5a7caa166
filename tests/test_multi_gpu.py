"""GPU parity of the N-species update (App. C-D) through the flbm_m* C-ABI,
against the FP64 N-species oracle on the same seeded inputs and the same
counter-based noise, plus conservation, launch-shape invariance, a sampled
check on the full-size 256^3 three-species box and the three-species
structure factors against the linearised-lattice covariance.

Tolerances (element by element, relative to max |f|) are those of the
two-species float path: 1e-6 per step, 1e-4 after 1000 steps."""
import numpy as np
import pytest

import oracle
import theory
from paper_1410_5584_gb300 import D2Q9, D3Q19, FlbmError, Lattice, MultiLattice
from paper_1410_5584_gb300 import inputs

pytestmark = pytest.mark.gpu

RHOS = [1.0, 0.8, 0.6, 0.9]
TAUS = [1.0, 0.8, 1.25, 0.9]


def _couplings(ns, g, seed=0):
    rng = np.random.default_rng(seed)
    G = rng.uniform(0.5, 1.0, (ns, ns)) * g
    G = 0.5 * (G + G.T)
    np.fill_diagonal(G, 0.0)
    return G


def _state(lat, ns, shape, eps=0.02, seed=3):
    c, w, T, N = oracle.tables(lat)
    return inputs.random_populations(np.stack([w * r for r in RHOS[:ns]]), shape, eps, seed=seed)


def _pair(lat, ns, shape, kT, G, seed, **kw):
    nz, ny, nx = shape
    g = MultiLattice(lat, ns, nx, ny, nz, TAUS[:ns], kT, G, seed, **kw)
    o = oracle.MultiOracle(lat, ns, nx, ny, nz, TAUS[:ns], kT, G, seed)
    return g, o


def _rel(fg, fo):
    return np.max(np.abs(fg - fo)) / np.max(np.abs(fo))


CASES = [
    (D2Q9, 2, (1, 23, 37)),    # ragged: x not a multiple of the warp, odd y
    (D2Q9, 3, (1, 23, 37)),
    (D2Q9, 4, (1, 2, 2)),      # smallest box: every neighbour wraps
    (D2Q9, 3, (1, 64, 160)),   # several thread blocks along x plus a ragged tail
    (D3Q19, 2, (5, 4, 6)),
    (D3Q19, 3, (7, 6, 13)),
    (D3Q19, 4, (2, 2, 2)),
    (D3Q19, 3, (16, 12, 136)),
]


@pytest.mark.parametrize("lat,ns,shape", CASES)
@pytest.mark.parametrize("g", [0.0, 0.6])
def test_single_steps_match_oracle(lat, ns, shape, g):
    """Both in-place streaming parities (steps 1 and 2), with and without
    forces, unequal tau: <= 1e-6 relative per step."""
    G = _couplings(ns, g, seed=ns)
    f0 = _state(lat, ns, shape)
    gp, o = _pair(lat, ns, shape, 1e-4, G, 77)
    gp.set_populations(f0, step=41)
    o.set_f(f0, step=41)
    for k in range(1, 3):
        gp.step(1)
        o.step(1)
        assert _rel(gp.get_populations(), o.get_f()) <= 1e-6 * k
    assert gp.step_count == 43


@pytest.mark.parametrize("lat,ns,shape,nsteps", [
    (D2Q9, 3, (1, 48, 40), 1000),
    (D2Q9, 4, (1, 20, 24), 1000),
    (D3Q19, 3, (6, 8, 10), 300),
])
def test_many_steps_match_oracle(lat, ns, shape, nsteps):
    nz, ny, nx = shape
    G = _couplings(ns, 0.5, seed=1)
    rho = np.stack([inputs.perturbed_density(shape, RHOS[s], 1e-3, seed=1, species=s) for s in range(ns)])
    gp, o = _pair(lat, ns, shape, 1e-5, G, 1)
    gp.init(rho)
    o.set_f(gp.get_populations(), step=0)  # the oracle starts from the same float-rounded rest state
    gp.step(nsteps)
    o.step(nsteps)
    assert _rel(gp.get_populations(), o.get_f()) <= 1e-4


@pytest.mark.parametrize("lat,ns,shape", [(D2Q9, 3, (1, 17, 29)), (D3Q19, 4, (5, 6, 7))])
def test_moments_and_totals_match_oracle(lat, ns, shape):
    G = _couplings(ns, 0.7, seed=2)
    f0 = _state(lat, ns, shape, seed=5)
    gp, o = _pair(lat, ns, shape, 1e-4, G, 5)
    gp.set_populations(f0, step=0)
    o.set_f(f0, step=0)
    for k in range(2):  # natural and swapped layouts
        rg, ug, cg = gp.moments()
        ro, uo, co = o.moments()
        assert np.max(np.abs(rg - ro)) <= 1e-6 * np.max(ro)
        assert np.max(np.abs(ug - uo)) <= 1e-6 * np.max(np.abs(uo)) + 1e-9
        assert np.allclose(cg[:ns], co[:ns], rtol=1e-7)
        # total momentum: a sum of site momenta that largely cancel; the scale of
        # its rounding is the sum of their magnitudes
        assert np.max(np.abs(cg[ns:] - co[ns:])) <= 1e-6 * np.sum(np.abs(uo)) * sum(RHOS[:ns])
        gp.step(1)
        o.step(1)


@pytest.mark.parametrize("lat,ns,shape", [(D2Q9, 3, (1, 128, 128)), (D3Q19, 3, (32, 32, 32))])
def test_conservation_on_the_gpu(lat, ns, shape):
    """Every species mass (closed on the stored values) and the total momentum
    (projected momentum noise sums to zero) over 500 steps of a forced,
    fluctuating mixture."""
    nz, ny, nx = shape
    G = _couplings(ns, 0.6, seed=3)
    rho = np.stack([inputs.perturbed_density(shape, RHOS[s], 1e-2, seed=4, species=s) for s in range(ns)])
    gp = MultiLattice(lat, ns, nx, ny, nz, TAUS[:ns], 1e-5, G, 9, rho0=RHOS[:ns])
    gp.init(rho)
    _, _, c0 = gp.moments()
    gp.step(500)
    _, _, c1 = gp.moments()
    n = nx * ny * nz
    # each site and step rounds the stored rest population (the mass closure) by
    # at most half an ulp of w_0 rho0^s: a random walk of n * 500 uniform errors
    w0 = 4.0 / 9.0 if lat == D2Q9 else 1.0 / 3.0
    for s in range(ns):
        sigma = np.spacing(np.float32(w0 * RHOS[s])) / np.sqrt(12.0) * np.sqrt(n * 500)
        assert abs(c1[s] - c0[s]) <= 6 * sigma, (s, c1[s] - c0[s], sigma)
    # momentum: float rounding of the zero-sum noise and of the forces only
    assert np.all(np.abs(c1[ns:] - c0[ns:]) <= 1e-7 * n)


def test_launch_shapes_give_identical_results():
    shape, ns = (6, 20, 100), 3
    G = _couplings(ns, 0.6, seed=4)
    f0 = _state(D3Q19, ns, shape, seed=6)
    out = []
    for block in ((128, 1), (64, 2), (32, 4)):
        gp = MultiLattice(D3Q19, ns, 100, 20, 6, TAUS[:ns], 1e-4, G, 3, block=block)
        gp.set_populations(f0, step=0)
        gp.step(3)
        out.append(gp.get_populations())
        gp.close()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


@pytest.mark.parametrize("nsteps", [4, 5])
def test_checkpoint_restore_is_bit_identical(nsteps):
    """A checkpoint taken after an even or odd number of steps, restored into a
    fresh context, continues bit-identically; a corrupt or mismatched image is
    refused."""
    shape, ns = (4, 6, 10), 3
    G = _couplings(ns, 0.5, seed=9)
    a = MultiLattice(D3Q19, ns, 10, 6, 4, TAUS[:ns], 1e-4, G, 8, rho0=RHOS[:ns])
    a.set_populations(_state(D3Q19, ns, shape, seed=4), step=2)
    a.step(nsteps)
    img = a.checkpoint()
    a.step(6)
    b = MultiLattice(D3Q19, ns, 10, 6, 4, TAUS[:ns], 1e-4, G, 8, rho0=RHOS[:ns])
    b.restore(img)
    assert b.step_count == 2 + nsteps
    b.step(6)
    assert np.array_equal(a.get_populations(), b.get_populations())
    bad = bytearray(img)
    bad[-1] ^= 0x40
    with pytest.raises(FlbmError, match="FLBM_EINVAL"):
        b.restore(bytes(bad))
    other = MultiLattice(D3Q19, ns, 10, 6, 5, TAUS[:ns], 1e-4, G, 8)
    with pytest.raises(FlbmError, match="FLBM_EINVAL"):
        other.restore(img)


def test_two_species_without_noise_match_the_binary_context():
    """kT = 0: the N-species path with two species is the two-species update
    (lambdabar_d = 2 / (tau_A + tau_B) in both), to float rounding."""
    shape = (1, 30, 40)
    f0 = _state(D2Q9, 2, shape, seed=8)
    G = 0.9
    gm = MultiLattice(D2Q9, 2, 40, 30, 1, [0.8, 1.0], 0.0, [[0, G], [G, 0]], 1)
    gb = Lattice(D2Q9, 40, 30, 1, 0.8, 1.0, 0.0, G, 1)
    gm.set_populations(f0)
    gb.set_populations(f0)
    gm.step(20)
    gb.step(20)
    assert _rel(gm.get_populations(), gb.get_populations().reshape(2, 9, 1, 30, 40)) <= 2e-6


def test_nonpositive_density_is_reported():
    shape, ns = (1, 8, 8), 3
    f0 = _state(D2Q9, ns, shape)
    f0[1, :, 0, 3, 3] = -0.01
    gp = MultiLattice(D2Q9, ns, 8, 8, 1, TAUS[:ns], 1e-4, _couplings(ns, 0.3), 1)
    gp.set_populations(f0)
    gp.step(1)
    with pytest.raises(FlbmError, match="FLBM_ENONFINITE"):
        gp.sync()


def _axis_sk_definition(rho, axis):
    """S_st(k_m) = Re(rhohat_s conj rhohat_t) / N of one snapshot, from the
    densities [ns][z][y][x] (Sec. IV A, App. D)."""
    ax = 3 - axis
    prof = rho.sum(axis=tuple(a for a in (1, 2, 3) if a != ax))
    n = prof.shape[1]
    f = np.fft.fft(prof, axis=1)[:, 1:n // 2 + 1]
    return np.einsum("sk,tk->stk", f, np.conj(f)).real / rho[0].size


@pytest.mark.parametrize("lat,ns,shape", [(D2Q9, 3, (1, 12, 20)), (D2Q9, 2, (1, 7, 33)), (D3Q19, 4, (6, 10, 8)),
                                          (D3Q19, 3, (5, 7, 9))])
def test_structure_factor_snapshot_matches_oracle(lat, ns, shape):
    """One snapshot along every axis, in both streaming parities, against the
    DFT definition on the oracle's densities of the same state."""
    G = _couplings(ns, 0.5, seed=7)
    f0 = _state(lat, ns, shape, eps=0.05, seed=11)
    gp, o = _pair(lat, ns, shape, 1e-4, G, 3)
    gp.set_populations(f0, step=0)
    o.set_f(f0, step=0)
    D = 2 if lat == D2Q9 else 3
    for k in range(2):
        rho_o = o.moments()[0]
        for axis in range(D):
            gp.sf_reset()
            gp.sf_sample(axis)
            S, n = gp.structure_factor(axis)
            want = _axis_sk_definition(rho_o, axis)
            assert n == 1 and S.shape == want.shape
            assert np.max(np.abs(S - want)) <= 1e-4 * np.max(np.abs(want)), (k, axis)
        gp.step(1)
        o.step(1)


def test_structure_factor_accumulates_means():
    shape, ns = (1, 16, 24), 3
    gp = MultiLattice(D2Q9, ns, 24, 16, 1, TAUS[:ns], 1e-4, _couplings(ns, 0.3), 5, rho0=RHOS[:ns])
    gp.init()
    got = []
    for _ in range(3):
        gp.step(7)
        gp.sf_sample(1)
        got.append(_axis_sk_definition(gp.moments()[0], 1))
    S, n = gp.structure_factor(1, nk=5)
    assert n == 3
    assert np.allclose(S, np.mean(got, axis=0)[:, :, :5], rtol=1e-4, atol=1e-12)


def test_runtime_argument_errors():
    gp = MultiLattice(D2Q9, 3, 8, 8, 1, TAUS[:3], 1e-4, _couplings(3, 0.3), 1)
    with pytest.raises(FlbmError, match="FLBM_ESTATE"):
        gp.step(1)
    gp.init()
    with pytest.raises(FlbmError, match="FLBM_ESTATE"):
        gp.structure_factor(0)                      # no snapshot yet
    with pytest.raises(FlbmError, match="FLBM_EINVAL"):
        gp.sf_sample(2)                             # no z axis in 2D
    gp.sf_sample(0)
    with pytest.raises(FlbmError, match="FLBM_EINVAL"):
        gp.structure_factor(0, nk=5)                # nk > n_x / 2
    with pytest.raises(FlbmError, match="FLBM_EINVAL"):
        gp.site_populations([64])
    with pytest.raises(FlbmError, match="FLBM_EINVAL"):
        gp.init(-np.ones((3, 1, 8, 8)))


def _block_check(lat, ns, shape, steps_before, nsample, seed):
    """Sampled parity on a full-size box: for sampled sites r, the GPU's
    post-collision values f_i(r + c_i, n+1) against the oracle's update of the
    3^D block around r, drawn with r's global noise counters."""
    nz, ny, nx = shape
    D = 2 if lat == D2Q9 else 3
    c, w, T, N = oracle.tables(lat)
    Q = len(w)
    G = _couplings(ns, 0.5, seed=seed)
    gp = MultiLattice(lat, ns, nx, ny, nz, TAUS[:ns], 1e-5, G, seed, rho0=RHOS[:ns])
    gp.init(np.stack([inputs.perturbed_density(shape, RHOS[s], 1e-3, seed, s) for s in range(ns)]))
    gp.step(steps_before)
    rng = np.random.default_rng(seed)
    pts = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (nz // 2, 0, nx - 1)]
    pts += [tuple(int(rng.integers(0, m)) for m in (nz, ny, nx)) for _ in range(nsample)]
    if D == 2:
        pts = [(0, y, x) for (_, y, x) in pts]
    offs = [(dz, dy, dx) for dz in ((-1, 0, 1) if D == 3 else (0,)) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    blocks = [[(((z + dz) % nz) * ny + (y + dy) % ny) * nx + (x + dx) % nx for (dz, dy, dx) in offs]
              for (z, y, x) in pts]
    before = gp.site_populations(np.concatenate(blocks)).reshape(len(pts), len(offs), ns, Q)
    gp.step(1)
    dst = [[(((z + c[i, 2]) % nz) * ny + (y + c[i, 1]) % ny) * nx + (x + c[i, 0]) % nx for i in range(Q)]
           for (z, y, x) in pts]
    after = gp.site_populations(np.concatenate(dst)).reshape(len(pts), Q, ns, Q)
    bz = 3 if D == 3 else 1
    cz = 1 if D == 3 else 0
    worst = 0.0
    for k, (z, y, x) in enumerate(pts):
        fb = np.zeros((ns, Q, bz, 3, 3))
        for j, (dz, dy, dx) in enumerate(offs):
            fb[:, :, dz + 1 if D == 3 else 0, dy + 1, dx + 1] = before[k, j]
        o = oracle.MultiOracle(lat, ns, 3, 3, bz, TAUS[:ns], 1e-5, G, seed)
        o.set_rng_origin((nz, ny, nx), ((z - 1) % nz if D == 3 else 0, (y - 1) % ny, (x - 1) % nx))
        o.set_f(fb, step=steps_before)
        o.step(1)
        fo = o.get_f()
        for i in range(Q):
            ref = fo[:, i, (cz + c[i, 2]) % bz, 1 + c[i, 1], 1 + c[i, 0]]
            worst = max(worst, np.max(np.abs(after[k, i, :, i] - ref)) / np.max(np.abs(fo)))
        o.close()
    return worst


@pytest.mark.parametrize("steps_before", [2, 3])
def test_full_size_three_species_sampled_parity(steps_before):
    """The 256^3 D3Q19 three-species box the benchmark times, both parities."""
    assert _block_check(D3Q19, 3, (256, 256, 256), steps_before, 30, seed=1) <= 1e-6


def test_full_size_d2q9_four_species_sampled_parity():
    assert _block_check(D2Q9, 4, (1, 512, 512), 3, 40, seed=2) <= 1e-6


@pytest.mark.filterwarnings("ignore:An ill-conditioned matrix")
def test_three_species_structure_factors_against_lattice_theory():
    """64 x 16 box, rho = (1, 0.8, 0.6), tau = (1, 0.8, 1.25), G = 0.3 between
    all pairs: the device S_{s s'}(k_x) in bands of k against the
    linearised-lattice covariance, 20 batches of 200 snapshots."""
    nx, ny, ns, kT = 64, 16, 3, 1e-4
    rhos, taus = np.array(RHOS[:ns]), TAUS[:ns]
    G = 0.3 * (1 - np.eye(ns))
    gp = MultiLattice(D2Q9, ns, nx, ny, 1, taus, kT, G, 21, rho0=rhos)
    gp.init()
    gp.step(3000)
    batches = []
    for _ in range(20):
        gp.sf_reset()
        for _ in range(200):
            gp.step(10)
            gp.sf_sample(0)
        S, n = gp.structure_factor(0)
        assert n == 200
        batches.append(S)
    B = np.array(batches)
    c, w, T, N = oracle.tables(D2Q9)
    k = 2 * np.pi * np.arange(1, nx // 2 + 1) / nx
    lat = np.array([theory.multi_lattice_linear_sk(c, w, T, N, (kk, 0), G, rhos, taus, kT) for kk in k])
    for s in range(ns):
        for t in range(ns):
            scale = 3 * kT * np.sqrt(rhos[s] * rhos[t])
            for band in (k < 0.5, (k >= 0.5) & (k < 1.5), (k >= 1.5) & (k < 2.5), k >= 2.5):
                got = B[:, s, t, band].mean(axis=1)
                m, se = got.mean(), got.std(ddof=1) / np.sqrt(len(got))
                assert abs(m - lat[band, s, t].mean()) < 4 * se + 0.01 * scale, (s, t, m, lat[band, s, t].mean())


@pytest.mark.parametrize("lat,ns,shape", [(D2Q9, 3, (1, 17, 33)), (D2Q9, 2, (1, 2, 2)), (D3Q19, 4, (5, 7, 9)),
                                          (D3Q19, 3, (2, 2, 2))])
@pytest.mark.parametrize("full", [False, True])
def test_streaming_modes_are_bitwise_identical(lat, ns, shape, full):
    """In-place and two-array streaming of the N-species update give the same
    bits: populations after odd and even step counts, moments, S(k).  With
    every rate 1 (full) the two-array run is the moment-fed pair (the collide
    reads m_0 .. m_D from the density pass, not the populations) and the
    in-place run the population-reading collide: the same update, bit for bit
    on D2Q9 and to a few float roundings on D3Q19 (measured: up to 3e-8 on
    populations of 0.3 after a step, as close to the oracle either way)."""
    nz, ny, nx = shape
    G = _couplings(ns, 0.6, seed=12)
    f0 = _state(lat, ns, shape, seed=13)
    taus = [1.0] * ns if full else TAUS[:ns]
    runs = []
    for mode in ("in_place", "two_arrays"):
        gp = MultiLattice(lat, ns, nx, ny, nz, taus, 1e-4, G, 5, streaming=mode)
        gp.set_populations(f0, step=2)
        got = []
        for n in (1, 2, 4):
            gp.step(n)
            gp.sf_sample(0)
            got.append([gp.get_populations(), *gp.moments()])
        got.append([gp.structure_factor(0)[0]])
        runs.append(got)
    for a, b in zip(runs[0], runs[1]):
        for x, y in zip(a, b):
            if full and lat == D3Q19:
                # populations to 2e-7 of their size; velocities and S(k), small
                # differences of large numbers, to 1e-4 of theirs
                tol = 2e-7 if np.shape(x) == f0.shape else 1e-4
                assert np.max(np.abs(x - y)) <= tol * np.max(np.abs(y))
            else:
                assert np.array_equal(x, y)


def test_checkpoints_move_between_streaming_modes():
    shape, ns = (4, 6, 10), 3
    G = _couplings(ns, 0.5, seed=14)
    mk = lambda mode: MultiLattice(D3Q19, ns, 10, 6, 4, TAUS[:ns], 1e-4, G, 8, rho0=RHOS[:ns], streaming=mode)
    a = mk("two_arrays")
    a.set_populations(_state(D3Q19, ns, shape, seed=15), step=1)
    a.step(3)
    img = a.checkpoint()
    a.step(4)
    b = mk("in_place")
    b.restore(img)
    b.step(4)
    assert np.array_equal(a.get_populations(), b.get_populations())
    b.step(1)                                   # odd: swapped layout
    odd = b.checkpoint()
    with pytest.raises(FlbmError, match="FLBM_EINVAL"):
        mk("two_arrays").restore(odd)
    c = mk("in_place")
    c.restore(odd)
    assert np.array_equal(c.get_populations(), b.get_populations())


@pytest.mark.filterwarnings("ignore:An ill-conditioned matrix")
def test_d3q19_three_species_structure_factors_against_lattice_theory():
    """D3Q19, 24 x 6 x 6 box, rho = (1, 0.8, 0.6), tau = (1, 0.8, 1.25), G = 0.3
    between all pairs: the device S_{s s'}(k_x) in bands of k against the
    linearised-lattice covariance of the N-species D3Q19 update, 20 batches
    of 300 snapshots."""
    nx, ny, nz, ns, kT = 24, 6, 6, 3, 1e-4
    rhos, taus = np.array(RHOS[:ns]), TAUS[:ns]
    G = 0.3 * (1 - np.eye(ns))
    gp = MultiLattice(D3Q19, ns, nx, ny, nz, taus, kT, G, 31, rho0=rhos)
    gp.init()
    gp.step(3000)
    batches = []
    for _ in range(20):
        gp.sf_reset()
        for _ in range(300):
            gp.step(10)
            gp.sf_sample(0)
        batches.append(gp.structure_factor(0)[0])
    B = np.array(batches)
    c, w, T, N = oracle.tables(D3Q19)
    k = 2 * np.pi * np.arange(1, nx // 2 + 1) / nx
    lat = np.array([theory.multi_lattice_linear_sk(c, w, T, N, (kk, 0, 0), G, rhos, taus, kT) for kk in k])
    for s in range(ns):
        for t in range(ns):
            scale = 3 * kT * np.sqrt(rhos[s] * rhos[t])
            for band in (k < 1.0, (k >= 1.0) & (k < 2.2), k >= 2.2):
                got = B[:, s, t, band].mean(axis=1)
                m, se = got.mean(), got.std(ddof=1) / np.sqrt(len(got))
                assert abs(m - lat[band, s, t].mean()) < 4 * se + 0.015 * scale, (s, t, m, lat[band, s, t].mean())


@pytest.mark.parametrize("mode", ["two_arrays", "in_place"])
def test_graph_steps_match_direct_launches(mode):
    """N-species steps replayed from CUDA graphs (4, then 3 steps a graph)
    give the same bits as direct launches across calls of any length."""
    from paper_1410_5584_gb300 import flbm as F
    shape, ns = (1, 18, 26), 3
    G = _couplings(ns, 0.5, seed=21)
    f0 = _state(D2Q9, ns, shape, seed=22)
    runs = []
    for graphs in (0, 1):
        gp = MultiLattice(D2Q9, ns, 26, 18, 1, TAUS[:ns], 1e-4, G, 4, streaming=mode)
        if graphs:
            gp.set_option(F.OPT_GRAPH_STEPS, 4)
        gp.set_populations(f0, step=1)
        for n in (5, 1, 8):
            gp.step(n)
        if graphs:
            gp.set_option(F.OPT_GRAPH_STEPS, 3)
        gp.step(7)
        assert gp.step_count == 22
        runs.append(gp.get_populations())
    assert np.array_equal(runs[0], runs[1])


@pytest.mark.parametrize("lat,ns,shape", [(D2Q9, 3, (1, 23, 37)), (D3Q19, 3, (7, 6, 13)), (D3Q19, 4, (5, 4, 6))])
def test_moment_fed_pair_matches_oracle(lat, ns, shape):
    """Every rate 1 with two arrays: the moment-fed pair against the FP64
    oracle, element by element, 3 steps."""
    nz, ny, nx = shape
    G = _couplings(ns, 0.6, seed=21)
    f0 = _state(lat, ns, shape, seed=22)
    g = MultiLattice(lat, ns, nx, ny, nz, [1.0] * ns, 1e-4, G, 9)
    o = oracle.MultiOracle(lat, ns, nx, ny, nz, [1.0] * ns, 1e-4, G, 9)
    g.set_populations(f0, step=4)
    o.set_f(f0, step=4)
    g.step(3)
    o.step(3)
    assert _rel(g.get_populations(), o.get_f()) <= 3e-6
