"""GPU parity: the CUDA library, called through its C-ABI, against the FP64
oracle on the same seeded inputs and the same counter-based noise.

Tolerances (element by element, relative to max |f|): 1e-6 per step and 1e-4
after 1000 steps for float storage; the 16-bit formats are bounded by their
rounding of the stored deviation (2^-11 relative for half, 2^-8 for bfloat16).
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1410_5584_gb300 import D2Q9, D3Q19, FlbmError, Lattice
from paper_1410_5584_gb300 import flbm as F
from paper_1410_5584_gb300 import inputs

pytestmark = pytest.mark.gpu

ORACLE_THREADS = 8


def _pair(lat, shape, tau=(1.0, 1.0), kT=1e-4, G=0.0, seed=1, storage="f32", **opts):
    nz, ny, nx = shape
    g = Lattice(lat, nx, ny, nz, tau[0], tau[1], kT, G, seed, storage=storage, **opts)
    o = oracle.Oracle(lat, nx, ny, nz, tau[0], tau[1], kT, G, seed, **opts)
    o.set_threads(ORACLE_THREADS)
    return g, o


def _random_state(lat, shape, rho=(1.0, 0.8), eps=0.02, seed=3):
    c, w, T, N = oracle.tables(lat)
    return inputs.random_populations(np.stack([w * rho[0], w * rho[1]]), shape, eps, seed=seed)


def _rel(fg, fo):
    return np.max(np.abs(fg - fo)) / np.max(np.abs(fo))


SHAPES = [
    (D2Q9, (1, 23, 37)),   # ragged: x not a multiple of the warp, odd y
    (D2Q9, (1, 2, 2)),     # smallest box: every neighbour wraps
    (D2Q9, (1, 64, 160)),  # several thread blocks along x plus a ragged tail
    (D3Q19, (7, 6, 13)),
    (D3Q19, (2, 2, 2)),
    (D3Q19, (16, 12, 136)),
]


@pytest.mark.parametrize("lat,shape", SHAPES)
@pytest.mark.parametrize("G,tau", [(0.0, (1.0, 1.0)), (0.9, (0.8, 1.0))])
def test_single_steps_match_oracle(lat, shape, G, tau):
    """Both in-place streaming parities (steps 1 and 2), G = 0 and G > 0,
    tau_A != tau_B: <= 1e-6 relative per step."""
    f0 = _random_state(lat, shape)
    g, o = _pair(lat, shape, tau=tau, kT=1e-4, G=G, seed=77)
    g.set_populations(f0, step=41)
    o.set_f(f0, step=41)
    for k in range(1, 3):
        g.step(1)
        o.step(1)
        assert _rel(g.get_populations(), o.get_f()) <= 1e-6 * k
    assert g.step_count == 43


@pytest.mark.parametrize("lat,shape,tau,kT,G,rho", [
    (D2Q9, (1, 64, 64), (1.0, 1.0), 1e-4, 0.0, (0.5, 0.5)),     # the 64^2 ideal-mixture workload
    (D2Q9, (1, 48, 40), (0.8, 1.0), 1e-5, 0.9, (1.0, 1.0)),     # Shan-Chen mixture, G rho0 = 0.9
    (D3Q19, (12, 10, 16), (1.0, 1.0), 1e-5, 0.9, (1.0, 1.0)),
])
def test_thousand_steps_match_oracle(lat, shape, tau, kT, G, rho):
    nz, ny, nx = shape
    n = nx * ny * nz
    ra = inputs.perturbed_density(shape, rho[0], 1e-3, seed=1, species=0)
    rb = inputs.perturbed_density(shape, rho[1], 1e-3, seed=1, species=1)
    g, o = _pair(lat, shape, tau=tau, kT=kT, G=G, seed=1)
    g.init(ra, rb)
    # the oracle starts from the same float-rounded rest state
    o.set_f(g.get_populations(), step=0)
    g.step(1000)
    o.step(1000)
    assert _rel(g.get_populations(), o.get_f()) <= 1e-4
    assert n > 0


@pytest.mark.parametrize("lat,shape", [(D2Q9, (1, 9, 11)), (D3Q19, (4, 5, 6))])
@pytest.mark.parametrize("opts", [
    dict(sdf=0),
    dict(noise_rho=1, rho0_a=1.1, rho0_b=0.7),
    dict(force_velocity=1),
    dict(lambda_d=1.3),
])
def test_options_match_oracle(lat, shape, opts):
    f0 = _random_state(lat, shape, rho=(1.1, 0.7))
    g, o = _pair(lat, shape, tau=(0.9, 1.2), kT=3e-4, G=0.5, seed=5, **opts)
    g.set_populations(f0, step=0)
    o.set_f(f0, step=0)
    g.step(2)
    o.step(2)
    assert _rel(g.get_populations(), o.get_f()) <= 2e-6


@pytest.mark.parametrize("lat,shape", [(D2Q9, (1, 9, 11)), (D3Q19, (4, 5, 6))])
def test_per_mode_rates_match_oracle(lat, shape):
    Q = 9 if lat == D2Q9 else 19
    D = 2 if lat == D2Q9 else 3
    f0 = _random_state(lat, shape)
    g, o = _pair(lat, shape, tau=(1.0, 1.0), kT=1e-4, G=0.4, seed=8)
    for s in range(2):
        for a in range(D + 1, Q):
            lam = 0.6 + 0.05 * a + 0.3 * s
            g.set_mode_rate(s, a, lam)
            o.set_mode_rate(s, a, lam)
    g.set_populations(f0)
    o.set_f(f0)
    g.step(2)
    o.step(2)
    assert _rel(g.get_populations(), o.get_f()) <= 2e-6


@pytest.mark.parametrize("lat,shape", [(D2Q9, (1, 20, 24)), (D3Q19, (6, 7, 8))])
def test_moments_and_totals_match_oracle(lat, shape):
    f0 = _random_state(lat, shape)
    g, o = _pair(lat, shape, tau=(0.8, 1.0), kT=1e-4, G=0.9, seed=4)
    g.set_populations(f0)
    o.set_f(f0)
    g.step(3)
    o.step(3)
    ga, gb, gu, gc = g.moments()
    oa, ob, ou, oc = o.moments()
    assert np.max(np.abs(ga - oa)) <= 1e-6 * np.max(oa)
    assert np.max(np.abs(gb - ob)) <= 1e-6 * np.max(ob)
    assert np.max(np.abs(gu - ou)) <= 1e-6 * np.max(np.abs(ou)) + 1e-9
    assert np.allclose(gc[:2], oc[:2], rtol=1e-7)
    assert np.all(np.abs(gc[2:] - oc[2:]) <= 1e-6 * oc[0])


@pytest.mark.parametrize("lat,shape", [(D2Q9, (1, 64, 64)), (D3Q19, (16, 16, 16))])
def test_conservation_on_the_gpu(lat, shape):
    """Mass of each species and total momentum over 1000 float steps (G = 0.9):
    drift bounded by float rounding, ~1e-6 relative."""
    nz, ny, nx = shape
    g = Lattice(lat, nx, ny, nz, 0.8, 1.0, 1e-5, 0.9, 3)
    g.init(inputs.perturbed_density(shape, 1.0, 1e-3, 3, 0), inputs.perturbed_density(shape, 1.0, 1e-3, 3, 1))
    c0 = g.moments(fields=False)
    g.step(1000)
    c1 = g.moments(fields=False)
    assert abs(c1[0] - c0[0]) <= 2e-6 * c0[0]
    assert abs(c1[1] - c0[1]) <= 2e-6 * c0[1]
    assert np.all(np.abs(c1[2:] - c0[2:]) <= 2e-6 * c0[0])


@pytest.mark.parametrize("lat,shape,axis", [(D2Q9, (1, 16, 32), 0), (D2Q9, (1, 16, 32), 1),
                                            (D3Q19, (8, 6, 10), 2)])
def test_structure_factor_matches_oracle(lat, shape, axis):
    f0 = _random_state(lat, shape, eps=0.01)
    g, o = _pair(lat, shape, tau=(1.0, 1.0), kT=1e-4, G=0.3, seed=9)
    g.set_option("sf_axis", axis)
    g.set_populations(f0)
    o.set_f(f0)
    for _ in range(3):
        g.step(2)
        o.step(2)
        g.sf_sample()
        o.sf_sample(axis)
    gs = g.structure_factor(axis)
    os_ = o.structure_factor()
    assert gs[4] == os_[4] == 3
    # The two states differ by float rounding of the populations (~1e-7), so each
    # Fourier amplitude carries a relative error ~1e-5 after the large mean
    # cancels; S_ab's error therefore scales with sqrt(S_aa S_bb).
    for k in (0, 2, 3):
        assert np.allclose(gs[k], os_[k], rtol=2e-5, atol=0)
    assert np.all(np.abs(gs[1] - os_[1]) <= 2e-5 * np.sqrt(os_[0] * os_[2]))


@pytest.mark.parametrize("storage,bits", [("f16", 11), ("bf16", 8)])
@pytest.mark.parametrize("lat,shape", [(D2Q9, (1, 16, 24)), (D3Q19, (6, 6, 8))])
def test_sixteen_bit_storage_against_oracle(storage, bits, lat, shape):
    """Populations stored as 16-bit deviations from w_i rho0: after one step
    the error is the rounding of the stored deviation."""
    c, w, T, N = oracle.tables(lat)
    base = np.stack([w, w])[:, :, None, None, None]
    f0 = _random_state(lat, shape, rho=(1.0, 1.0), eps=0.01)
    g, o = _pair(lat, shape, tau=(1.0, 1.0), kT=1e-5, G=0.9, seed=2, storage=storage)
    g.set_populations(f0)
    start = g.get_populations()  # f0 with its deviations rounded to the format
    assert np.max(np.abs(start - f0)) <= 2.0 ** -bits * np.max(np.abs(f0 - base))
    o.set_f(start)
    g.step(1)
    o.step(1)
    fo = o.get_f()
    dev = np.max(np.abs(fo - base))
    assert np.max(np.abs(g.get_populations() - fo)) <= 2.0 ** -bits * dev + 1e-6 * np.max(fo)


@pytest.mark.parametrize("nsteps", [10, 11])
def test_checkpoint_restore_is_bit_identical(nsteps):
    shape = (5, 6, 7)
    g = Lattice(D3Q19, 7, 6, 5, 0.8, 1.0, 1e-4, 0.9, 123)
    g.init(inputs.perturbed_density(shape, 1.0, 1e-3, 1, 0), inputs.perturbed_density(shape, 1.0, 1e-3, 1, 1))
    g.step(nsteps)
    image = g.checkpoint()
    g.step(7)
    a = g.get_populations()
    h = Lattice(D3Q19, 7, 6, 5, 1.0, 1.0, 0.0, 0.0, 999)  # parameters come from the image
    h.restore(image)
    assert h.step_count == nsteps
    h.step(7)
    assert np.array_equal(a, h.get_populations())
    bad = bytearray(image)
    bad[-1] ^= 0xFF
    with pytest.raises(FlbmError) as e:
        h.restore(bytes(bad))
    assert e.value.status == F.EINVAL
    wrong = Lattice(D3Q19, 8, 6, 5, 1.0, 1.0, 0.0, 0.0, 1)
    with pytest.raises(FlbmError):
        wrong.restore(image)


def test_nonpositive_density_is_reported():
    """A site whose density is driven negative is flagged on the device and
    reported by the next synchronising call; re-initialising clears it."""
    shape = (1, 8, 8)
    g = Lattice(D2Q9, 8, 8, 1, 1.0, 1.0, 1e-4, 0.0, 1)
    f0 = _random_state(D2Q9, shape)
    f0[0, :, 0, 3, 3] = -0.05  # species A density -0.45 at one site
    g.set_populations(f0)
    g.step(1)
    with pytest.raises(FlbmError) as e:
        g.sync()
    assert e.value.status == F.ENONFINITE
    g.init()
    g.step(2)
    g.sync()


def test_runtime_argument_errors():
    g = Lattice(D2Q9, 8, 8, 1, 1.0, 1.0, 1e-4, 0.0, 1)
    g.init()
    with pytest.raises(FlbmError):
        g.site_populations([64])
    with pytest.raises(FlbmError):
        g.structure_factor(0)  # no snapshot yet
    with pytest.raises(FlbmError):
        g.set_option("storage", 1)  # buffers exist
    g.sf_sample()
    with pytest.raises(FlbmError):
        g.structure_factor(0, nk=5)  # nk > nx/2


def _block_check(lat, shape, steps_before, nsample, seed, tau=(0.8, 1.0), storage="f32", bits=None):
    """Sampled parity on a full-size box: for sampled sites r, the GPU's
    post-collision values f_i(r + c_i, n+1) against the oracle's update of the
    3^D block around r, drawn with r's global noise counters.  Returns the
    worst error relative to max |f|; with ``bits`` (16-bit storage) the error
    is first reduced by the format's rounding of the stored deviation,
    2^-bits max |f - w rho0|, and the rest is returned relative to max |f|."""
    nz, ny, nx = shape
    D = 2 if lat == D2Q9 else 3
    Q = 9 if lat == D2Q9 else 19
    c, w, T, N = oracle.tables(lat)
    g = Lattice(lat, nx, ny, nz, tau[0], tau[1], 1e-5, 0.9, seed, storage=storage)
    g.init(inputs.perturbed_density(shape, 1.0, 1e-3, seed, 0), inputs.perturbed_density(shape, 1.0, 1e-3, seed, 1))
    g.step(steps_before)
    rng = np.random.default_rng(seed)
    pts = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (nz // 2, 0, nx - 1)]
    pts += [tuple(int(rng.integers(0, m)) for m in (nz, ny, nx)) for _ in range(nsample)]
    if D == 2:
        pts = [(0, y, x) for (_, y, x) in pts]
    offs = [(dz, dy, dx) for dz in ((-1, 0, 1) if D == 3 else (0,)) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    blocks = []
    for (z, y, x) in pts:
        ids = [(((z + dz) % nz) * ny + (y + dy) % ny) * nx + (x + dx) % nx for (dz, dy, dx) in offs]
        blocks.append(ids)
    before = g.site_populations(np.concatenate(blocks)).reshape(len(pts), len(offs), 2, Q)
    g.step(1)
    bz = 3 if D == 3 else 1
    worst = 0.0
    dst_ids = []
    for (z, y, x) in pts:
        dst_ids.append([(((z + c[i, 2]) % nz) * ny + (y + c[i, 1]) % ny) * nx + (x + c[i, 0]) % nx for i in range(Q)])
    after = g.site_populations(np.concatenate(dst_ids)).reshape(len(pts), Q, 2, Q)
    for k, (z, y, x) in enumerate(pts):
        fb = np.zeros((2, Q, bz, 3, 3))
        for j, (dz, dy, dx) in enumerate(offs):
            fb[:, :, dz + 1 if D == 3 else 0, dy + 1, dx + 1] = before[k, j]
        o = oracle.Oracle(lat, 3, 3, bz, tau[0], tau[1], 1e-5, 0.9, seed)
        o.set_rng_origin((nz, ny, nx), ((z - 1) % nz if D == 3 else 0, (y - 1) % ny, (x - 1) % nx))
        o.set_f(fb, step=steps_before)
        o.step(1)
        fo = o.get_f()
        cz = 1 if D == 3 else 0
        ref = np.stack([fo[:, i, (cz + c[i, 2]) % bz, 1 + c[i, 1], 1 + c[i, 0]] for i in range(Q)], axis=1)
        got = np.stack([after[k, i, :, i] for i in range(Q)], axis=1)  # [species][i]
        err = np.abs(got - ref)
        if bits is not None:
            # a moving population's word rounds its own deviation; the rest
            # population closes the site's mass on the stored words, so it
            # carries the rounding of all of them
            dev = np.abs(ref - w[None, :])
            allow = 2.0 ** -bits * dev
            allow[:, 0] = 2.0 ** -bits * dev.sum(axis=1)
            err = np.maximum(0.0, err - allow)
        worst = max(worst, np.max(err) / np.max(np.abs(fo)))
        o.close()
    return worst


@pytest.mark.parametrize("steps_before", [2, 3])
def test_full_size_d3q19_sampled_parity(steps_before):
    """The 256^3 D3Q19 box the benchmark times, both streaming parities."""
    assert _block_check(D3Q19, (256, 256, 256), steps_before, 40, seed=1) <= 1e-6


def test_full_size_d2q9_sampled_parity():
    """The 512^2 D2Q9 Shan-Chen box."""
    assert _block_check(D2Q9, (1, 512, 512), 3, 60, seed=2) <= 1e-6


@pytest.mark.parametrize("steps_before", [2, 3])
def test_full_size_d3q19_sampled_parity_full_relaxation(steps_before):
    """The instance the benchmark times: D3Q19 256^3 at tau = 1 on both
    species, two-array streaming, so the moment-fed collide runs (the density
    pass stores m_0 .. m_D and the collide reads those instead of the
    populations)."""
    assert _block_check(D3Q19, (256, 256, 256), steps_before, 40, seed=4, tau=(1.0, 1.0)) <= 1e-6


@pytest.mark.parametrize("storage,bits", [("f16", 11), ("bf16", 8)])
def test_full_size_d3q19_sampled_parity_sixteen_bit(storage, bits):
    """The 16-bit storage forms at 256^3 and tau = 1 (moment-fed collide):
    within the format's rounding of the stored deviation plus the float
    tolerance of 1e-6 relative."""
    assert _block_check(D3Q19, (256, 256, 256), 2, 30, seed=5, tau=(1.0, 1.0), storage=storage, bits=bits) <= 1e-6


def _unstream_np(f, c):
    out = np.empty_like(f)
    for i in range(f.shape[1]):
        out[:, i] = np.roll(f[:, i], shift=(-c[i, 2], -c[i, 1], -c[i, 0]), axis=(1, 2, 3))
    return out


@pytest.mark.parametrize("lat,shape", [(D2Q9, (1, 24, 40)), (D3Q19, (6, 8, 12))])
@pytest.mark.parametrize("tau", [(1.0, 1.0), (0.8, 1.0)])
def test_noise_itself_matches_oracle(lat, shape, tau):
    """Parity on the noise alone (Eq. new-noise, Box-Muller on the Philox
    uniforms): the same state is stepped with kT and with kT = 0 on both
    sides, and the difference, projected on the moment basis, is compared mode
    by mode and species by species relative to that mode's own largest value.
    The start is close to the rest state, so the float deviations the GPU
    stores are small and their rounding is far below the noise.  Every
    non-conserved mode, the shared momentum noise, and all three Box-Muller
    pairs of each Philox block are covered, as are draws with u1 > 31/32
    (checked below on the oracle's own uniforms)."""
    nz, ny, nx = shape
    D = 2 if lat == D2Q9 else 3
    Q = 9 if lat == D2Q9 else 19
    c, w, T, N = oracle.tables(lat)
    f0 = _random_state(lat, shape, rho=(1.0, 0.8), eps=1e-4, seed=9)
    seed, step0, kT = 12345, 17, 1e-3
    res = {}
    for side in ("gpu", "oracle"):
        for t in (kT, 0.0):
            if side == "gpu":
                h = Lattice(lat, nx, ny, nz, tau[0], tau[1], t, 0.6, seed, rho0_a=1.0, rho0_b=0.8)
                h.set_populations(f0, step=step0)
                h.step(1)
                res[side, t] = h.get_populations()
            else:
                o = oracle.Oracle(lat, nx, ny, nz, tau[0], tau[1], t, 0.6, seed)
                o.set_f(f0, step=step0)
                o.step(1)
                res[side, t] = o.get_f()
                o.close()
    dm = {}
    for side in ("gpu", "oracle"):
        df = _unstream_np(res[side, kT] - res[side, 0.0], c)
        dm[side] = np.einsum("ai,sixyz->saxyz", T, df).reshape(2, Q, -1)
    ref, got = dm["oracle"], dm["gpu"]
    # the noise carries no mass (R_0 = 0): exactly on the oracle, to the float
    # rounding of the stored deviations on the GPU
    assert np.max(np.abs(ref[:, 0])) < 1e-12 and np.max(np.abs(got[:, 0])) < 1e-6 * np.max(np.abs(got))
    for s in range(2):
        for a in range(1, Q):
            scale = np.max(np.abs(ref[s, a]))
            assert scale > 1e-4
            assert np.max(np.abs(got[s, a] - ref[s, a])) <= 1e-5 * scale, (s, a)
    # the draws include radii from the series branch (u1 > 31/32)
    nsite = nx * ny * nz
    hits = 0
    for site in range(nsite):
        for sp in range(2):
            for b in range((Q + 4) // 6):
                x = oracle.philox4x32_10([site, step0, sp, b], [seed & 0xFFFFFFFF, seed >> 32])
                words = [x[0] >> 11, x[2] >> 11, ((x[0] & 0x7FF) << 10) | (x[1] & 0x3FF)]
                hits += sum(((u + 1) / 2.0 ** 21) > 31 / 32 for u in words)
    assert hits > 0


@pytest.mark.parametrize("lat,shape", [(D2Q9, (1, 2, 37)), (D2Q9, (1, 3, 130)), (D2Q9, (1, 64, 64)),
                                       (D3Q19, (2, 5, 7)), (D3Q19, (3, 4, 9)), (D3Q19, (9, 6, 140))])
def test_fused_and_two_kernel_schedules_agree(lat, shape):
    """The fused single-launch step (densities reused from L2) is deterministic
    run to run (bitwise), and agrees with the density-then-collide kernels to
    rounding (the two instantiations may contract multiply-adds differently),
    both parities, including boxes with fewer than four slices."""
    nz, ny, nx = shape
    f0 = _random_state(lat, shape)
    out = []
    for sched in ("fused", "fused", "two_kernels"):
        g = Lattice(lat, nx, ny, nz, 0.8, 1.0, 1e-4, 0.9, 6, streaming=F.STREAMING["in_place"])
        g.set_option("schedule", F.SCHEDULE[sched])
        g.set_populations(f0, step=3)
        g.step(5)
        out.append(g.get_populations())
    assert np.array_equal(out[0], out[1])
    assert _rel(out[0], out[2]) <= 5e-7


@pytest.mark.parametrize("lat,shape,slabs", [(D2Q9, (1, 2, 37), 8), (D2Q9, (1, 3, 130), 8), (D2Q9, (1, 17, 33), 8),
                                             (D2Q9, (1, 64, 64), 5), (D3Q19, (2, 5, 7), 8), (D3Q19, (3, 4, 9), 3),
                                             (D3Q19, (9, 6, 140), 8), (D3Q19, (16, 8, 8), 16)])
def test_overlap_schedule_matches_two_kernels_bitwise(lat, shape, slabs):
    """The slab-overlapped schedule runs the same per-site arithmetic as the
    two-kernel schedule, so after any number of steps, split into any calls
    (both streaming parities, both starting slabs of the alternation), the
    states agree bit for bit, in place and with two arrays; boxes with fewer
    than 3 planes fall back to the two-kernel schedule.  Kernel timing does
    not change the result."""
    nz, ny, nx = shape
    f0 = _random_state(lat, shape)
    ref = Lattice(lat, nx, ny, nz, 0.8, 1.0, 1e-4, 0.9, 6, streaming=F.STREAMING["in_place"])
    ref.set_option("schedule", F.SCHEDULE["two_kernels"])
    ref.set_populations(f0, step=3)
    ref.step(8)
    want = ref.get_populations()
    for timing, streaming in ((0, "in_place"), (1, "in_place"), (0, "two_arrays"), (1, "two_arrays")):
        g = Lattice(lat, nx, ny, nz, 0.8, 1.0, 1e-4, 0.9, 6, streaming=F.STREAMING[streaming])
        g.set_option("schedule", F.SCHEDULE["overlap"])
        g.set_option("slabs", slabs)
        g.set_option("kernel_timing", timing)
        g.set_populations(f0, step=3)
        for n in (1, 2, 5):
            g.step(n)
        assert g.step_count == 11
        assert np.array_equal(g.get_populations(), want)
        if timing:
            ms, cnt = g.kernel_times()
            assert cnt["collide"] == 8 and ms["collide"] > 0 and ms["density"] > 0


def test_fused_step_wait_timeout_is_reported():
    """Failure detection without a GPU fault: a dependency wait that can never
    be satisfied gives up after its time limit, the kernel returns, the host
    reads FLBM_ETIMEOUT, and re-initialising restores a usable context."""
    g = Lattice(D3Q19, 16, 8, 6, 1.0, 1.0, 1e-4, 0.5, 1, streaming=F.STREAMING["in_place"])
    g.set_option("schedule", F.SCHEDULE["fused"])
    g.init()
    g.set_option("wait_limit_ms", 50)
    g.set_option("test_stall", 1)
    g.step(1)
    with pytest.raises(FlbmError) as e:
        g.sync()
    assert e.value.status == F.ETIMEOUT
    g.set_option("test_stall", 0)
    g.init()
    g.step(3)
    g.sync()
    assert g.moments(fields=False)[0] == pytest.approx(16 * 8 * 6, rel=1e-6)


@pytest.mark.parametrize("lat,shape", [(D2Q9, (1, 2, 37)), (D2Q9, (1, 17, 33)), (D3Q19, (2, 2, 2)),
                                       (D3Q19, (5, 7, 45))])
@pytest.mark.parametrize("tau", [(1.0, 1.0), (0.8, 1.0)])
def test_streaming_modes_are_bitwise_identical(lat, shape, tau):
    """In-place and two-array streaming compute the same update bit for bit:
    populations after odd and even step counts split over several calls,
    observables and the axis structure factor; with all rates 1 (the collide
    that skips the non-conserved projections and reads the moments m_0 .. m_D
    that the density pass stored instead of the populations) and with general
    rates."""
    nz, ny, nx = shape
    f0 = _random_state(lat, shape)
    runs = []
    for mode in ("in_place", "two_arrays"):
        g = Lattice(lat, nx, ny, nz, tau[0], tau[1], 1e-4, 0.7, 6, streaming=F.STREAMING[mode])
        assert g.get_option("streaming") == F.STREAMING[mode]
        g.set_populations(f0, step=3)
        got = []
        for n in (1, 2, 4):
            g.step(n)
            g.sf_sample()
            got.append((g.get_populations(), g.moments()))
        got.append(g.structure_factor(0))
        runs.append(got)
    for a, b in zip(runs[0][:-1], runs[1][:-1]):
        assert np.array_equal(a[0], b[0])
        for x, y in zip(a[1], b[1]):
            assert np.array_equal(x, y)
    for x, y in zip(runs[0][-1], runs[1][-1]):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_checkpoints_move_between_streaming_modes():
    """An image holds the current state in its layout: a two-array image (always
    the natural layout) restores into either mode and continues bitwise; an
    in-place image taken after an odd step count (swapped layout) restores
    into an in-place context only."""
    shape = (4, 6, 10)
    f0 = _random_state(D3Q19, shape)
    mk = lambda mode: Lattice(D3Q19, 10, 6, 4, 0.8, 1.0, 1e-4, 0.7, 6, streaming=F.STREAMING[mode])
    a = mk("two_arrays")
    a.set_populations(f0, step=3)
    a.step(3)
    img = a.checkpoint()
    a.step(4)
    b = mk("in_place")
    b.restore(img)
    b.step(4)
    assert np.array_equal(a.get_populations(), b.get_populations())
    c = mk("in_place")
    c.set_populations(f0, step=3)
    c.step(1)
    odd = c.checkpoint()
    d = mk("two_arrays")
    with pytest.raises(FlbmError, match="FLBM_EINVAL"):
        d.restore(odd)
    e = mk("in_place")
    e.restore(odd)
    assert np.array_equal(e.get_populations(), c.get_populations())


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("lat,shape", [(D2Q9, (1, 9, 70)), (D3Q19, (4, 6, 33))])
def test_moment_fed_collide_matches_the_population_reading_one(lat, shape, storage):
    """At full relaxation the two-kernel step feeds the collide the moments
    m_0 .. m_D that the density pass stored; the overlap schedule keeps the
    collide that reads the populations.  Both give bitwise the same update, in
    both streaming modes, launched directly and replayed from CUDA graphs."""
    nz, ny, nx = shape
    f0 = _random_state(lat, shape)
    out = []
    for mode, sched, graphs in (("two_arrays", "overlap", 0), ("in_place", "overlap", 0),
                                ("two_arrays", "two_kernels", 0), ("in_place", "two_kernels", 0),
                                ("two_arrays", "two_kernels", 4), ("in_place", "two_kernels", 4)):
        g = Lattice(lat, nx, ny, nz, 1.0, 1.0, 1e-4, 0.8, 9, storage=storage, streaming=F.STREAMING[mode])
        g.set_option("schedule", F.SCHEDULE[sched])
        g.set_option("slabs", 3)
        g.set_option("graph_steps", graphs)
        g.set_populations(f0, step=5)
        g.step(3)
        g.step(6)
        out.append(g.get_populations())
    for o in out[1:]:
        assert np.array_equal(out[0], o)


@pytest.mark.parametrize("lat,shape", [(D2Q9, (1, 17, 33)), (D3Q19, (5, 7, 45))])
@pytest.mark.parametrize("mode", ["two_arrays", "in_place"])
def test_full_relaxation_collide_matches_the_general_one(lat, shape, mode):
    """With every rate 1 the collide that skips the non-conserved projections
    runs.  It is deterministic run to run (bitwise), and it agrees with the
    general kernel (forced by a test hook) to rounding: the two instances may
    contract multiply-adds differently."""
    nz, ny, nx = shape
    f0 = _random_state(lat, shape)
    out = []
    for general in (0, 0, 1):
        g = Lattice(lat, nx, ny, nz, 1.0, 1.0, 1e-4, 0.7, 6, streaming=F.STREAMING[mode],
                    test_general_collide=general)
        g.set_populations(f0, step=3)
        g.step(5)
        out.append(g.get_populations())
    assert np.array_equal(out[0], out[1])
    assert _rel(out[0], out[2]) <= 5e-7


@pytest.mark.parametrize("lat,shape", [(D2Q9, (1, 17, 33)), (D3Q19, (5, 7, 9))])
@pytest.mark.parametrize("mode", ["two_arrays", "in_place"])
def test_graph_steps_match_direct_launches(lat, shape, mode):
    """Steps replayed from CUDA graphs (graph_steps = 4, then 3) give the same
    bits as steps launched one by one, over calls that are not multiples of
    the graph length and start at either parity; an option changed between
    calls (no species-momentum noise) takes effect in the graphs too."""
    nz, ny, nx = shape
    f0 = _random_state(lat, shape)
    runs = []
    for graphs in (0, 1):
        g = Lattice(lat, nx, ny, nz, 0.8, 1.0, 1e-4, 0.7, 6, streaming=F.STREAMING[mode])
        if graphs:
            g.set_option("graph_steps", 4)
        g.set_populations(f0, step=3)
        for n in (5, 1, 8):
            g.step(n)
        if graphs:
            g.set_option("graph_steps", 3)
        g.set_option("sdf", 0)
        g.step(7)
        assert g.step_count == 24
        runs.append(g.get_populations())
    assert np.array_equal(runs[0], runs[1])


@pytest.mark.parametrize("shape", [(50, 60, 70), (3, 5, 7)])
@pytest.mark.parametrize("direct", [0, 1])
def test_moments_copy_out_through_the_staging_buffer(shape, direct):
    """flbm_moments hands the fields to the caller's (pageable) buffers through
    the pinned staging buffer in alternating chunks, copied on host threads
    (direct_host 0), or, where the GPU shares the host's page tables, stored
    by the kernel straight into them (direct_host 1, the default): on a box
    whose fields span several chunks (210,000 sites) and on a tiny one, the
    densities come back as the initial field (float-rounded), the velocity of
    the rest state is exactly zero, and after a few noisy steps both routes
    give the same bits, also into arrays viewed at an odd offset."""
    nz, ny, nx = shape
    rng = np.random.default_rng(4)
    ra = rng.uniform(0.5, 1.5, size=shape).astype(np.float32).astype(np.float64)
    rb = rng.uniform(0.2, 0.9, size=shape).astype(np.float32).astype(np.float64)
    g = Lattice(D3Q19, nx, ny, nz, 1.0, 1.0, 1e-4, 0.0, 1, rho0_a=1.0, rho0_b=0.55, direct_host=direct)
    g.init(ra, rb)
    fa, fb, u, cons = g.moments()
    assert np.max(np.abs(fa - ra)) <= 1e-6 and np.max(np.abs(fb - rb)) <= 1e-6
    assert np.all(u == 0.0)
    assert cons[0] == pytest.approx(ra.sum(), rel=1e-6) and cons[1] == pytest.approx(rb.sum(), rel=1e-6)
    # a few noisy steps; then the other route into buffers that start 8 bytes
    # past an allocation (not page-aligned)
    g.step(3)
    a = g.moments()
    g.set_option("direct_host", 1 - direct)
    n = nx * ny * nz
    big = np.zeros(5 * n + 3)
    out = [big[1:1 + n], big[2 + n:2 + 2 * n], big[3 + 2 * n:3 + 5 * n], np.empty(5)]
    F.check(g._h, F.lib().flbm_moments(g._h, *[o.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for o in out]))
    assert np.array_equal(out[0], a[0].ravel()) and np.array_equal(out[1], a[1].ravel())
    assert np.array_equal(out[2], a[2].ravel()) and np.array_equal(out[3], a[3])


@pytest.mark.parametrize("direct", [0, 1])
def test_init_reads_the_densities_and_rejects_bad_ones(direct):
    """flbm_init through either route (kernels reading the caller's arrays
    directly, or host threads through the staging buffer) gives the same rest
    state; a density that is not positive and finite is refused with the
    first bad site of its species, leaving the state as it was."""
    shape = (9, 10, 11)
    ra = inputs.perturbed_density(shape, 1.0, 1e-3, 5, 0)
    rb = inputs.perturbed_density(shape, 0.7, 1e-3, 5, 1)
    ref = Lattice(D3Q19, 11, 10, 9, 1.0, 1.0, 1e-4, 0.9, 3, direct_host=1 - direct)
    ref.init(ra, rb)
    g = Lattice(D3Q19, 11, 10, 9, 1.0, 1.0, 1e-4, 0.9, 3, direct_host=direct)
    # the option reads back the route in effect: never direct when 0 was asked
    assert g.get_option("direct_host") in ((0, 1) if direct else (0,))
    g.init(ra, rb)
    assert np.array_equal(g.get_populations(), ref.get_populations())
    g.step(2)
    before = g.get_populations()
    for which, site, value in ((0, 17, -0.5), (0, 40, np.nan), (1, 5, 0.0), (1, 900, np.inf)):
        a, b = ra.copy().ravel(), rb.copy().ravel()
        (a if which == 0 else b)[site] = value
        if site != 5:
            (a if which == 0 else b)[site + 3] = -1.0  # a later bad site is not the one reported
        with pytest.raises(FlbmError) as e:
            g.init(a, b)
        assert e.value.status == F.EINVAL and f"at site {site} " in str(e.value)
        assert g.step_count == 2 and np.array_equal(g.get_populations(), before)
