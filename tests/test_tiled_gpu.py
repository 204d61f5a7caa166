"""The tiled two-array step of D2Q9 boxes (FLBM_SCHEDULE_TILED): one launch a
step in which each thread block forms the densities of its tile (32 x 16 sites,
or 32 x 4 on boxes of at most 512 such tiles) and of the one-site ring around
it in shared memory, then collides the tile.  It runs
the per-site arithmetic of the two-kernel step, so the two must agree bit for
bit on every box shape (tiles cut by the box edges, boxes smaller than a tile
whose ring wraps more than once), rate set, storage format and option; the
oracle must agree with it directly too.  The batch form (every replica's tiles
in one launch) must agree bit for bit with the batch's two-kernel step."""
import numpy as np
import pytest

import oracle
from paper_1410_5584_gb300 import D2Q9, D3Q19, Batch, Lattice
from paper_1410_5584_gb300 import flbm as F
from paper_1410_5584_gb300 import inputs

pytestmark = pytest.mark.gpu

RHO = (1.0, 0.8)


def _state(lat, shape, eps=0.02, seed=3):
    c, w, T, N = oracle.tables(lat)
    return inputs.random_populations(np.stack([w * RHO[0], w * RHO[1]]), shape, eps, seed=seed)


def _run(lat, shape, tau, sched, f0, nsteps, storage="f32", graph_steps=0, timing=False, **opts):
    nz, ny, nx = shape
    ctor = {k: opts.pop(k) for k in ("streaming",) if k in opts}  # fixed before the buffers exist
    g = Lattice(lat, nx, ny, nz, tau[0], tau[1], 1e-4, 0.9, 11, storage=storage, rho0_a=RHO[0], rho0_b=RHO[1],
                **ctor)
    g.set_option("schedule", F.SCHEDULE[sched])
    g.set_option("graph_steps", graph_steps)
    for k, v in opts.items():
        g.set_option(k, v)
    g.set_populations(f0, step=5)
    if timing:
        g.set_option("kernel_timing", 1)
    for k in (1, nsteps - 1):  # two calls: both arrays of the pair as the source
        g.step(k)
    out = g.get_populations()
    launches = g.kernel_times()[1] if timing else None
    g.close()
    return out, launches


# whole tiles; tiles cut along x and y; boxes smaller than one tile
SHAPES = [(1, 64, 96), (1, 50, 70), (1, 33, 7), (1, 5, 3), (1, 2, 40)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("tau", [(1.0, 1.0), (0.8, 1.0)])
def test_tiled_step_is_bitwise_the_two_kernel_step(shape, tau):
    """Full relaxation (moments kept in shared memory) and unequal rates (the
    population-reading collide): identical populations after 5 steps, and the
    tiled kernel really ran (one launch a step, no density launch)."""
    f0 = _state(D2Q9, shape)
    a, launches = _run(D2Q9, shape, tau, "tiled", f0, 5, timing=True)
    b, _ = _run(D2Q9, shape, tau, "two_kernels", f0, 5)
    assert launches == {"density": 0, "collide": 5}
    assert np.array_equal(a, b)


@pytest.mark.parametrize("tau", [(1.0, 1.0), (0.8, 1.0)])
def test_tiled_step_on_a_box_of_many_tiles(tau):
    """Boxes of more than 512 tiles of 32 x 16 take the 32 x 16 tiles (four
    rows a thread), smaller ones 32 x 4 tiles (one row a thread): a ragged box
    of the first kind, bitwise the two-kernel step and one launch a step."""
    shape = (1, 601, 1030)
    f0 = _state(D2Q9, shape, eps=0.01)
    a, launches = _run(D2Q9, shape, tau, "tiled", f0, 3, timing=True)
    b, _ = _run(D2Q9, shape, tau, "two_kernels", f0, 3)
    assert launches == {"density": 0, "collide": 3}
    assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_tiled_step_sixteen_bit_storage(storage):
    f0 = _state(D2Q9, (1, 50, 70), eps=0.01)
    a, _ = _run(D2Q9, (1, 50, 70), (1.0, 1.0), "tiled", f0, 4, storage=storage)
    b, _ = _run(D2Q9, (1, 50, 70), (1.0, 1.0), "two_kernels", f0, 4, storage=storage)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("opts", [dict(ghost_noise=1), dict(force_velocity=1, noise_rho=1), dict(sdf=0)])
def test_tiled_step_options(opts):
    """The population-space noise reads the ring's densities at the
    destinations; the other options change only per-site arithmetic."""
    f0 = _state(D2Q9, (1, 40, 45))
    a, _ = _run(D2Q9, (1, 40, 45), (1.0, 1.0), "tiled", f0, 3, **opts)
    b, _ = _run(D2Q9, (1, 40, 45), (1.0, 1.0), "two_kernels", f0, 3, **opts)
    assert np.array_equal(a, b)


def test_tiled_step_in_graphs():
    """CUDA graphs of 4 tiled steps (the counter read on the device) give the
    directly launched steps: 11 steps = 1 direct + 2 graphs + 2 direct."""
    f0 = _state(D2Q9, (1, 64, 64))
    a, _ = _run(D2Q9, (1, 64, 64), (1.0, 1.0), "tiled", f0, 11, graph_steps=4)
    b, _ = _run(D2Q9, (1, 64, 64), (1.0, 1.0), "two_kernels", f0, 11)
    assert np.array_equal(a, b)


def test_tiled_schedule_falls_back_where_it_does_not_apply():
    """D3Q19 and in-place streaming run the two-kernel step under the tiled
    schedule (density and collide launches), with its results."""
    f0 = _state(D3Q19, (6, 5, 7))
    a, launches = _run(D3Q19, (6, 5, 7), (1.0, 1.0), "tiled", f0, 3, timing=True)
    b, _ = _run(D3Q19, (6, 5, 7), (1.0, 1.0), "two_kernels", f0, 3)
    assert launches == {"density": 3, "collide": 3}
    assert np.array_equal(a, b)
    f0 = _state(D2Q9, (1, 20, 24))
    a, launches = _run(D2Q9, (1, 20, 24), (1.0, 1.0), "tiled", f0, 3, timing=True, streaming=0)
    b, _ = _run(D2Q9, (1, 20, 24), (1.0, 1.0), "two_kernels", f0, 3, streaming=0)
    assert launches == {"density": 3, "collide": 3}
    assert np.array_equal(a, b)


def test_tiled_step_matches_oracle():
    shape = (1, 37, 45)
    f0 = _state(D2Q9, shape, seed=8)
    a, _ = _run(D2Q9, shape, (0.8, 1.0), "tiled", f0, 3)
    o = oracle.Oracle(D2Q9, shape[2], shape[1], 1, 0.8, 1.0, 1e-4, 0.9, 11)
    o.set_f(f0, step=5)
    o.step(3)
    fo = o.get_f()
    assert np.max(np.abs(a - fo)) <= 3e-6 * np.max(np.abs(fo))


def _batch_reps():
    shapes = [(64, 64), (37, 23), (8, 130), (129, 5), (2, 2), (96, 32)]
    return [dict(nx=nx, ny=ny, tau_a=1.0 if k % 2 == 0 else 0.8, tau_b=1.0, kT=10.0 ** (-4 - 0.3 * k), G=0.15 * k,
                 seed=500 + 13 * k, rho0_a=1.0, rho0_b=0.9) for k, (nx, ny) in enumerate(shapes)]


def _batch_states(reps, seed=2):
    c, w, T, N = oracle.tables(D2Q9)
    return np.concatenate([inputs.random_populations(np.stack([w * r["rho0_a"], w * r["rho0_b"]]),
                                                     (1, r["ny"], r["nx"]), 0.02, seed + k).ravel()
                           for k, r in enumerate(reps)])


@pytest.mark.parametrize("full", [True, False])
@pytest.mark.parametrize("graph_steps", [0, 4])
def test_batch_tiled_step_is_bitwise_the_batch_two_kernel_step(full, graph_steps):
    """Every replica's tiles in one launch a step (uneven, ragged and tiny
    boxes), against the batch's own two-kernel step with two arrays and with
    one array updated in place: bit for bit, 9 steps over graph boundaries."""
    reps = _batch_reps()
    if full:
        reps = [dict(r, tau_a=1.0) for r in reps]
    flat = _batch_states(reps)
    out = {}
    for name, opts in (("tiled", dict(schedule=3)), ("two", dict(schedule=1)), ("in_place", dict(streaming=0))):
        b = Batch(D2Q9, reps, graph_steps=graph_steps, **opts)
        b.set_populations(flat, step=3)
        b.step(2)
        b.step(7)
        out[name] = b.get_populations()
        b.close()
    assert np.array_equal(out["tiled"], out["two"])
    assert np.array_equal(out["two"], out["in_place"])


def test_batch_two_array_checkpoint_and_restore():
    """A two-array batch saves its current array (natural layout) after an odd
    number of steps, continues bit for bit after a restore into a fresh batch,
    and refuses an in-place image saved in the swapped layout."""
    reps = _batch_reps()
    b = Batch(D2Q9, reps, schedule=3, graph_steps=4)
    b.init()
    b.step(7)
    img = b.checkpoint()
    b.step(6)
    a = b.get_populations()
    b2 = Batch(D2Q9, reps, schedule=3)
    b2.restore(img)
    assert b2.step_count == 7
    b2.step(6)
    assert np.array_equal(a, b2.get_populations())
    c = Batch(D2Q9, reps, streaming=0)
    c.init()
    c.step(1)
    swapped = c.checkpoint()
    with pytest.raises(F.FlbmError) as e:
        Batch(D2Q9, reps).restore(swapped)
    assert e.value.status == F.EINVAL


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_batch_tiled_step_sixteen_bit_storage(storage):
    """The tiled batch step on 16-bit deviations is the batch's two-kernel
    step bit for bit."""
    reps = [dict(r, tau_a=1.0) for r in _batch_reps()]
    flat = _batch_states(reps)
    out = []
    for sched in (3, 1):
        b = Batch(D2Q9, reps, storage=storage, schedule=sched, graph_steps=4)
        b.set_populations(flat, step=1)
        b.step(7)
        out.append(b.get_populations())
        b.close()
    assert np.array_equal(out[0], out[1])


def test_batch_views_follow_the_current_array():
    """With two arrays a replica view reads whichever array holds the current
    state: after odd and even step counts its populations and moments are
    the batch's slice, and a lone context stepped alike agrees."""
    reps = _batch_reps()
    flat = _batch_states(reps, seed=7)
    b = Batch(D2Q9, reps, schedule=3)
    b.set_populations(flat, step=0)
    sizes = [r["nx"] * r["ny"] for r in reps]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    for n in (3, 4):
        b.step(n)
        f = b.get_populations()
        ra, rb, u, cons = b.moments()
        for k, r in enumerate(reps):
            v = b.replicas[k]
            fv = v.get_populations()
            assert np.array_equal(fv.ravel(), f[2 * 9 * offs[k]:2 * 9 * offs[k + 1]])
            va, vb, vu, _ = v.moments()
            assert np.array_equal(va.ravel(), ra[offs[k]:offs[k + 1]])
            assert np.array_equal(vb.ravel(), rb[offs[k]:offs[k + 1]])
    k = 3
    r = reps[k]
    g = Lattice(D2Q9, r["nx"], r["ny"], 1, r["tau_a"], r["tau_b"], r["kT"], r["G"], r["seed"], rho0_a=r["rho0_a"],
                rho0_b=r["rho0_b"])
    g.set_populations(flat[2 * 9 * offs[k]:2 * 9 * offs[k + 1]].reshape(2, 9, 1, r["ny"], r["nx"]), step=0)
    g.step(7)
    assert np.max(np.abs(g.get_populations() - b.replicas[k].get_populations())) <= 2e-6
