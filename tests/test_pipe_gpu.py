"""The pipelined two-array step (the fused schedule with two-array
streaming): one persistent launch per step in which densities, moments and
collisions of the slices are ordered through a ring of slice slots in L2.
It runs the per-site arithmetic of the two-kernel step, so both must agree
bit for bit; it must also report a dependency wait that runs out, and the
oracle must agree with it on its own (through the two-kernel equality and the
direct comparison below)."""
import numpy as np
import pytest

import oracle
from paper_1410_5584_gb300 import D2Q9, D3Q19, FlbmError, Lattice
from paper_1410_5584_gb300 import flbm as F
from paper_1410_5584_gb300 import inputs

pytestmark = pytest.mark.gpu


def _state(lat, shape, rho=(1.0, 0.8), eps=0.02, seed=3):
    c, w, T, N = oracle.tables(lat)
    return inputs.random_populations(np.stack([w * rho[0], w * rho[1]]), shape, eps, seed=seed)


def _run(lat, shape, tau, sched, f0, nsteps, storage="f32", lag=0, timing=False):
    nz, ny, nx = shape
    g = Lattice(lat, nx, ny, nz, tau[0], tau[1], 1e-4, 0.9, 11, storage=storage, rho0_a=1.0, rho0_b=0.8)
    g.set_option("schedule", F.SCHEDULE[sched])
    if lag:
        g.set_option("pipe_lag", lag)
    g.set_populations(f0, step=5)
    if timing:
        g.set_option("kernel_timing", 1)
    for k in (1, nsteps - 1):  # split over two calls: both parities of the array pair
        g.step(k)
    out = g.get_populations()
    launches = g.kernel_times()[1] if timing else None
    g.close()
    return out, launches


# boxes with enough slices for a lag of 2 or 3 (S >= 3 lag + 10), ragged x tiles
SHAPES = [(D3Q19, (24, 6, 40)), (D3Q19, (19, 3, 64)), (D2Q9, (1, 40, 70)), (D2Q9, (1, 33, 32))]


@pytest.mark.parametrize("lat,shape", SHAPES)
@pytest.mark.parametrize("tau", [(1.0, 1.0), (0.8, 1.0)])
@pytest.mark.parametrize("lag", [2, 3])
def test_pipeline_is_bitwise_the_two_kernel_step(lat, shape, tau, lag):
    """Full relaxation (the moment-fed collide, moments through the ring) and
    unequal rates (the population-reading collide): identical populations
    after 4 steps, and the pipelined kernel really ran (one launch a step, no
    density launch)."""
    if 3 * lag + 10 > (shape[0] if lat == D3Q19 else shape[1]):
        pytest.skip("too few slices for this lag")
    f0 = _state(lat, shape)
    a, launches = _run(lat, shape, tau, "fused", f0, 4, lag=lag, timing=True)
    b, _ = _run(lat, shape, tau, "two_kernels", f0, 4)
    assert launches == {"density": 0, "collide": 4}
    assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_pipeline_sixteen_bit_storage(storage):
    shape = (22, 5, 36)
    f0 = _state(D3Q19, shape, eps=0.01)
    a, _ = _run(D3Q19, shape, (1.0, 1.0), "fused", f0, 3, storage=storage, lag=2)
    b, _ = _run(D3Q19, shape, (1.0, 1.0), "two_kernels", f0, 3, storage=storage)
    assert np.array_equal(a, b)


def test_pipeline_matches_oracle():
    """One pipelined step against the FP64 oracle directly (1e-6 relative)."""
    shape = (20, 4, 33)
    nz, ny, nx = shape
    f0 = _state(D3Q19, shape)
    g = Lattice(D3Q19, nx, ny, nz, 1.0, 1.0, 1e-4, 0.9, 11, rho0_a=1.0, rho0_b=0.8)
    g.set_option("schedule", F.SCHEDULE["fused"])
    g.set_option("pipe_lag", 2)
    g.set_populations(f0, step=5)
    g.step(2)
    o = oracle.Oracle(D3Q19, nx, ny, nz, 1.0, 1.0, 1e-4, 0.9, 11)
    o.set_f(f0, step=5)
    o.step(2)
    fo = o.get_f()
    assert np.max(np.abs(g.get_populations() - fo)) <= 2e-6 * np.max(np.abs(fo))


@pytest.mark.parametrize("tau", [(1.0, 1.0), (0.8, 1.0)])
def test_default_geometry_is_bitwise_the_two_kernel_step(tau):
    """The automatic lag and ring on a box whose slices hold 5 MB of
    populations (256 x 128 sites): the lag is cut by the L2 budget below two
    waves; the pipelined kernel runs (one launch a step) and gives the
    two-kernel step's bits."""
    shape = (40, 128, 256)
    f0 = _state(D3Q19, shape, eps=0.01)
    a, launches = _run(D3Q19, shape, tau, "fused", f0, 3, timing=True)
    b, _ = _run(D3Q19, shape, tau, "two_kernels", f0, 3)
    assert launches == {"density": 0, "collide": 3}
    assert np.array_equal(a, b)


def test_small_boxes_fall_back_to_two_kernels():
    """A box with too few slices for the pipeline runs the two-kernel step."""
    shape = (6, 5, 40)
    f0 = _state(D3Q19, shape)
    a, launches = _run(D3Q19, shape, (1.0, 1.0), "fused", f0, 3, timing=True)
    b, _ = _run(D3Q19, shape, (1.0, 1.0), "two_kernels", f0, 3)
    assert launches["density"] == 3
    assert np.array_equal(a, b)


def test_full_size_pipeline_is_bitwise_the_two_kernel_step():
    """The benchmark box, D3Q19 256^3 at tau = 1, automatic lag: three steps
    from the same state, compared on the device."""
    import torch

    out = []
    for sched in ("fused", "two_kernels"):
        g = Lattice(D3Q19, 256, 256, 256, 1.0, 1.0, 1e-5, 0.9, 1)
        g.set_option("schedule", F.SCHEDULE[sched])
        g.init(inputs.perturbed_density((256, 256, 256), 1.0, 1e-3, 1, 0),
               inputs.perturbed_density((256, 256, 256), 1.0, 1e-3, 1, 1))
        g.step(3)
        g.sync()
        out.append(g.pop_buffer)
    assert torch.equal(out[0], out[1])


def test_pipeline_wait_timeout_is_reported():
    """Failure detection without a GPU fault: the test hook makes every
    dependency wait of the pipelined step wait for work that never comes; the
    waits give up after the limit, the kernel returns, the host reads
    FLBM_ETIMEOUT, and re-initialising gives a usable context again."""
    g = Lattice(D3Q19, 32, 4, 22, 1.0, 1.0, 1e-4, 0.5, 1)
    g.set_option("schedule", F.SCHEDULE["fused"])
    g.set_option("pipe_lag", 2)
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
    assert g.moments(fields=False)[0] == pytest.approx(32 * 4 * 22, rel=1e-6)
