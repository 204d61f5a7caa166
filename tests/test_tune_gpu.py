"""Launch settings and the autotuner: the thread-block shape, the schedule and
the CUDA-graph length change how the same kernels are launched, never the
update, so every setting gives bitwise the same populations, and tuning leaves
the simulation where it was."""
import json

import numpy as np
import pytest

import oracle
from paper_1410_5584_gb300 import D2Q9, D3Q19, Batch, Lattice
from paper_1410_5584_gb300 import inputs

pytestmark = pytest.mark.gpu


def _state(lat, shape, seed=5):
    c, w, T, N = oracle.tables(lat)
    return inputs.random_populations(np.stack([w * 1.0, w * 0.8]), shape, 0.02, seed=seed)


def _run(lat, shape, steps, **options):
    nz, ny, nx = shape
    g = Lattice(lat, nx, ny, nz, 0.8, 1.0, 1e-4, 0.9, 6, **options)
    g.set_populations(_state(lat, shape), step=3)
    g.step(steps)
    return g.get_populations()


@pytest.mark.parametrize("lat,shape", [(D2Q9, (1, 13, 70)), (D2Q9, (1, 2, 33)), (D3Q19, (5, 7, 45)),
                                       (D3Q19, (3, 2, 2))])
def test_block_shapes_are_bitwise_identical(lat, shape):
    """Blocks of 128x1, 64x2, 32x4 and 32x1 sites, on boxes whose rows and
    columns leave ragged blocks, both parities."""
    want = _run(lat, shape, 5)
    for bx, by in ((64, 2), (32, 4), (32, 1)):
        got = _run(lat, shape, 5, block_x=bx, block_y=by)  # x first: x * 1 is always allowed
        assert np.array_equal(got, want), (bx, by)


@pytest.mark.parametrize("lat,shape", [(D2Q9, (1, 48, 64)), (D3Q19, (12, 10, 16))])
def test_autotune_keeps_the_state_and_the_results(lat, shape, tmp_path):
    nz, ny, nx = shape
    f0 = _state(lat, shape, seed=8)
    g = Lattice(lat, nx, ny, nz, 0.8, 1.0, 1e-4, 0.9, 6)
    g.set_populations(f0, step=3)
    g.step(3)
    before = g.get_populations()
    cache = tmp_path / "tune.json"
    chosen = g.autotune(steps=3, cache=str(cache))
    assert g.step_count == 6
    assert np.array_equal(g.get_populations(), before)
    assert chosen["schedule"] in (0, 1, 2, 3) and chosen["block_x"] * chosen["block_y"] <= 128
    g.step(7)
    ref = Lattice(lat, nx, ny, nz, 0.8, 1.0, 1e-4, 0.9, 6)
    ref.set_populations(f0, step=3)
    ref.step(10)
    assert np.array_equal(g.get_populations(), ref.get_populations())
    # the choice is cached per device and problem and applied without timing
    entries = json.loads(cache.read_text())
    assert len(entries) == 1
    (key, rec), = entries.items()
    assert f"{nx}x{ny}x{nz}" in key and rec["ms_per_step"] > 0
    h = Lattice(lat, nx, ny, nz, 1.0, 1.0, 0.0, 0.0, 1)
    h.init()
    assert h.autotune(steps=3, cache=str(cache)) == chosen
    assert h.step_count == 0


def test_batch_autotune_picks_a_graph_length_and_keeps_the_state(tmp_path):
    reps = [dict(nx=40, ny=24, tau_a=1.0, tau_b=0.9, kT=1e-5, G=0.5, seed=3),
            dict(nx=16, ny=64, tau_a=0.8, tau_b=1.0, kT=1e-4, G=0.2, seed=4)]
    b = Batch(D2Q9, reps)
    b.init()
    b.step(5)
    before = b.get_populations()
    chosen = b.autotune(steps=8, cache=str(tmp_path / "tune.json"))
    assert chosen["graph_steps"] in (0, 4, 16, 64) and chosen["schedule"] in (1, 3)
    assert b.step_count == 5
    assert np.array_equal(b.get_populations(), before)
    b.step(9)
    ref = Batch(D2Q9, reps)
    ref.init()
    ref.step(14)
    assert np.array_equal(b.get_populations(), ref.get_populations())
