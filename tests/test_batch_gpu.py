"""The batching form: many independent replicas of uneven size and parameters
in one launch per kernel (CUDA graphs of several steps).  Each replica must be
the same problem as a lone context with its parameters (replica-local site
index, own Philox key)."""
import numpy as np
import pytest

import oracle
from paper_1410_5584_gb300 import D2Q9, D3Q19, Batch, FlbmError, Lattice
from paper_1410_5584_gb300 import flbm as F
from paper_1410_5584_gb300 import inputs

pytestmark = pytest.mark.gpu


def _replicas(lat):
    if lat == D2Q9:
        shapes = [(37, 23, 1), (64, 64, 1), (8, 130, 1), (129, 5, 1), (2, 2, 1)]
    else:
        shapes = [(13, 7, 6), (16, 16, 16), (5, 9, 2)]
    reps = []
    for k, (nx, ny, nz) in enumerate(shapes):
        reps.append(dict(nx=nx, ny=ny, nz=nz, tau_a=0.8 + 0.05 * k, tau_b=1.0 + 0.03 * k, kT=10.0 ** (-4 - 0.3 * k),
                         G=0.15 * k, seed=1000 + 17 * k, rho0_a=1.0, rho0_b=0.9))
    return reps


def _states(lat, reps, seed=4):
    c, w, T, N = oracle.tables(lat)
    out = []
    for k, r in enumerate(reps):
        shape = (r["nz"], r["ny"], r["nx"])
        out.append(inputs.random_populations(np.stack([w * r["rho0_a"], w * r["rho0_b"]]), shape, 0.02, seed + k))
    return out


@pytest.mark.parametrize("lat", [D2Q9, D3Q19])
@pytest.mark.parametrize("graph_steps", [0, 4])
def test_batch_replicas_match_lone_contexts(lat, graph_steps):
    reps = _replicas(lat)
    states = _states(lat, reps)
    b = Batch(lat, reps, graph_steps=graph_steps)
    b.set_populations(np.concatenate([s.ravel() for s in states]), step=5)
    b.step(9)  # two graphs of 4 steps plus one direct step when graph_steps = 4
    assert b.step_count == 14
    for k, r in enumerate(reps):
        g = Lattice(lat, r["nx"], r["ny"], r["nz"], r["tau_a"], r["tau_b"], r["kT"], r["G"], r["seed"],
                    rho0_a=r["rho0_a"], rho0_b=r["rho0_b"])
        g.set_populations(states[k], step=5)
        g.step(9)
        ref = g.get_populations()
        got = b.replicas[k].get_populations()
        assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref)), k


def test_batch_replica_against_oracle():
    reps = _replicas(D2Q9)
    states = _states(D2Q9, reps, seed=9)
    b = Batch(D2Q9, reps)
    b.set_populations(np.concatenate([s.ravel() for s in states]), step=0)
    b.step(3)
    k = 0
    r = reps[k]
    o = oracle.Oracle(D2Q9, r["nx"], r["ny"], 1, r["tau_a"], r["tau_b"], r["kT"], r["G"], r["seed"])
    o.set_f(states[k])
    o.step(3)
    fo = o.get_f()
    assert np.max(np.abs(b.replicas[k].get_populations() - fo)) <= 3e-6 * np.max(fo)


def test_batch_observables_checkpoint_and_views():
    reps = _replicas(D2Q9)
    b = Batch(D2Q9, reps, graph_steps=8)
    b.init()
    c0 = b.moments()[3]
    b.step(20)
    ra, rb, u, c1 = b.moments()
    assert abs(c1[0] - c0[0]) <= 1e-6 * c0[0] and abs(c1[1] - c0[1]) <= 1e-6 * c0[1]
    assert ra.size == sum(r["nx"] * r["ny"] for r in reps)
    # per-replica structure factors through the views
    b.sf_sample()
    s_aa = b.replicas[1].structure_factor(0)[0]
    assert s_aa.size == 32 and np.all(s_aa > 0)
    # checkpoint / restore continues bit for bit
    img = b.checkpoint()
    b.step(13)
    a = b.get_populations()
    b2 = Batch(D2Q9, reps)
    b2.restore(img)
    assert b2.step_count == 20
    b2.step(13)
    assert np.array_equal(a, b2.get_populations())
    # views observe but do not step alone
    with pytest.raises(FlbmError) as e:
        F.check(b.replicas[0]._h, F.lib().flbm_step(b.replicas[0]._h, 1))
    assert e.value.status == F.ESTATE


@pytest.mark.parametrize("lat", [D2Q9, D3Q19])
def test_full_relaxation_batch_matches_lone_contexts_and_the_general_collide(lat):
    """Replicas with every rate 1 run the batch collide that skips the
    non-conserved projections: each replica agrees with a lone context to
    rounding, and with the batch forced onto the general collide (a test
    hook) to rounding; the replica sizes exercise the exact dividers that
    replace the per-site integer division (rows of 37, 129 and 2 sites)."""
    reps = [dict(r, tau_a=1.0, tau_b=1.0) for r in _replicas(lat)]
    states = _states(lat, reps, seed=6)
    flat = np.concatenate([s.ravel() for s in states])
    runs = []
    for general in (0, 1):
        b = Batch(lat, reps, graph_steps=4, test_general_collide=general)
        b.set_populations(flat, step=2)
        b.step(9)
        runs.append([b.replicas[k].get_populations() for k in range(len(reps))])
        b.close()
    for k, r in enumerate(reps):
        g = Lattice(lat, r["nx"], r["ny"], r["nz"], 1.0, 1.0, r["kT"], r["G"], r["seed"],
                    rho0_a=r["rho0_a"], rho0_b=r["rho0_b"])
        g.set_populations(states[k], step=2)
        g.step(9)
        ref = g.get_populations()
        assert np.max(np.abs(runs[0][k] - ref)) <= 2e-6 * np.max(np.abs(ref)), k
        assert np.max(np.abs(runs[0][k] - runs[1][k])) <= 2e-6 * np.max(np.abs(ref)), k
