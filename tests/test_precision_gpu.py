"""Accuracy of the 16-bit population storage (populations kept as half or
bfloat16 deviations from w_i rho0, collided in float) against the FP64 oracle
and the float-storage run, on a 32^3 D3Q19 Shan-Chen case: densities,
velocities, the axis structure factors sampled along the same noise history,
and mass drift.  Writes the measured errors to precision.json in the folder
named by the FLBM_REPORT_DIR environment variable, when it is set."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1410_5584_gb300 import D3Q19, Lattice
from paper_1410_5584_gb300 import inputs

pytestmark = pytest.mark.gpu

N3, STEPS, EVERY = 32, 200, 10
TAU, KT, G, SEED = 1.0, 1e-5, 0.9, 11


def _run_gpu(storage, f0):
    g = Lattice(D3Q19, N3, N3, N3, TAU, TAU, KT, G, SEED, storage=storage)
    g.set_populations(f0)
    c0 = g.moments(fields=False)
    for _ in range(STEPS // EVERY):
        g.step(EVERY)
        g.sf_sample()
    ra, rb, u, c1 = g.moments()
    return dict(ra=ra, rb=rb, u=u, c0=c0, c1=c1, sk=np.stack(g.structure_factor(0)[:4]))


def _run_oracle(f0):
    o = oracle.Oracle(oracle.D3Q19, N3, N3, N3, TAU, TAU, KT, G, SEED)
    o.set_threads(min(16, os.cpu_count() or 1))
    o.set_f(f0)
    c0 = o.moments()[3]
    for _ in range(STEPS // EVERY):
        o.step(EVERY)
        o.sf_sample(0)
    ra, rb, u, c1 = o.moments()
    return dict(ra=ra, rb=rb, u=u, c0=c0, c1=c1, sk=np.stack(o.structure_factor()[:4]))


def _errors(run, ref):
    rho_err = max(np.max(np.abs(run["ra"] - ref["ra"])), np.max(np.abs(run["rb"] - ref["rb"])))
    u_err = np.max(np.abs(run["u"] - ref["u"])) / np.max(np.abs(ref["u"]))
    s_ref = ref["sk"][0] + ref["sk"][2]
    sk_err = np.max(np.abs((run["sk"][0] + run["sk"][2]) - s_ref) / s_ref)
    mass = max(abs(run["c1"][k] - run["c0"][k]) / run["c0"][k] for k in (0, 1))
    return dict(rho_abs=float(rho_err), u_rel=float(u_err), sk_rel=float(sk_err), mass_drift=float(mass))


def test_sixteen_bit_storage_accuracy_report():
    c, w, T, N = oracle.tables(oracle.D3Q19)
    shape = (N3, N3, N3)
    ra0 = inputs.perturbed_density(shape, 1.0, 1e-3, SEED, 0)
    rb0 = inputs.perturbed_density(shape, 1.0, 1e-3, SEED, 1)
    f0 = np.stack([w[:, None, None, None] * ra0[None], w[:, None, None, None] * rb0[None]])
    f0 = f0.astype(np.float32).astype(np.float64)
    ref = _run_oracle(f0)
    runs = {s: _run_gpu(s, f0) for s in ("f32", "f16", "bf16")}
    report = {s: {"vs_oracle": _errors(runs[s], ref), "vs_f32": _errors(runs[s], runs["f32"])} for s in runs}
    report["case"] = f"D3Q19 {N3}^3, tau={TAU}, kT={KT}, G={G}, {STEPS} steps, S(k) every {EVERY}"
    if os.environ.get("FLBM_REPORT_DIR"):
        with open(os.path.join(os.environ["FLBM_REPORT_DIR"], "precision.json"), "w") as f:
            json.dump(report, f, indent=1)
    print(json.dumps(report))
    # float storage: parity-level agreement
    assert report["f32"]["vs_oracle"]["rho_abs"] < 1e-5
    assert report["f32"]["vs_oracle"]["mass_drift"] < 1e-6
    # 16-bit storage: the stored deviations (~1e-3 here) carry 11 (half) or 8
    # (bfloat16) significant bits; over 200 steps the rounding errors add up like a
    # random walk, bounding density errors well below 1e-4 (half) and 1e-3
    # (bfloat16); mass is conserved to the rounding of the deviations
    assert report["f16"]["vs_oracle"]["rho_abs"] < 1e-4
    assert report["bf16"]["vs_oracle"]["rho_abs"] < 1e-3
    assert report["f16"]["vs_oracle"]["sk_rel"] < 0.05
    assert report["f16"]["vs_oracle"]["mass_drift"] < 1e-4
    assert report["bf16"]["vs_oracle"]["mass_drift"] < 1e-3
