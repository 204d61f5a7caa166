"""Writes profiles/precision_vs_oracle.json: the errors of the FP32, FP16 and
BF16 storage forms against the FP64 oracle on a D3Q19 32^3 sub-case of the
benchmark mixture (G rho0 = 0.9, tau = 1, kT = 1e-5, rho = 1 + 1e-3 g), run
for 200 steps on both sides from the same densities with the same noise, the
axis structure factors sampled every 10 steps along that shared history.

Reported per form: the largest density error, the largest velocity error
relative to the largest velocity, the largest relative error of
S_AA + S_BB, and each side's relative mass drift.  bench.py reads the record
while the kernel sources match the digest stored in it.

Run on a GPU:  python tests/precision_vs_oracle.py [output path]
(default profiles/precision_vs_oracle.json)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_1410_5584_gb300 import Lattice, inputs  # noqa: E402

N3, STEPS, EVERY, SEED = 32, 200, 10, 1
TAU, KT, G, RHO0 = (1.0, 1.0), 1e-5, 0.9, 1.0


def run_oracle(ra, rb):
    o = oracle.Oracle(oracle.D3Q19, N3, N3, N3, TAU[0], TAU[1], KT, G, SEED)
    o.set_threads(os.cpu_count() or 1)
    o.init(ra, rb)
    c0 = o.moments()[3]
    for _ in range(STEPS // EVERY):
        o.step(EVERY)
        o.sf_sample(0)
    fa, fb, u, c1 = o.moments()
    sk = o.structure_factor()
    return dict(ra=fa, rb=fb, u=u, sk=np.stack(sk[:3]), drift=max(abs(c1[k] - c0[k]) / c0[k] for k in (0, 1)))


def run_gpu(storage, ra, rb):
    g = Lattice(1, N3, N3, N3, TAU[0], TAU[1], KT, G, SEED, storage=storage, rho0_a=RHO0, rho0_b=RHO0)
    g.init(ra, rb)
    c0 = g.moments(fields=False)
    for _ in range(STEPS // EVERY):
        g.step(EVERY)
        g.sf_sample()
    fa, fb, u, c1 = g.moments()
    sk = np.stack(g.structure_factor(0)[:3])
    g.close()
    return dict(ra=fa, rb=fb, u=u, sk=sk, drift=max(abs(c1[k] - c0[k]) / c0[k] for k in (0, 1)))


def main():
    shape = (N3, N3, N3)
    ra = inputs.perturbed_density(shape, RHO0, 1e-3, SEED, 0)
    rb = inputs.perturbed_density(shape, RHO0, 1e-3, SEED, 1)
    ref = run_oracle(ra, rb)
    s_ref = ref["sk"][0] + ref["sk"][2]
    forms = {}
    for st in ("f32", "f16", "bf16"):
        r = run_gpu(st, ra, rb)
        forms[st] = {
            "rho_abs": float(max(np.max(np.abs(r["ra"] - ref["ra"])), np.max(np.abs(r["rb"] - ref["rb"])))),
            "u_rel": float(np.max(np.abs(r["u"] - ref["u"])) / np.max(np.abs(ref["u"]))),
            "sk_rel": float(np.max(np.abs(r["sk"][0] + r["sk"][2] - s_ref) / s_ref)),
            "mass_drift": float(r["drift"]), "mass_drift_oracle": float(ref["drift"])}
    rec = {"case": f"D3Q19 {N3}^3, G rho0 = {G}, tau = {TAU[0]}, kT = {KT}, rho = 1 + 1e-3 g (seed {SEED}), "
                   f"{STEPS} steps, axis S(k) every {EVERY}; GPU against the FP64 oracle from the same densities",
           "sources_sha256": bench.sources_digest(), "forms": forms,
           "command": "python tests/precision_vs_oracle.py"}
    path = sys.argv[1] if len(sys.argv) > 1 else os.path.join(ROOT, "profiles", "precision_vs_oracle.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
