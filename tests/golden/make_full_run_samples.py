"""Writes full_run_samples.json: oracle states at the end of two whole runs at
full size, sampled, for the GPU full-run parity test.

  * isentropic vortex, 256 x 256 mesh, p = 3, SSP-RK3, 200 steps;
  * perturbed vortex, 256 x 256 mesh, p = 2, SSP-RK3, 400 steps (the forward run
    of the adjoint workload).

Only the oracle computes these values (the runs take a few minutes on one
core).  For each run the file holds 1024 coefficient indices drawn with a seeded
generator, the oracle's values there, the L2 norm of the whole final state and
its conserved totals.  Run from the repository root:

    python tests/golden/make_full_run_samples.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1601_07944_gb300 import inputs as I  # noqa: E402

RUNS = [dict(name="vortex_256_p3_200", n=256, p=3, ic="vortex", steps=200),
        dict(name="perturbed_vortex_256_p2_400", n=256, p=2, ic="perturbed_vortex", steps=400)]
N_SAMPLES = 1024
SEED = 17


def main():
    out = {"generator": "tests/golden/make_full_run_samples.py (oracle only)", "runs": []}
    for r in RUNS:
        mesh = I.periodic_mesh(r["n"])
        f = getattr(I, r["ic"])
        o = oracle.OracleDG.from_mesh(mesh, r["p"])
        c0 = o.project_ic(f)
        dt = I.fixed_dt(mesh, f, r["p"])
        c = o.ssp_rk3(c0, dt, r["steps"])
        flat = c.reshape(-1)
        idx = np.sort(np.random.default_rng(SEED).choice(flat.size, N_SAMPLES, replace=False))
        out["runs"].append(dict(r, dt=dt, shape=list(c.shape), index=idx.tolist(),
                                value=[float(v) for v in flat[idx]],
                                l2_norm=float(np.linalg.norm(flat)),
                                totals=[float(v) for v in o.totals(c)]))
        print(r["name"], "done", flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_run_samples.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
