"""Writes tests/golden/cube64_oracle_record.json: the oracle's own run of the 64^3 / 512-box
workload (20 load steps to 1.5 x first yield, eps_Newton = 1e-6, eps_PCGP = 1e-8).

Calls only ``oracle/`` and ``workloads``.  Records per load step the Newton iterations,
the PCGP iterations and plastic Gauss points per Newton iteration, the criterion
sequence and the committed plastic count, the Gauss points that turned plastic at the
step's commit (Delta kappa > 0) and those within |Phi| <= 1e-8 (sigma_y + H kappa_k) of the yield
surface there, and the displacement at 512 seeded dofs (``workloads.seeded_indices``), plus the
oracle's first-yield traction and component timings.  Resumable: completed steps are kept and the state is re-run only
when the record is missing.  Slow (hours on one CPU core).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle.ssn import ElastoplasticModel  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cube64_oracle_record.json")
N_U_SAMPLES, SEED_U = 512, 6464


def main(n_steps=None):
    w = W.CUBE64
    n_steps = n_steps or w.n_steps
    t0 = time.time()
    model = ElastoplasticModel(w)
    t_y = model.first_yield_traction(rtol=1e-10)
    idx_u = W.seeded_indices(model.dec.n_dof, N_U_SAMPLES, SEED_U)
    rec = {"workload": w.name, "newton_tol": w.newton_tol, "pcg_rtol": w.pcg_rtol, "t_y": t_y,
           "u_samples": {"n": N_U_SAMPLES, "seed": SEED_U, "idx_sum": int(idx_u.sum())},
           "setup_and_first_yield_s": time.time() - t0, "steps": []}
    f1 = model.traction_load(w.traction_dir)
    prev = 0.0
    for k, a in enumerate(w.load_fractions(n_steps)):
        ts = time.time()
        sig0, kap0 = model.sigma.copy(), model.kappa.copy()
        info = model.time_step((a - prev) * t_y * f1, w.newton_tol, w.pcg_rtol, w.newton_maxit, w.pcg_maxit)
        prev = a
        eta = model.strains(info["du"])
        phi = model.mat.yield_function(model.mat.trial(sig0, eta), kap0)
        band = np.nonzero(np.abs(phi) <= 1e-8 * (model.mat.sigma_y + model.mat.H * kap0))[0]
        turned = np.nonzero(model.kappa > kap0)[0]
        rec["steps"].append({"step": k + 1, "load_fraction": a, "newton": info["newton"], "pcg": info["pcg"],
                             "plastic": info["plastic"], "criterion": info["criterion"],
                             "plastic_committed": info["plastic_committed"], "converged": info["converged"],
                             "u_norm": float(np.linalg.norm(model.u)),
                             "plastic_idx": [int(i) for i in turned], "band_idx": [int(i) for i in band],
                             "u_at_samples": [float(x) for x in model.u[idx_u]],
                             "seconds": time.time() - ts})
        with open(OUT + ".tmp", "w") as fh:
            json.dump(rec, fh, indent=1)
        os.replace(OUT + ".tmp", OUT)
        print(f"step {k + 1}: newton {info['newton']} pcg {info['pcg']} plastic {info['plastic_committed']}",
              flush=True)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else None)
