"""Writes tests/golden/cube64_oracle_record.json: the oracle's own run of the 64^3 / 512-box
workload (20 load steps to 1.5 x first yield, eps_Newton = 1e-6, eps_PCGP = 1e-8).

Calls only ``oracle/`` and ``workloads``.  Records per load step the Newton iterations,
the PCGP iterations and plastic Gauss points per Newton iteration, the criterion
sequence and the committed plastic count, plus the oracle's first-yield traction and
component timings.  Resumable: completed steps are kept and the state is re-run only
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


def main(n_steps=None):
    w = W.CUBE64
    n_steps = n_steps or w.n_steps
    t0 = time.time()
    model = ElastoplasticModel(w)
    t_y = model.first_yield_traction(rtol=1e-10)
    rec = {"workload": w.name, "newton_tol": w.newton_tol, "pcg_rtol": w.pcg_rtol, "t_y": t_y,
           "setup_and_first_yield_s": time.time() - t0, "steps": []}
    f1 = model.traction_load(w.traction_dir)
    prev = 0.0
    for k, a in enumerate(w.load_fractions(n_steps)):
        ts = time.time()
        info = model.time_step((a - prev) * t_y * f1, w.newton_tol, w.pcg_rtol, w.newton_maxit, w.pcg_maxit)
        prev = a
        rec["steps"].append({"step": k + 1, "load_fraction": a, "newton": info["newton"], "pcg": info["pcg"],
                             "plastic": info["plastic"], "criterion": info["criterion"],
                             "plastic_committed": info["plastic_committed"], "converged": info["converged"],
                             "u_norm": float(np.linalg.norm(model.u)), "seconds": time.time() - ts})
        with open(OUT + ".tmp", "w") as fh:
            json.dump(rec, fh, indent=1)
        os.replace(OUT + ".tmp", OUT)
        print(f"step {k + 1}: newton {info['newton']} pcg {info['pcg']} plastic {info['plastic_committed']}",
              flush=True)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else None)
