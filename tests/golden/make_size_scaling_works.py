"""Writes size_scaling_works.json: the two smallest points of the finite-size
study (Sec. IV.A) in the CPU FP64 oracle -- bcc 5^3 (250 atoms) and 6^3 (432
atoms), a = 2.87 A, at 1000 K, dt = 1 fs, damping 0.1 ps, one spring
k = 2.9 eV/A^2 for both, lambda function 2, four seeds each of the
four-phase schedule (500 steps at lambda = 0, 1000 switching forward, 500 at
lambda = 1, 1000 switching back), then eq. fl + eq. cm per size.

Replica r of the batch (sizes in this order, seeds 1-4 within a size) uses
seed s and Philox replica index r, as workflow.size_scaling numbers them.
Calls only the oracle.  Under a minute on eight host cores:

    python tests/golden/make_size_scaling_works.py
"""
import json
import multiprocessing as mp
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

T, A, K = 1000.0, 2.87, 2.9
SIZES = [5, 6]
SEEDS = [1, 2, 3, 4]
T_EQ, T_S = 500, 1000


def run(job):
    import oracle as O
    from paper_2201_04622_gb300 import workloads as W
    n, seed, rid = job
    p = O.eam(**W.EAM_FE_LIKE)
    x0, box = O.create_crystal(O.BCC, A, n, n, n)
    m = O.md(dt=1e-3, T=T, damp=0.1, mass=W.MASS_FE_AMU * O.amu(), k_spring=K, lambda_fn=2, path=O.PATH_FL,
             t_eq=T_EQ, t_s=T_S, seed=seed, replica=rid, fix_cm=1)
    v = O.init_velocities(m, len(x0))
    out = O.switch_run(p, O.eam_theta(p), m, x0, v, x0, box)
    return dict(cells=n, seed=seed, replica=rid, W_f=out["W_f"], W_b=out["W_b"])


def main():
    import oracle as O
    from paper_2201_04622_gb300 import workloads as W
    O.build()
    t0 = time.time()
    jobs = [(n, s, q * len(SEEDS) + i) for q, n in enumerate(SIZES) for i, s in enumerate(SEEDS)]
    with ProcessPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        rows = list(ex.map(run, jobs))
    sizes = []
    for n in SIZES:
        x0, box = O.create_crystal(O.BCC, A, n, n, n)
        rs = [r for r in rows if r["cells"] == n]
        F, se, ed = O.free_energy(len(x0), float(box[0] * box[1] * box[2]), T, W.MASS_FE_AMU * O.amu(), K,
                                  [r["W_f"] for r in rs], [r["W_b"] for r in rs])
        sizes.append(dict(cells=n, natoms=len(x0), F_per_atom=F, stderr_per_atom=se, Ediss_per_atom=ed))
    doc = {"_source": "CPU FP64 oracle (oracle/), written by tests/golden/make_size_scaling_works.py",
           "cite": "Sec. IV.A (free energy against system size), eq. fl + eq. cm",
           "lattice": "bcc", "a": A, "T": T, "k": K, "dt_ps": 1e-3, "damping_ps": 0.1, "lambda_fn": 2,
           "t_eq": T_EQ, "t_s": T_S, "seeds": SEEDS, "rows": rows, "sizes": sizes}
    with open(os.path.join(HERE, "size_scaling_works.json"), "w") as f:
        json.dump(doc, f, indent=1)
    print(" ".join("n=%d F=%.7f+-%.7f" % (s["cells"], s["F_per_atom"], s["stderr_per_atom"]) for s in sizes),
          "in %.0f s" % (time.time() - t0))


if __name__ == "__main__":
    main()
