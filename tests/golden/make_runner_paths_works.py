"""Writes runner_paths_works.json: forward and backward works of the CPU FP64
oracle for the two other paths the crystal runner takes, at lengths where a
trajectory has long decorrelated from its start:

- reversible scaling (Sec. III.C, eq. rs): bcc 6^3 (432 atoms, a = 2.87 A) at
  T0 = 300 K, lambda 1 -> 0.25 (300 -> 1200 K), t_eq = 1 ps, t_s = 10 ps,
  seeds 1 and 2;
- Frenkel-Ladd (Sec. III.B) on ideal hcp 6^3 (the orthohexagonal 4-atom cell,
  864 atoms, a = 2.581 A) at 1000 K with k = 3.0 eV/A^2, t_eq = 1 ps,
  t_s = 10 ps, seeds 1 and 2;

dt = 1 fs, damping 0.1 ps, lambda function 2, the centre of mass fixed;
replica index 0 and 1 for the two seeds of each set.

Calls only the oracle.  A few minutes on four host cores:

    python tests/golden/make_runner_paths_works.py
"""
import json
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

T_EQ, T_S = 1000, 10000
# (name, lattice, a, n, T, k, path, lambda_f, seed, replica)
JOBS = [("rs_bcc6", 0, 2.87, 6, 300.0, 5.0, 1, 0.25, s, s - 1) for s in (1, 2)] + \
       [("fl_hcp6", 2, 2.581, 6, 1000.0, 3.0, 0, 0.5, s, s - 1) for s in (1, 2)]


def run(job):
    import oracle as O
    from paper_2201_04622_gb300 import workloads as W
    name, lat, a, n, T, k, path, lam_f, seed, rep = job
    p = O.eam(**W.EAM_FE_LIKE)
    th = O.eam_theta(p)
    x0, box = O.create_crystal(lat, a, n, n, n)
    m = O.md(dt=1e-3, T=T, damp=0.1, mass=W.MASS_FE_AMU * O.amu(), k_spring=k, lambda_fn=2, path=path,
             t_eq=T_EQ, t_s=T_S, lambda_f=lam_f, seed=seed, replica=rep, fix_cm=1)
    v = O.init_velocities(m, len(x0))
    out = O.switch_run(p, th, m, x0, v, x0, box)
    return dict(set=name, lattice=lat, a=a, n=n, T=T, k=k, path=path, lambda_f=lam_f, seed=seed, replica=rep,
                natoms=len(x0), W_f=out["W_f"], W_b=out["W_b"])


def main():
    import oracle as O
    O.build()
    t0 = time.time()
    with ProcessPoolExecutor(max_workers=min(4, os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        rows = list(ex.map(run, JOBS))
    doc = {"_source": "CPU FP64 oracle (oracle/), written by tests/golden/make_runner_paths_works.py",
           "cite": "Sec. III.C (reversible scaling, eq. rs) and Sec. III.B (Frenkel-Ladd, eq. fl) on hcp",
           "t_eq": T_EQ, "t_s": T_S, "dt_ps": 1e-3, "damping_ps": 0.1, "lambda_fn": 2, "rows": rows}
    with open(os.path.join(HERE, "runner_paths_works.json"), "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote %d rows in %.0f s" % (len(rows), time.time() - t0))


if __name__ == "__main__":
    main()
