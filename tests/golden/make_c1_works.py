"""Writes c1_works.json: the small Frenkel-Ladd case at full length in the CPU
FP64 oracle -- bcc 4x4x4 (128 atoms, a = 2.87 A) at 100 K, dt = 1 fs, damping
0.1 ps, lambda function 2 (Sec. III.A-B):

  1. the spring constant from eq. msd (seed 1, replica 0: 2000 steps to
     equilibrate, then 2000 samples every 5 steps at lambda = 0);
  2. ten seeds (seed s, replica s - 1) of the four-phase schedule with that
     spring: 2000 steps at lambda = 0, 5000 switching forward, 2000 at
     lambda = 1, 5000 switching back;
  3. eq. fl + eq. cm over the ten seeds.

Calls only the oracle.  About a minute on eight host cores:

    python tests/golden/make_c1_works.py
"""
import json
import multiprocessing as mp
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

T = 100.0
A, NCELL = 2.87, 4
T_EQ, T_S = 2000, 5000
FIT = dict(n_eq=2000, n_samples=2000, stride=5, seed=1, replica=0)
SEEDS = list(range(1, 11))


def _setup():
    import oracle as O
    from paper_2201_04622_gb300 import workloads as W
    p = O.eam(**W.EAM_FE_LIKE)
    x0, box = O.create_crystal(O.BCC, A, NCELL, NCELL, NCELL)
    return O, W, p, O.eam_theta(p), x0, box


def fit():
    O, W, p, th, x0, box = _setup()
    m = O.md(dt=1e-3, T=T, damp=0.1, mass=W.MASS_FE_AMU * O.amu(), k_spring=1.0, lambda_fn=2,
             path=O.PATH_FL, seed=FIT["seed"], replica=FIT["replica"], fix_cm=1)
    v = O.init_velocities(m, len(x0))
    return O.msd_fit(p, th, m, x0, v, x0, box, FIT["n_eq"], FIT["n_samples"], FIT["stride"])


def run(job):
    seed, k = job
    O, W, p, th, x0, box = _setup()
    m = O.md(dt=1e-3, T=T, damp=0.1, mass=W.MASS_FE_AMU * O.amu(), k_spring=k, lambda_fn=2,
             path=O.PATH_FL, t_eq=T_EQ, t_s=T_S, seed=seed, replica=seed - 1, fix_cm=1)
    v = O.init_velocities(m, len(x0))
    out = O.switch_run(p, th, m, x0, v, x0, box)
    return dict(seed=seed, replica=seed - 1, W_f=out["W_f"], W_b=out["W_b"])


def main():
    import oracle as O
    O.build()
    t0 = time.time()
    msd, k = fit()
    with ProcessPoolExecutor(max_workers=min(10, os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        rows = list(ex.map(run, [(s, k) for s in SEEDS]))
    _, W, _, _, x0, box = _setup()
    n, V = len(x0), float(box[0] * box[1] * box[2])
    F, se, ed = O.free_energy(n, V, T, W.MASS_FE_AMU * O.amu(), k, [r["W_f"] for r in rows],
                              [r["W_b"] for r in rows])
    doc = {"_source": "CPU FP64 oracle (oracle/), written by tests/golden/make_c1_works.py",
           "cite": "Sec. III.A (eq. msd) and Sec. III.B (Frenkel-Ladd switching, eq. fl + eq. cm)",
           "lattice": "bcc", "a": A, "cells": NCELL, "natoms": n, "T": T, "dt_ps": 1e-3,
           "damping_ps": 0.1, "lambda_fn": 2, "t_eq": T_EQ, "t_s": T_S, "fit": FIT,
           "msd": msd, "k": k, "rows": rows, "F_per_atom": F, "stderr_per_atom": se,
           "Ediss_per_atom": ed}
    with open(os.path.join(HERE, "c1_works.json"), "w") as f:
        json.dump(doc, f, indent=1)
    print("k = %.6f eV/A^2, F = %.7f +- %.7f eV/atom; %d seeds in %.0f s"
          % (k, F, se, len(rows), time.time() - t0))


if __name__ == "__main__":
    main()
