"""Writes config4_prefix_works.json: a stated prefix of the reversible-scaling
workload in the CPU FP64 oracle -- bcc 16x16x16 (8192 atoms, a = 2.87 A),
T0 = 100 K, lambda 1 -> 0.0625 (100 -> 1600 K), t_eq = 10 ps, t_s = 100 ps,
dt = 1 fs, damping 0.1 ps (Sec. III.C) -- for seeds 1 and 2 (replica 0).
The prefix is the first 12,000 steps: the equilibration at lambda = 1 and
the first 2000 steps of the forward switch.  Stored: the work after the
prefix and the cumulative work every 10 switching steps.

The full schedule (220,000 steps of 8192 atoms, about 4 h per seed on one
core) is out of reach of the oracle in a test budget; a multi-kernel run of
the same schedule on the GPU can be compared with this prefix step for step.

Calls only the oracle.  About 15 minutes on two host cores:

    python tests/golden/make_config4_prefix_works.py
"""
import json
import multiprocessing as mp
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

N_CELL, A = 16, 2.87
T0, LAMBDA_F = 100.0, 0.0625
T_EQ, T_S = 10000, 100000
PREFIX = T_EQ + 2000
EVERY = 10
SEEDS = [1, 2]


def run(seed):
    import oracle as O
    from paper_2201_04622_gb300 import workloads as W
    p = O.eam(**W.EAM_FE_LIKE)
    th = O.eam_theta(p)
    x0, box = O.create_crystal(O.BCC, A, N_CELL, N_CELL, N_CELL)
    m = O.md(dt=1e-3, T=T0, damp=0.1, mass=W.MASS_FE_AMU * O.amu(), k_spring=1.0, path=O.PATH_RS,
             lambda_f=LAMBDA_F, t_eq=T_EQ, t_s=T_S, seed=seed, replica=0, fix_cm=1)
    v = O.init_velocities(m, len(x0))
    t0 = time.time()
    out = O.switch_run_prefix(p, th, m, x0, v, x0, box, PREFIX, cumulative=True)
    k_end = PREFIX - T_EQ
    return dict(seed=seed, replica=0, W_f=out["W_f"],
                Wcum_f_every_10=[float(w) for w in out["Wcum_f"][:k_end + 1:EVERY]],
                oracle_seconds=time.time() - t0)


def main():
    import oracle as O
    O.build()
    t0 = time.time()
    with ProcessPoolExecutor(max_workers=len(SEEDS), mp_context=mp.get_context("spawn")) as ex:
        rows = list(ex.map(run, SEEDS))
    doc = {"_source": "CPU FP64 oracle (oracle/), written by tests/golden/make_config4_prefix_works.py",
           "cite": "Sec. III.C: reversible scaling, cumulative work of the forward switch (eq. rs)",
           "lattice": "bcc", "a": A, "cells": N_CELL, "natoms": 2 * N_CELL ** 3, "T0": T0,
           "lambda_f": LAMBDA_F, "t_eq": T_EQ, "t_s": T_S, "dt_ps": 1e-3, "damping_ps": 0.1,
           "prefix_steps": PREFIX, "every": EVERY, "rows": rows}
    with open(os.path.join(HERE, "config4_prefix_works.json"), "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote %d rows in %.0f s" % (len(rows), time.time() - t0))


if __name__ == "__main__":
    main()
