"""Writes fl1400_works.json: forward and backward Frenkel-Ladd works of the
CPU FP64 oracle for eight replicas of the 1400 K batch (bcc 10^3 with
k = 2.38 eV/A^2 and fcc 8^3 with k = 2.68 eV/A^2, seeds 1-4 of each; the
lattice parameters, potential and schedule of the headline 20-replica
batch: t_eq = 10 ps, t_s = 50 ps, dt = 1 fs, damping 0.1 ps, lambda
function 2, Sec. III.A-B).  Replica indices are the ones the 20-replica
batch gives them (bcc seeds 1-10 first, then fcc seeds 1-10), because the
Philox noise is keyed by (seed, replica).

Calls only the oracle.  About half an hour on eight host cores:

    python tests/golden/make_fl1400_works.py

With --all it writes fl1400_all_works.json for all twenty replicas of the
batch (seeds 1-10 of each lattice), taking the eight rows of
fl1400_works.json as they are (the oracle is deterministic) and running the
other twelve: about an hour on eight host cores.
"""
import json
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

T = 1400.0
T_EQ, T_S = 10000, 50000
# (lattice, a, n, k, seed, replica index in the 20-replica batch)
JOBS = [(0, 2.87, 10, 2.38, s, s - 1) for s in (1, 2, 3, 4)] + \
       [(1, 3.65, 8, 2.68, s, 10 + s - 1) for s in (1, 2, 3, 4)]
JOBS_ALL = [(0, 2.87, 10, 2.38, s, s - 1) for s in range(1, 11)] + \
           [(1, 3.65, 8, 2.68, s, 10 + s - 1) for s in range(1, 11)]


def run(job):
    import oracle as O
    from paper_2201_04622_gb300 import workloads as W
    lat, a, n, k, seed, rep = job
    p = O.eam(**W.EAM_FE_LIKE)
    th = O.eam_theta(p)
    x0, box = O.create_crystal(lat, a, n, n, n)
    m = O.md(dt=1e-3, T=T, damp=0.1, mass=W.MASS_FE_AMU * O.amu(), k_spring=k, lambda_fn=2,
             path=O.PATH_FL, t_eq=T_EQ, t_s=T_S, seed=seed, replica=rep, fix_cm=1)
    v = O.init_velocities(m, len(x0))
    out = O.switch_run(p, th, m, x0, v, x0, box)
    return dict(lattice=lat, a=a, n=n, k=k, seed=seed, replica=rep, natoms=len(x0),
                W_f=out["W_f"], W_b=out["W_b"])


def main():
    import oracle as O
    O.build()
    t0 = time.time()
    everything = "--all" in sys.argv
    jobs, done = (JOBS_ALL, []) if everything else (JOBS, [])
    if everything:
        with open(os.path.join(HERE, "fl1400_works.json")) as f:
            done = json.load(f)["rows"]
        have = {(r["lattice"], r["seed"]) for r in done}
        jobs = [j for j in JOBS_ALL if (j[0], j[4]) not in have]
    with ProcessPoolExecutor(max_workers=min(8, os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        rows = sorted(done + list(ex.map(run, jobs)), key=lambda r: r["replica"])
    doc = {"_source": "CPU FP64 oracle (oracle/), written by tests/golden/make_fl1400_works.py",
           "cite": "Sec. III.A-B: Frenkel-Ladd switching, forward and backward works (eq. fl)",
           "T": T, "t_eq": T_EQ, "t_s": T_S, "dt_ps": 1e-3, "damping_ps": 0.1, "lambda_fn": 2,
           "batch": "10 x bcc 10^3 (a 2.87, k 2.38, seeds 1-10) then 10 x fcc 8^3 (a 3.65, k 2.68, seeds 1-10)",
           "rows": rows}
    with open(os.path.join(HERE, "fl1400_all_works.json" if everything else "fl1400_works.json"), "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote %d rows in %.0f s" % (len(rows), time.time() - t0))


if __name__ == "__main__":
    main()
