"""Writes config3_subset_works.json: forward and backward Frenkel-Ladd works of
the CPU FP64 oracle for a stated subset of the 256-replica uneven set
(workloads.batched_replicas(256, seed=1): bcc n^3 x 2 with n in 6..12, fcc
n^3 x 4 with n in 5..10, T uniform in 300..1600 K), at full length: t_eq =
10 ps, t_s = 20 ps, dt = 1 fs, damping 0.1 ps, lambda function 2, springs of
the 1400 K fit by lattice, seed 1 and Philox replica index r (Sec. III.B).

The subset: the 16 replicas with the fewest atoms (ties by index) and 8
drawn from the other 240 by numpy PCG64(3) without replacement.

Calls only the oracle.  About half an hour on eight host cores:

    python tests/golden/make_config3_subset_works.py
"""
import json
import multiprocessing as mp
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

T_EQ, T_S = 10000, 20000


def subset():
    import numpy as np
    from paper_2201_04622_gb300 import workloads as W
    reps = W.batched_replicas(256, seed=1)
    natoms = [(2 if r["lattice"] == W.BCC else 4) * r["n"] ** 3 for r in reps]
    order = sorted(range(len(reps)), key=lambda q: (natoms[q], q))
    small = order[:16]
    rest = order[16:]
    rand = sorted(int(q) for q in np.random.Generator(np.random.PCG64(3)).choice(rest, 8, replace=False))
    return reps, natoms, small, rand


def run(q):
    import numpy as np
    import oracle as O
    from paper_2201_04622_gb300 import workloads as W
    reps, natoms, _, _ = subset()
    r = reps[q]
    a = W.A_BCC if r["lattice"] == W.BCC else W.A_FCC
    k = W.K_BCC_1400 if r["lattice"] == W.BCC else W.K_FCC_1400
    p = O.eam(**W.EAM_FE_LIKE)
    th = O.eam_theta(p)
    x0, box = O.create_crystal(r["lattice"], a, r["n"], r["n"], r["n"])
    mass = W.MASS_FE_AMU * O.amu()
    m = O.md(dt=1e-3, T=r["T"], damp=0.1, mass=mass, k_spring=k, lambda_fn=2, path=O.PATH_FL,
             t_eq=T_EQ, t_s=T_S, seed=r["seed"], replica=r["replica"], fix_cm=1)
    v = O.init_velocities(m, len(x0))
    t0 = time.time()
    out = O.switch_run(p, th, m, x0, v, x0, box)
    F, _, ed = O.free_energy(len(x0), float(np.prod(box)), r["T"], mass, k, [out["W_f"]], [out["W_b"]])
    return dict(replica=q, lattice=r["lattice"], n=r["n"], natoms=len(x0), T=r["T"], a=a, k=k,
                seed=r["seed"], W_f=out["W_f"], W_b=out["W_b"], F_per_atom=F, Ediss_per_atom=ed,
                oracle_seconds=time.time() - t0)


def main():
    import oracle as O
    O.build()
    _, natoms, small, rand = subset()
    jobs = sorted(small + rand, key=lambda q: -natoms[q])  # largest first
    t0 = time.time()
    with ProcessPoolExecutor(max_workers=min(8, os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        rows = sorted(ex.map(run, jobs), key=lambda d: d["replica"])
    doc = {"_source": "CPU FP64 oracle (oracle/), written by tests/golden/make_config3_subset_works.py",
           "cite": "Sec. III.B: Frenkel-Ladd switching, forward and backward works, eq. fl + eq. cm",
           "set": "workloads.batched_replicas(256, seed=1)", "t_eq": T_EQ, "t_s": T_S,
           "dt_ps": 1e-3, "damping_ps": 0.1, "lambda_fn": 2,
           "subset": {"smallest": small, "random_pcg64_3": rand}, "rows": rows}
    with open(os.path.join(HERE, "config3_subset_works.json"), "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote %d rows in %.0f s" % (len(rows), time.time() - t0))


if __name__ == "__main__":
    main()
