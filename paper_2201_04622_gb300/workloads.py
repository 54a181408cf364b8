"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds data and random draws only -- none of the method's
arithmetic.  Both the CUDA path and the CPU oracle receive what it returns.

The paper's workloads are bcc/fcc iron crystals described by the Meyer-Entel
EAM potential, which is not available here; an analytic Fe-like EAM stands in
for it (Johnson-type exponential pair and density, Finnis-Sinclair square-root
embedding, quintic taper from r_s to r_c).  A and B put the bcc lattice at
a = 2.87 A at -4.28 eV/atom and zero static pressure.
"""
from __future__ import annotations

import numpy as np

# Fe-like analytic EAM (builder-chosen parameters; tabulated on 5000 knots).
EAM_FE_LIKE = dict(A=0.3743608608532552, alpha=8.0, beta=4.0, B=1.7094801525746224,
                   r_e=2.4855, r_s=4.6, r_c=5.3, rho_max=100.0, n_knots=5000)
MASS_FE_AMU = 55.845
# Spring constants k = 3 k_B T / <msd> (eq. msd) of this potential at 1400 K,
# fitted with the library on bcc 10^3 and fcc 8^3 (2 ps + 5 ps, every 10 steps).
K_BCC_1400 = 2.38
K_FCC_1400 = 2.68
A_BCC = 2.87
A_FCC = 3.65
A_HCP = 2.581  # ideal hcp with the fcc nearest-neighbour distance, A_FCC / sqrt(2)
BCC, FCC, HCP = 0, 1, 2


def eam_params(**over):
    p = dict(EAM_FE_LIKE)
    p.update(over)
    return p


def displaced(x0, amp, seed):
    """Sites plus independent uniform displacements in [-amp, amp] per component."""
    g = np.random.Generator(np.random.PCG64(seed))
    return np.asarray(x0, np.float64) + g.uniform(-amp, amp, size=np.shape(x0))


def gaussian_velocities(n, sigma, seed):
    """Zero-mean Gaussian velocities (total momentum removed)."""
    g = np.random.Generator(np.random.PCG64(seed))
    v = g.normal(0.0, sigma, size=(n, 3))
    return v - v.mean(axis=0)


def batched_replicas(n_rep=256, seed=1, T_lo=300.0, T_hi=1600.0):
    """Uneven replica set: structure, supercell edge and temperature per replica.

    bcc n^3 x 2 atoms with n in [6, 12], fcc n^3 x 4 with n in [5, 10], chosen
    with equal odds; T uniform in [T_lo, T_hi]; replica r uses Philox key
    (seed, r)."""
    g = np.random.Generator(np.random.PCG64(seed))
    reps = []
    for r in range(n_rep):
        if g.uniform() < 0.5:
            lat, n = BCC, int(g.integers(6, 13))
        else:
            lat, n = FCC, int(g.integers(5, 11))
        T = float(g.uniform(T_lo, T_hi))
        reps.append(dict(lattice=lat, n=n, T=T, seed=seed, replica=r))
    return reps


# Workload definitions (sizes of the paper-style bcc/fcc runs).
C1 = dict(name="fl_bcc4_T100", lattice=BCC, n=4, a=A_BCC, T=100.0, dt=1e-3, damp=0.1,
          t_eq=2000, t_s=5000, seeds=[1])
C2 = dict(name="fl_bcc10_fcc8_T1400_10seeds",
          systems=[dict(lattice=BCC, n=10, a=A_BCC), dict(lattice=FCC, n=8, a=A_FCC)],
          T=1400.0, dt=1e-3, damp=0.1, t_eq=10000, t_s=50000, seeds=list(range(1, 11)))
C4 = dict(name="rs_bcc16_T100_1600", lattice=BCC, n=16, a=A_BCC, T0=100.0, Tf=1600.0,
          dt=1e-3, damp=0.1, t_eq=10000, t_s=100000)
