"""The paper's protocol over the C ABI (Sec. III): spring constant from the
mean-squared displacement, batched forward/backward Frenkel-Ladd switching,
and free-energy assembly.  Orchestration only -- every step runs in libne.so.
"""
from __future__ import annotations

import numpy as np

from . import ne

AMU = 1.0364269656262175e-4  # eV ps^2 / A^2


def crystal_sites(lattice, a, n):
    return ne.ne_create_crystal(lattice, a, n, n, n)


def fit_spring_constant(ctx, lattice, a, n, T, mass, prec=ne.NE_MIXED, seed=1, n_eq=2000,
                        n_samples=500, stride=10, skin=1.0, device="cuda"):
    """k = 3 k_B T / <msd> (eq. msd) from a lambda = 0 Langevin run of the
    same size and temperature as the switching runs (Sec. III.A)."""
    import torch
    x0_np, box = crystal_sites(lattice, a, n)
    md = ne.md_params(T=T, mass=mass, skin=skin, prec=prec, seed=seed, replica=0, fix_cm=1)
    x0 = torch.tensor(x0_np, dtype=torch.float64, device=device)
    x, v = x0.clone(), torch.zeros_like(x0)
    ne.ne_init_velocities(ctx, md, v)
    msd, k = ne.ne_msd_fit(ctx, md, x, v, x0, box, n_eq, n_samples, stride)
    return k, msd


def fl_batch(ctx, crystals, T, ks, seeds, t_eq, t_s, mass, prec=ne.NE_MIXED, runner="crystal",
             skin=2.6, device="cuda", chunk=None):
    """Forward and backward FL works of a batch of crystal replicas.

    crystals: list of (lattice, a, n) per replica; ks, seeds: per replica.
    runner: "crystal" (persistent cluster runner, mixed precision) or
    "general" (multi-kernel path, FP64 or mixed).  Returns (W_f, W_b) numpy
    arrays and the final positions."""
    import torch
    x0s, offs, boxes, mds, crs = [], [0], [], [], []
    for r, ((lat, a, n), k, seed) in enumerate(zip(crystals, ks, seeds)):
        x0, box = crystal_sites(lat, a, n)
        x0s.append(x0)
        offs.append(offs[-1] + len(x0))
        boxes.append(box)
        crs.append((lat, a, n, n, n))
        mds.append(ne.md_params(T=T, mass=mass, k_spring=k, skin=skin, prec=prec, t_eq=t_eq, t_s=t_s,
                                seed=seed, replica=r, fix_cm=1))
    x0 = torch.tensor(np.concatenate(x0s), dtype=torch.float64, device=device)
    x, v = x0.clone(), torch.zeros_like(x0)
    for r, m in enumerate(mds):
        ne.ne_init_velocities(ctx, m, v[offs[r]:offs[r + 1]])
    W = torch.zeros((len(mds), 2), dtype=torch.float64, device=device)
    S = 2 * t_eq + 2 * t_s
    step = chunk or S
    for s0 in range(0, S, step):
        ns = min(step, S - s0)
        if runner == "crystal":
            ne.ne_crystal_run_segment(ctx, mds, crs, x, v, W, s0, ns)
        else:
            ne.ne_switch_run_segment(ctx, mds, offs, x, v, x0, boxes, W, s0, ns)
    Wn = W.cpu().numpy()
    return Wn[:, 0], Wn[:, 1], x


def free_energy(lattice, a, n, T, mass, k, W_f, W_b):
    """(F per atom, standard error, dissipation per atom) from eq. fl + eq. cm."""
    x0, box = crystal_sites(lattice, a, n)
    return ne.ne_free_energy(len(x0), float(np.prod(box)), T, mass, k, W_f, W_b)
