"""Autotuners, each timing real steps of the caller's own batch with the
state restored after every trial:
  tune          -- the multi-kernel path: threads per atom of the pair
                   kernels and the neighbour-list skin (ne_profile_segment:
                   CUDA events around every launch, on the launching stream);
  tune_crystal  -- the persistent crystal runner: CTAs per thread-block
                   cluster, i.e. atoms per CTA against clusters resident at
                   once (ne_ctx_last_run_ms: events around the launch)."""
from __future__ import annotations

import itertools

from . import ne


def tune(ctx, mds, offsets, x, v, x0, boxes, W, step_begin=0, n_steps=100,
         threads_per_atom=(1, 2, 4, 8), skins=None):
    """Return (best, table): best = dict(tpa, skin, ms_per_step); table = all
    candidates.  The state (x, v, W) is restored after every trial."""
    rc = ne.ctx_cutoff(ctx)
    if rc is None:
        raise ValueError("context not created through this binding: its cutoff is unknown")
    skins = skins or [m.skin for m in mds[:1]]
    L_min = min(min(b) for b in boxes)
    fits = [(tpa, skin) for tpa, skin in itertools.product(threads_per_atom, skins)
            if 2 * (rc + skin) < L_min]  # the list range must stay under half the box
    if not fits:
        raise ValueError("no candidate skin fits the smallest box (%.3f A) with r_c = %.3f A" % (L_min, rc))
    import torch
    saved = (x.clone(), v.clone(), W.clone())
    old = [m.skin for m in mds]
    table = []
    for tpa, skin in fits:
        for m in mds:
            m.skin = skin
        ne.ne_ctx_set_tuning(ctx, tpa)
        ms, _ = ne.ne_profile_segment(ctx, mds, offsets, x, v, x0, boxes, W, step_begin, n_steps)
        table.append(dict(tpa=tpa, skin=skin, ms_per_step=sum(ms), per_kernel_ms=ms))
        x.copy_(saved[0])
        v.copy_(saved[1])
        W.copy_(saved[2])
    for m, s in zip(mds, old):
        m.skin = s
    best = min(table, key=lambda t: t["ms_per_step"])
    ne.ne_ctx_set_tuning(ctx, best["tpa"])
    for m in mds:
        m.skin = best["skin"]
    torch.cuda.synchronize()
    return best, table


def tune_crystal(ctx, mds, crystals, x, v, W, step_begin=0, n_steps=200, sizes=None, brick=True):
    """The crystal runner for a batch, by timing n_steps of it: the cluster
    runner at every cluster size from the smallest that holds the largest
    replica up to 8 (the portable cluster limit), or `sizes`, and (with
    brick) the brick runner; the fastest is fixed with ne_ctx_set_runner and
    ne_ctx_set_cluster_size.  Returns (best, table): best = dict(runner,
    ctas, us_per_step) (ctas 0 for the brick runner); table = all candidates
    (one the device cannot launch is left out).  x, v, W are restored after
    every trial."""
    import torch
    per_cta = ne.CRYSTAL_RUNNER_ATOMS_PER_CTA
    n_max = max((2 if int(c[0]) == ne.NE_BCC else 4) * int(c[2]) * int(c[3]) * int(c[4]) for c in crystals)
    c_min = max(1, -(-n_max // per_cta))
    cand = list(sizes) if sizes else list(range(c_min, 9))
    saved = (x.clone(), v.clone(), W.clone())
    batch = ne.CrystalBatch(mds, crystals)
    table = []
    trials = [("cluster", C) for C in cand] + ([("brick", 0)] if brick else [])
    try:
        for runner, C in trials:
            try:
                ne.ne_ctx_set_runner(ctx, 1 if runner == "cluster" else 2)
                ne.ne_ctx_set_cluster_size(ctx, C)
                ne.ne_crystal_run_segment(ctx, batch, None, x, v, W, step_begin, min(20, n_steps))  # plan, warm
                x.copy_(saved[0])
                v.copy_(saved[1])
                W.copy_(saved[2])
                ne.ne_crystal_run_segment(ctx, batch, None, x, v, W, step_begin, n_steps)
                ms = ne.ne_ctx_last_run_ms(ctx)
                table.append(dict(runner=runner, ctas=C, us_per_step=ms * 1e3 / n_steps))
            except ne.NeError:
                pass  # too few CTAs for a replica, or more than the device co-schedules
            finally:
                x.copy_(saved[0])
                v.copy_(saved[1])
                W.copy_(saved[2])
    finally:
        torch.cuda.synchronize()
    if not table:
        ne.ne_ctx_set_cluster_size(ctx, 0)
        ne.ne_ctx_set_runner(ctx, 0)
        raise ValueError("no crystal runner could run this batch")
    best = min(table, key=lambda t: t["us_per_step"])
    ne.ne_ctx_set_runner(ctx, 1 if best["runner"] == "cluster" else 2)
    ne.ne_ctx_set_cluster_size(ctx, best["ctas"])
    return best, table
