"""Autotuner of the multi-kernel path: threads per atom of the pair kernels
and the neighbour-list skin, chosen by timing real steps of the caller's own
batch (ne_profile_segment: CUDA events around every launch, on the launching
stream).  The persistent crystal runner has no free tile parameters."""
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
