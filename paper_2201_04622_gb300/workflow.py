"""The paper's protocol over the C ABI (Sec. III): spring constant from the
mean-squared displacement, batched forward/backward Frenkel-Ladd switching,
and free-energy assembly.  Orchestration only -- every step runs in libne.so.
"""
from __future__ import annotations

import numpy as np

from . import ne

AMU = 1.0364269656262175e-4  # eV ps^2 / A^2
KB = 8.617333262e-5  # eV / K
EV_PER_A3_IN_GPA = 160.21766339999999


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


def fit_spring_constants(ctx, crystals, Ts, mass, prec=ne.NE_MIXED, seed=1, n_eq=2000, n_samples=500,
                         stride=10, skin=1.0, device="cuda", replica_ids=None):
    """One spring per replica of a batch (eq. msd at each replica's own N and
    T, Sec. III.A: the fit must use the size and temperature of the switching
    runs), all replicas in one batched run (ne_msd_fit_batched).  crystals:
    (lattice, a, n) per replica; Ts: one temperature per replica.  Returns
    numpy (k, msd) arrays."""
    import torch
    ids = list(range(len(crystals))) if replica_ids is None else list(replica_ids)
    x0s, offs, boxes, mds = [], [0], [], []
    for (lat, a, n), Tr, rid in zip(crystals, Ts, ids):
        x0, box = crystal_sites(lat, a, n)
        x0s.append(x0)
        offs.append(offs[-1] + len(x0))
        boxes.append(box)
        mds.append(ne.md_params(T=Tr, mass=mass, skin=skin, prec=prec, seed=seed, replica=rid, fix_cm=1))
    x0 = torch.tensor(np.concatenate(x0s), dtype=torch.float64, device=device)
    x, v = x0.clone(), torch.zeros_like(x0)
    for r, m in enumerate(mds):
        ne.ne_init_velocities(ctx, m, v[offs[r]:offs[r + 1]])
    msd, k = ne.ne_msd_fit_batched(ctx, mds, offs, x, v, x0, boxes, n_eq, n_samples, stride)
    return k, msd


def uneven_campaign(ctx, replicas, mass, t_eq, t_s, fit=dict(n_eq=2000, n_samples=500, stride=10), chunk=5000,
                    device="cuda"):
    """The uneven-batch workload of the batching pattern: replicas given as
    dicts (lattice, n, T, seed, replica; workloads.batched_replicas), each
    with its own spring from eq. msd at its own size and temperature (one
    batched fit), then one forward and one backward FL switch per replica on
    the batch advancer (crystal runner, and the multi-kernel path for any
    replica that leaves its range).  Returns per replica (k, W_f, W_b, F per
    atom) as a list of dicts."""
    from . import workloads as WL
    crystals = [(r["lattice"], WL.A_BCC if r["lattice"] == WL.BCC else WL.A_FCC, r["n"]) for r in replicas]
    Ts = [r["T"] for r in replicas]
    ids = [r["replica"] for r in replicas]
    k, _ = fit_spring_constants(ctx, crystals, Ts, mass, replica_ids=ids, device=device, **fit)
    Wf, Wb, _ = fl_batch(ctx, crystals, Ts, list(k), [r["seed"] for r in replicas], t_eq, t_s, mass,
                         runner="auto", chunk=chunk, replica_ids=ids, device=device)
    out = []
    for q, ((lat, a, n), Tr) in enumerate(zip(crystals, Ts)):
        F, se, ed = free_energy(lat, a, n, Tr, mass, k[q], [Wf[q]], [Wb[q]])
        out.append(dict(k=float(k[q]), W_f=float(Wf[q]), W_b=float(Wb[q]), F=F))
    return out


def fl_batch(ctx, crystals, T, ks, seeds, t_eq, t_s, mass, prec=ne.NE_MIXED, runner="crystal",
             skin=2.6, device="cuda", chunk=None, replica_ids=None):
    """Forward and backward FL works of a batch of crystal replicas.

    crystals: list of (lattice, a, n) per replica; ks, seeds: per replica;
    T: one temperature or one per replica; replica_ids: the Philox replica
    index of each replica (default 0 .. n-1).
    runner: "crystal" (persistent cluster runner, mixed precision),
    "general" (multi-kernel path, FP64 or mixed), or "auto": the crystal
    runner in chunks (`chunk` steps, default 5000) on a BatchAdvancer; a
    replica that leaves the runner's stencil range (NE_ERANGE: a hop or
    melting at high T) continues on the general mixed path from its state
    before that chunk, alongside the crystal runner for the others.
    Returns (W_f, W_b) numpy arrays and the final positions."""
    import torch
    ids = list(range(len(crystals))) if replica_ids is None else list(replica_ids)
    if runner == "auto":
        return _fl_batch_auto(ctx, crystals, T, ks, seeds, t_eq, t_s, mass, prec, skin, device, chunk, ids)
    x0s, offs, boxes, mds, crs = [], [0], [], [], []
    Ts = list(T) if np.ndim(T) else [T] * len(crystals)
    for r, ((lat, a, n), k, seed, Tr) in enumerate(zip(crystals, ks, seeds, Ts)):
        x0, box = crystal_sites(lat, a, n)
        x0s.append(x0)
        offs.append(offs[-1] + len(x0))
        boxes.append(box)
        crs.append((lat, a, n, n, n))
        mds.append(ne.md_params(T=Tr, mass=mass, k_spring=k, skin=skin, prec=prec, t_eq=t_eq, t_s=t_s,
                                seed=seed, replica=ids[r], fix_cm=1))
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


class BatchAdvancer:
    """Advances a batch of crystal replicas over step ranges of the schedule:
    the crystal runner for the replicas inside its stencil range and the
    multi-kernel mixed path for the others, the two at once (a second
    context from ne_ctx_clone, its own stream and host thread).  A replica
    that leaves the range inside a chunk (NE_ERANGE: a hop or melting at high
    T) is rerun for that chunk from its state before it on the multi-kernel
    path and stays there.  Each replica's trajectory depends only on its own
    inputs and noise stream, so a move changes rounding only.

    mds, crystals, offsets, boxes, x0: as for ne_crystal_run_segment and
    ne_switch_run_segment (x0: the sites, device [N][3]); chunk: steps per
    crystal-runner call (None: the whole range in one call).  `moved` lists
    the replicas on the multi-kernel path, and `log` each call: (path,
    replicas, first step, steps).  Replicas larger than a cluster holds
    (ne.CRYSTAL_RUNNER_MAX_ATOMS) run on the library's brick runner with the
    rest; if the device cannot hold the batch's CTAs at once (NE_ENOMEM), they
    move to the multi-kernel path instead."""

    def __init__(self, ctx, mds, crystals, offsets, boxes, x0, chunk=None):
        import torch
        self.ctx, self.mds, self.crystals = ctx, list(mds), list(crystals)
        self.offs, self.boxes, self.x0 = list(offsets), list(boxes), x0
        self.chunk = chunk
        self.moved = []
        self.log = []
        self._ctx_g = None
        self._packed = None
        self._cuda = bool(getattr(x0, "is_cuda", False))
        self._sc = torch.cuda.Stream() if self._cuda else None
        # the multi-kernel path's short kernels at high priority: the crystal
        # runner's persistent clusters hold their SMs for a whole chunk, and a
        # freed SM should go to the moved replicas' next kernel first
        self._sg = torch.cuda.Stream(priority=-1) if self._cuda else None

    @staticmethod
    def _handle(st):
        return st.cuda_stream if st is not None else None

    def _sync(self):
        if self._cuda:
            import torch
            torch.cuda.synchronize()

    def close(self):
        if self._ctx_g is not None:
            ne.ne_ctx_destroy(self._ctx_g)
            self._ctx_g = None

    def _general_ctx(self):
        if self._ctx_g is None:
            self._ctx_g = ne.ne_ctx_clone(self.ctx, self.offs[-1], len(self.mds))
        return self._ctx_g

    def _gather(self, idx, x, v, W):
        """Compact copies of the replicas idx (views if idx is the batch)."""
        import torch
        if idx == list(range(len(self.mds))):
            return x, v, W, self.x0, self.offs
        so = [0]
        for r in idx:
            so.append(so[-1] + self.offs[r + 1] - self.offs[r])
        xs = torch.empty((so[-1], 3), dtype=x.dtype, device=x.device)
        vs, x0s = torch.empty_like(xs), torch.empty_like(xs)
        Ws = torch.empty((len(idx), 2), dtype=W.dtype, device=W.device)
        for q, r in enumerate(idx):
            a, b = self.offs[r], self.offs[r + 1]
            xs[so[q]:so[q + 1]].copy_(x[a:b])
            vs[so[q]:so[q + 1]].copy_(v[a:b])
            x0s[so[q]:so[q + 1]].copy_(self.x0[a:b])
            Ws[q].copy_(W[r])
        return xs, vs, Ws, x0s, so

    def _scatter(self, idx, so, xs, vs, Ws, x, v, W):
        if xs is x:
            return
        for q, r in enumerate(idx):
            a, b = self.offs[r], self.offs[r + 1]
            x[a:b].copy_(xs[so[q]:so[q + 1]])
            v[a:b].copy_(vs[so[q]:so[q + 1]])
            W[r].copy_(Ws[q])

    def _general(self, idx, xs, vs, x0s, so, Ws, s0, ns):
        ne.ne_switch_run_segment(self._general_ctx(), [self.mds[r] for r in idx], so, xs, vs, x0s,
                                 [self.boxes[r] for r in idx], Ws, s0, ns, stream=self._handle(self._sg))
        self.log.append(("general", list(idx), s0, ns))

    def advance(self, x, v, W, s0, ns):
        step = self.chunk or ns
        for c0 in range(s0, s0 + ns, step):
            self._advance_chunk(x, v, W, c0, min(step, s0 + ns - c0))

    def _crystal(self, on_c, x, v, W, c0, cn, stream):
        """The crystal runner over replicas on_c (x, v, W compact for them);
        returns the replicas (batch indices) that left its range.  A replica
        that raised an error keeps its state of step c0 (the runner writes back
        only replicas that completed the chunk)."""
        key = tuple(on_c)
        if self._packed is None or self._packed[0] != key:
            self._packed = (key, ne.CrystalBatch([self.mds[r] for r in on_c], [self.crystals[r] for r in on_c]))
        try:
            ne.ne_crystal_run_segment(self.ctx, self._packed[1], None, x, v, W, c0, cn, stream=stream)
        except ne.NeError as e:
            if "NE_ERANGE" not in str(e):
                raise
            st = ne.ne_ctx_replica_status(self.ctx, len(on_c))
            bad = [on_c[q] for q in range(len(on_c)) if st[q] == ne.NE_ERANGE]
            if not bad:
                raise
            return bad
        finally:
            self.log.append(("crystal", list(on_c), c0, cn))
        return []

    def _advance_chunk(self, x, v, W, c0, cn):
        import threading
        on_c = [r for r in range(len(self.mds)) if r not in self.moved]
        gen = list(self.moved)
        if not gen:
            # every replica on the crystal runner: one call on the caller's
            # stream, no copies and no extra synchronisation
            try:
                bad = self._crystal(on_c, x, v, W, c0, cn, None)
            except ne.NeError as e:
                large = [r for r in on_c if self.offs[r + 1] - self.offs[r] > ne.CRYSTAL_RUNNER_MAX_ATOMS]
                if "NE_ENOMEM" not in str(e) or not large:
                    raise
                # the batch's bricks do not fit the device at once: the large
                # replicas go to the multi-kernel path (nothing has run yet)
                self.moved = sorted(self.moved + large)
                return self._advance_chunk(x, v, W, c0, cn)
        else:
            xc, vc, Wc, _, sc = self._gather(on_c, x, v, W) if on_c else (None,) * 5
            xg, vg, Wg, x0g, sg = self._gather(gen, x, v, W)
            self._sync()
            errs, th = [], None
            if not on_c:
                self._general(gen, xg, vg, x0g, sg, Wg, c0, cn)
            else:
                def work():
                    try:
                        self._general(gen, xg, vg, x0g, sg, Wg, c0, cn)
                    except Exception as e:  # noqa: BLE001 -- re-raised below
                        errs.append(e)
                th = threading.Thread(target=work)
                th.start()
            bad = []
            try:
                if on_c:
                    bad = self._crystal(on_c, xc, vc, Wc, c0, cn, self._handle(self._sc))
            finally:
                if th is not None:
                    th.join()
            if errs:
                raise errs[0]
            self._sync()
            if on_c:
                self._scatter(on_c, sc, xc, vc, Wc, x, v, W)
            self._scatter(gen, sg, xg, vg, Wg, x, v, W)
        if bad:
            import warnings
            warnings.warn("replicas %s left the crystal runner's stencil range at steps %d-%d; they continue "
                          "on the multi-kernel path" % (bad, c0, c0 + cn))
            # their state of step c0 is in place: rerun the chunk on the multi-kernel path
            xb, vb, Wb, x0b, sb = self._gather(bad, x, v, W)
            self._sync()
            self._general(bad, xb, vb, x0b, sb, Wb, c0, cn)
            self._sync()
            self._scatter(bad, sb, xb, vb, Wb, x, v, W)
            self.moved = sorted(self.moved + bad)
            self._sync()


def _fl_batch_auto(ctx, crystals, T, ks, seeds, t_eq, t_s, mass, prec, skin, device, chunk, ids):
    """fl_batch(runner="auto") on a BatchAdvancer (chunks of 5000 steps unless given)."""
    import torch
    x0s, offs, boxes, mds, crs = [], [0], [], [], []
    Ts = list(T) if np.ndim(T) else [T] * len(crystals)
    for r, ((lat, a, n), k, seed, Tr) in enumerate(zip(crystals, ks, seeds, Ts)):
        x0, box = crystal_sites(lat, a, n)
        x0s.append(x0)
        offs.append(offs[-1] + len(x0))
        boxes.append(box)
        crs.append((lat, a, n, n, n))
        mds.append(ne.md_params(T=Tr, mass=mass, k_spring=k, skin=skin, prec=ne.NE_MIXED, t_eq=t_eq, t_s=t_s,
                                seed=seed, replica=ids[r], fix_cm=1))
    x0 = torch.tensor(np.concatenate(x0s), dtype=torch.float64, device=device)
    x, v = x0.clone(), torch.zeros_like(x0)
    for r, m in enumerate(mds):
        ne.ne_init_velocities(ctx, m, v[offs[r]:offs[r + 1]])
    W = torch.zeros((len(mds), 2), dtype=torch.float64, device=device)
    adv = BatchAdvancer(ctx, mds, crs, offs, boxes, x0, chunk=chunk or 5000)
    try:
        adv.advance(x, v, W, 0, 2 * t_eq + 2 * t_s)
    finally:
        adv.close()
    Wn = W.cpu().numpy()
    return Wn[:, 0], Wn[:, 1], x


def free_energy(lattice, a, n, T, mass, k, W_f, W_b):
    """(F per atom, standard error, dissipation per atom) from eq. fl + eq. cm."""
    x0, box = crystal_sites(lattice, a, n)
    return ne.ne_free_energy(len(x0), float(np.prod(box)), T, mass, k, W_f, W_b)


def pressure(ctx, lattice, a, n, T, mass, n_eq=2000, n_samples=50, stride=20, prec=ne.NE_MIXED, seed=1,
             skin=1.0, device="cuda"):
    """Pressure of an n^3 crystal at lattice parameter a and temperature T
    (NVT Langevin at lambda = 0 of the FL schedule): P = (N_dof k_B T + <W>) / (3V),
    W the configurational virial (ne_eam_virial) sampled every `stride` steps
    after n_eq steps.  Returns (P, standard error) in eV/A^3."""
    import torch
    x0_np, box = crystal_sites(lattice, a, n)
    nat = len(x0_np)
    t_eq = n_eq + n_samples * stride
    md = ne.md_params(T=T, mass=mass, skin=skin, prec=prec, t_eq=t_eq, t_s=1, seed=seed, replica=0, fix_cm=1)
    x0 = torch.tensor(x0_np, dtype=torch.float64, device=device)
    x, v = x0.clone(), torch.zeros_like(x0)
    ne.ne_init_velocities(ctx, md, v)
    Wd = torch.zeros((1, 2), dtype=torch.float64, device=device)
    w = torch.zeros(1, dtype=torch.float64, device=device)
    ne.ne_switch_run_segment(ctx, [md], [0, nat], x, v, x0, [box], Wd, 0, n_eq)
    ws, s0 = [], n_eq
    for _ in range(n_samples):
        ne.ne_switch_run_segment(ctx, [md], [0, nat], x, v, x0, [box], Wd, s0, stride)
        s0 += stride
        ne.ne_eam_virial(ctx, x, box, w)
        ws.append(float(w.item()))
    return ne.ne_pressure(3 * nat - 3, T, float(np.prod(box)), ws)


def lattice_parameter(ctx, lattice, n, T, mass, a_grid, **kw):
    """Zero-pressure lattice parameter at T (Sec. III.A: the crystal is set to
    P = 0 before switching): P(a) on a_grid, a straight line through the
    points, its root.  Returns (a0, [(a, P, err)])."""
    pts = [(a,) + tuple(pressure(ctx, lattice, a, n, T, mass, **kw)) for a in a_grid]
    A = np.array([[1.0, a] for a, _, _ in pts])
    c = np.linalg.lstsq(A, np.array([P for _, P, _ in pts]), rcond=None)[0]
    return -c[0] / c[1], pts


def fl_free_energies(lattice, a, n, T, mass, k, W_f, W_b):
    """Free energy per atom from one set of FL works: the two-sided estimate
    (eq. fl + eq. cm) with its standard error and dissipation, and the
    one-sided Jarzynski estimates (eq. jarz) from the forward works (the
    system goes EAM -> Einstein, work done on it -W_f) and from the backward
    works (Einstein -> EAM, work -W_b)."""
    x0, box = crystal_sites(lattice, a, n)
    nat, V = len(x0), float(np.prod(box))
    F, se, ed = ne.ne_free_energy(nat, V, T, mass, k, W_f, W_b)
    F_ref = ne.ne_free_energy(nat, V, T, mass, k, [0.0], [0.0])[0]  # F_E + dF_CM per atom
    return {"F": F, "stderr": se, "Ediss": ed,
            "F_jarzynski_fwd": F_ref - ne.ne_jarzynski(T, -np.asarray(W_f, np.float64)) / nat,
            "F_jarzynski_bwd": F_ref + ne.ne_jarzynski(T, -np.asarray(W_b, np.float64)) / nat}


def fl_convergence(ctx, lattice, a, n, T, mass, k, t_s_list, seeds, t_eq, **kw):
    """The FL free energy and dissipation against the switching time
    (the convergence study of Sec. III.B): for each t_s (steps), one forward
    and backward run per seed.  Returns one row per t_s."""
    rows = []
    for ts in t_s_list:
        Wf, Wb, _ = fl_batch(ctx, [(lattice, a, n)] * len(seeds), T, [k] * len(seeds), list(seeds), t_eq, ts,
                             mass, **kw)
        rows.append(dict(t_s=ts, **fl_free_energies(lattice, a, n, T, mass, k, Wf, Wb)))
    return rows


def size_scaling(ctx, lattice, a, sizes, T, mass, k, seeds, t_eq, t_s, **kw):
    """F(N) for n^3 cells (the finite-size study of Sec. IV.A), all sizes and
    seeds in one batch, and a straight-line fit in 1/N: returns the rows and
    (F at 1/N -> 0, slope).  k: one spring for every size, or one per size.
    With runner="auto" (fl_batch) a batch holding cells larger than a
    cluster holds runs on the brick runner (those cells move to the
    multi-kernel path if the batch's CTAs do not fit the device at once), so
    the sizes can reach the paper's ~1.1e4 atoms (bcc 18^3)."""
    ks = list(k) if np.ndim(k) else [k] * len(sizes)
    crystals = [(lattice, a, m) for m in sizes for _ in seeds]
    kr = [kq for kq in ks for _ in seeds]
    ids = kw.pop("replica_ids", None)
    Wf, Wb, _ = fl_batch(ctx, crystals, T, kr, list(seeds) * len(sizes), t_eq, t_s, mass, replica_ids=ids, **kw)
    rows, ns = [], len(seeds)
    for q, m in enumerate(sizes):
        x0, _ = crystal_sites(lattice, a, m)
        r = fl_free_energies(lattice, a, m, T, mass, ks[q], Wf[q * ns:(q + 1) * ns], Wb[q * ns:(q + 1) * ns])
        rows.append(dict(n=m, atoms=len(x0), k=ks[q], W_f=list(Wf[q * ns:(q + 1) * ns]),
                         W_b=list(Wb[q * ns:(q + 1) * ns]), **r))
    inv = np.array([1.0 / r["atoms"] for r in rows])
    Fs = np.array([r["F"] for r in rows])
    slope, F_inf = np.polyfit(inv, Fs, 1)
    return rows, (F_inf, slope)


def rs_works(ctx, lattice, a, n, T0, mass, lambda_f, t_eq, t_s, seeds, prec=ne.NE_MIXED, skin=1.0, npt=False,
             beta_T=1.2, tau_p=0.5, device="cuda", replica_ids=None, chunk=None):
    """Reversible scaling (Sec. III.C): per seed, t_eq steps at lambda = 1,
    a forward switch to lambda_f over t_s steps, t_eq steps there and the
    switch back, at T0, in the box of lattice parameter a or, with npt, at
    zero pressure under the isotropic barostat (beta_T, tau_p: its coupling).
    All seeds run as one batch on the multi-kernel path
    (ne_switch_run_segment_cum; replica index 0 for every seed unless
    replica_ids is given), in segments of `chunk` steps (all at once by
    default).  Returns the cumulative works [seeds][t_s + 1] (forward,
    backward) and, with npt, the final lattice parameters (box edge / cells)."""
    import torch
    x0_np, box = crystal_sites(lattice, a, n)
    nat, nr = len(x0_np), len(seeds)
    ids = [0] * nr if replica_ids is None else list(replica_ids)
    mds = [ne.md_params(T=T0, mass=mass, skin=skin, prec=prec, path=ne.NE_PATH_RS, lambda_f=lambda_f,
                        t_eq=t_eq, t_s=t_s, seed=seed, replica=rid, fix_cm=1, npt=int(npt), P0=0.0,
                        beta_T=beta_T, tau_p=tau_p) for seed, rid in zip(seeds, ids)]
    x0 = torch.tensor(np.concatenate([x0_np] * nr), dtype=torch.float64, device=device)
    x, v = x0.clone(), torch.zeros_like(x0)
    offs = [q * nat for q in range(nr + 1)]
    for r, m in enumerate(mds):
        ne.ne_init_velocities(ctx, m, v[offs[r]:offs[r + 1]])
    W = torch.zeros((nr, 2), dtype=torch.float64, device=device)
    Wc = torch.zeros(nr * 2 * (t_s + 1), dtype=torch.float64, device=device)
    boxes = [list(box)] * nr
    S = 2 * t_eq + 2 * t_s
    for s0 in range(0, S, chunk or S):
        ns = min(chunk or S, S - s0)
        ne.ne_switch_run_segment_cum(ctx, mds, offs, x, v, x0, boxes, W, Wc, s0, ns)
        if npt:  # the barostat moved the boxes: the next segment starts from them
            boxes = [list(b) for b in ne.ne_ctx_boxes(ctx, nr)]
    wc = Wc.cpu().numpy().reshape(nr, 2, t_s + 1)
    a_end = np.array([b[0] / n for b in boxes]) if npt else np.array([])
    return wc[:, 0], wc[:, 1], a_end


def rs_batch(ctx, crystals, T0, seeds, lambda_f, t_eq, t_s, mass, replica_ids=None, chunk=20000,
             device="cuda", npt=False, beta_T=1.2, tau_p=0.5):
    """Reversible scaling (Sec. III.C) for a batch of crystal replicas on the
    crystal runners (the cluster runner, or the brick runner for replicas
    above ne.CRYSTAL_RUNNER_MAX_ATOMS): per replica, t_eq steps at
    lambda = 1, the switch to lambda_f over t_s steps, t_eq steps there and
    the switch back, at T0 (one value or one per replica), in the box of the
    given lattice parameter or, with npt, at zero pressure under the
    isotropic barostat (beta_T, tau_p: its coupling; each chunk starts from
    the lattice parameter the last one reached).  Returns the cumulative
    works [n_rep][t_s + 1] (forward, backward) for eq. rs (rs_free_energy)
    and the final lattice parameters (box edge / cells; the given ones
    without npt)."""
    import torch
    n = len(crystals)
    ids = list(range(n)) if replica_ids is None else list(replica_ids)
    Ts = list(T0) if np.ndim(T0) else [T0] * n
    x0s, offs, mds, crs = [], [0], [], []
    for r, ((lat, a, nc), seed, Tr) in enumerate(zip(crystals, seeds, Ts)):
        x0, _ = crystal_sites(lat, a, nc)
        x0s.append(x0)
        offs.append(offs[-1] + len(x0))
        crs.append((lat, a, nc, nc, nc))
        mds.append(ne.md_params(T=Tr, mass=mass, k_spring=1.0, prec=ne.NE_MIXED, path=ne.NE_PATH_RS,
                                lambda_f=lambda_f, t_eq=t_eq, t_s=t_s, seed=seed, replica=ids[r], fix_cm=1,
                                npt=int(bool(npt)), P0=0.0, beta_T=beta_T, tau_p=tau_p))
    x = torch.tensor(np.concatenate(x0s), dtype=torch.float64, device=device)
    v = torch.zeros_like(x)
    for r, m in enumerate(mds):
        ne.ne_init_velocities(ctx, m, v[offs[r]:offs[r + 1]])
    W = torch.zeros((n, 2), dtype=torch.float64, device=device)
    Wc = torch.zeros(n * 2 * (t_s + 1), dtype=torch.float64, device=device)
    S = 2 * t_eq + 2 * t_s
    for s0 in range(0, S, chunk or S):
        ne.ne_crystal_run_segment_cum(ctx, mds, crs, x, v, W, Wc, s0, min(chunk or S, S - s0))
        if npt:  # the barostat moved the boxes: the next chunk starts from their lattice parameter
            crs = [(c[0], b[0] / c[2], c[2], c[3], c[4]) for c, b in zip(crs, ne.ne_ctx_boxes(ctx, n))]
    wc = Wc.cpu().numpy().reshape(n, 2, t_s + 1)
    return wc[:, 0], wc[:, 1], np.array([c[1] for c in crs])


def rs_free_energy(lattice, a, n, T0, F0_T0_per_atom, lambda_f, t_s, Wcum_f, Wcum_b, T_grid):
    """Eq. rs: free energy per atom on T_grid (T0 .. T0/lambda_f) from the
    cumulative works and the free energy at T0 (with the barostat at P = 0,
    the Gibbs free energy)."""
    x0, _ = crystal_sites(lattice, a, n)
    nat = len(x0)
    return ne.ne_rs_free_energy(nat, T0, F0_T0_per_atom * nat, lambda_f, t_s, Wcum_f, Wcum_b, T_grid)


def transition_temperatures(T_grid, F_a, F_b):
    """Temperatures where two phases exchange stability (Sec. IV): the sign
    changes of dF(T) = F_a(T) - F_b(T) on an ascending T_grid.  Between two
    consecutive grid points with nonzero dF of opposite sign the crossing is
    located by linear interpolation; when grid points with dF exactly zero
    separate them, it is the mean temperature of those points.  Returns a
    list of (T, phase stable above: 0 for a, 1 for b)."""
    T = np.asarray(T_grid, dtype=np.float64).ravel()
    d = np.asarray(F_a, dtype=np.float64).ravel() - np.asarray(F_b, dtype=np.float64).ravel()
    if T.size != d.size or T.size < 2 or np.any(np.diff(T) <= 0):
        raise ValueError("T_grid must be ascending with one F_a and F_b value per point")
    nz = np.flatnonzero(d != 0.0)
    out = []
    for q0, q1 in zip(nz[:-1], nz[1:]):
        if np.sign(d[q0]) == np.sign(d[q1]):
            continue
        if q1 == q0 + 1:
            Tc = T[q0] + (T[q1] - T[q0]) * d[q0] / (d[q0] - d[q1])
        else:
            Tc = T[q0 + 1:q1].mean()
        out.append((float(Tc), 0 if d[q1] < 0 else 1))
    return out


def theta_gradient(ctx, lattice, a, n, T, mass, k, t_eq, t_s, n_knots, seed=1, stride=10, prec=ne.NE_MIXED,
                   skin=1.0, device="cuda"):
    """Gradients with respect to the spline knots theta along one FL run
    (equilibration at lambda = 0, then the forward switch of Sec. III.B),
    with dU/dtheta from the backward pass every `stride` steps, fused into
    the run (ne_switch_run_segment_grad: the step's own list and rho):
      dF_dtheta  -- <dU/dtheta> over the equilibration at lambda = 0, the
                    free energy's parameter gradient dF_0/dtheta;
      dWf_dtheta -- sum over the forward switch of dlambda dU/dtheta(x), the
                    derivative of W_f at fixed trajectory (lambda increments
                    over `stride` steps).
    Returns (dF_dtheta, dWf_dtheta, samples at lambda = 0), the gradients as
    numpy [3][n_knots][2] (phi, f, F; value and slope per knot)."""
    import torch
    x0_np, box = crystal_sites(lattice, a, n)
    nat = len(x0_np)
    md = ne.md_params(T=T, mass=mass, k_spring=k, skin=skin, prec=prec, t_eq=t_eq, t_s=t_s, seed=seed,
                      replica=0, fix_cm=1)
    x0 = torch.tensor(x0_np, dtype=torch.float64, device=device)
    x, v = x0.clone(), torch.zeros_like(x0)
    ne.ne_init_velocities(ctx, md, v)
    Wd = torch.zeros((1, 2), dtype=torch.float64, device=device)
    g_eq = torch.zeros(6 * n_knots, dtype=torch.float64, device=device)
    g_sw = torch.zeros(6 * n_knots, dtype=torch.float64, device=device)
    # sample points s = stride, 2 stride, ... (and the end of the switch):
    # weight 1 at lambda = 0, the lambda increment since the previous sample
    # during the switch; one fused run per phase (ne_switch_run_segment_grad)
    S = t_eq + t_s
    samples = list(range(stride, S, stride)) + [S]
    w_eq = np.zeros(t_eq + 1)
    w_sw = np.zeros(t_s + 1)
    n_eq, prev = 0, 0
    for s in samples:
        if s <= t_eq:
            w_eq[s] = 1.0
            n_eq += 1
        else:
            w_sw[s - t_eq] = ne.ne_lambda(md, s) - ne.ne_lambda(md, max(prev, t_eq))
        prev = s
    for s0, ns, w, g in ((0, t_eq, w_eq, g_eq), (t_eq, t_s, w_sw, g_sw)):
        if ns > 0:
            wd = torch.tensor(w, dtype=torch.float64, device=device)
            ne.ne_switch_run_segment_grad(ctx, [md], [0, nat], x, v, x0, [box], Wd, s0, ns, wd, g)
    shape = (3, n_knots, 2)
    return (g_eq.cpu().numpy() / max(n_eq, 1)).reshape(shape), g_sw.cpu().numpy().reshape(shape), n_eq
