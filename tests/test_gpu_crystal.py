"""GPU parity of the persistent crystal runner (ne_crystal_run_segment,
mixed precision, one thread-block cluster per replica) against the oracle
and against the multi-kernel path on the same seeded inputs.

Tolerances: the runner computes pair distances as (r0_j - r0_i) + u_j - u_i
in FP32 with |u| < 2 A, so a distance carries ~2^-24 * 5 A ~ 3e-7 A of
rounding (finer than the wrapped-coordinate path); over 100 steps positions
follow the FP64 oracle to ~1e-6 A.  The tests allow 2e-5 A over 100 steps at
the small sizes and 2e-4 A on the 40k-atom batch (FP32 round-off grows with
the chaotic divergence of the trajectories).
"""
import numpy as np
import pytest

import oracle as O
from paper_2201_04622_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2201_04622_gb300 import ne  # noqa: E402

DEV = torch.device("cuda:0")
MASS = W.MASS_FE_AMU * 1.0364269656262175e-4


@pytest.fixture(scope="module")
def pot():
    p = O.eam(**W.EAM_FE_LIKE)
    return p, O.eam_theta(p)


@pytest.fixture(scope="module")
def ctx():
    c = ne.ne_ctx_create(ne.eam_params(**W.EAM_FE_LIKE), 60000, 64)
    yield c
    ne.ne_ctx_destroy(c)


def T(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def lat_a(lat):
    return {O.BCC: W.A_BCC, O.FCC: W.A_FCC, O.HCP: W.A_HCP}[lat]


def md_pair(**kw):
    base = dict(dt=1e-3, T=300.0, damp=0.1, k_spring=6.0, lambda_fn=2, t_eq=20, t_s=30,
                lambda_f=0.5, seed=11, replica=2, fix_cm=1)
    base.update(kw)
    path = base.pop("path", O.PATH_FL)
    mo = O.md(mass=MASS, path=path, **base)
    mg = ne.md_params(mass=MASS, skin=1.0, prec=ne.NE_MIXED, path=path, **base)
    return mo, mg


def run_crystals(ctx, systems, s0, ns, x=None, v=None, Wd=None, **kw):
    mgs, crs, x0s, vs = [], [], [], []
    for r, (lat, n, Tk, seed) in enumerate(systems):
        mo, mg = md_pair(T=Tk, seed=seed, replica=r, **kw)
        x0, box = O.create_crystal(lat, lat_a(lat), n, n, n)
        x0s.append(x0)
        vs.append(O.init_velocities(mo, len(x0)))
        mgs.append(mg)
        crs.append((lat, lat_a(lat), n, n, n))
    if x is None:
        x, v = T(np.concatenate(x0s)), T(np.concatenate(vs))
        Wd = torch.zeros((len(systems), 2), dtype=torch.float64, device=DEV)
    ne.ne_crystal_run_segment(ctx, mgs, crs, x, v, Wd, s0, ns)
    return x, v, Wd, x0s, vs


@pytest.mark.parametrize("lat,n,path", [(O.BCC, 5, O.PATH_FL), (O.FCC, 4, O.PATH_FL),
                                        (O.BCC, 6, O.PATH_RS), (O.HCP, 5, O.PATH_FL)])
def test_crystal_runner_tracks_oracle_100_steps(ctx, pot, lat, n, path):
    p, th = pot
    x, v, Wd, x0s, vs = run_crystals(ctx, [(lat, n, 300.0, 5)], 0, 100, path=path)
    mo, _ = md_pair(T=300.0, seed=5, replica=0, path=path)
    x0, box = O.create_crystal(lat, lat_a(lat), n, n, n)
    ro = O.switch_run(p, th, mo, x0, vs[0], x0, box)
    assert np.abs(x.cpu().numpy() - ro["x"]).max() < 2e-5
    assert np.abs(v.cpu().numpy() - ro["v"]).max() < 2e-3
    Wg = Wd.cpu().numpy()[0]
    assert Wg[0] == pytest.approx(ro["W_f"], rel=1e-5, abs=1e-4)
    assert Wg[1] == pytest.approx(ro["W_b"], rel=1e-5, abs=1e-4)


def test_crystal_runner_matches_multikernel_mixed_path(ctx):
    systems = [(O.BCC, 6, 800.0, 3), (O.FCC, 5, 1200.0, 4), (O.BCC, 8, 400.0, 9)]
    x, v, Wd, x0s, vs = run_crystals(ctx, systems, 0, 100)
    offs = np.cumsum([0] + [len(a) for a in x0s])
    mgs = [md_pair(T=Tk, seed=seed, replica=r)[1] for r, (lat, n, Tk, seed) in enumerate(systems)]
    boxes = [O.create_crystal(lat, lat_a(lat), n, n, n)[1] for (lat, n, Tk, seed) in systems]
    X0 = T(np.concatenate(x0s))
    x2, v2 = X0.clone(), T(np.concatenate(vs))
    W2 = torch.zeros((len(systems), 2), dtype=torch.float64, device=DEV)
    for m in mgs:
        m.skin = 1.0
    ne.ne_switch_run_segment(ctx, mgs, list(offs), x2, v2, X0, boxes, W2, 0, 100)
    assert torch.abs(x - x2).max().item() < 2e-5
    assert torch.allclose(Wd, W2, rtol=1e-5, atol=1e-4)


def test_crystal_runner_full_size_batch(ctx, pot):
    """The benchmark batch (10 bcc 10^3 + 10 fcc 8^3 at 1400 K, 40,480 atoms)
    for 30 steps; replicas 0 and 19 atom by atom against the oracle."""
    p, th = pot
    systems = [(O.BCC, 10, 1400.0, 1 + r) for r in range(10)] + \
              [(O.FCC, 8, 1400.0, 1 + r) for r in range(10)]
    x, v, Wd, x0s, vs = run_crystals(ctx, systems, 0, 30, t_eq=5, t_s=10, k_spring=4.0)
    offs = np.cumsum([0] + [len(a) for a in x0s])
    xg = x.cpu().numpy()
    for r in (0, 19):
        lat, n, Tk, seed = systems[r]
        mo, _ = md_pair(T=Tk, seed=seed, replica=r, t_eq=5, t_s=10, k_spring=4.0)
        x0, box = O.create_crystal(lat, lat_a(lat), n, n, n)
        ro = O.switch_run(p, th, mo, x0, vs[r], x0, box)
        assert np.abs(xg[offs[r]:offs[r + 1]] - ro["x"]).max() < 2e-4
        assert float(Wd[r, 0]) == pytest.approx(ro["W_f"], rel=1e-4, abs=1e-3)
        assert float(Wd[r, 1]) == pytest.approx(ro["W_b"], rel=1e-4, abs=1e-3)
    # work counters advanced: every atom examined stencil entries and found pairs
    builds, visits, pairs, launches = ne.ne_ctx_counters(ctx)
    assert pairs > 30 * offs[-1] * 40 and launches >= 2


def test_crystal_runner_resume_is_bitwise(ctx):
    systems = [(O.BCC, 6, 900.0, 1), (O.FCC, 5, 700.0, 2)]
    S = 2 * 40 + 2 * 150
    x, v, Wd, _, _ = run_crystals(ctx, systems, 0, S, t_eq=40, t_s=150)
    ref = (x.clone(), v.clone(), Wd.clone())
    x, v, Wd, _, _ = run_crystals(ctx, systems, 0, 77, t_eq=40, t_s=150)
    for a, b in ((77, 230), (230, S)):
        run_crystals(ctx, systems, a, b - a, x=x, v=v, Wd=Wd, t_eq=40, t_s=150)
    for p_, q_ in zip(ref, (x, v, Wd)):
        assert torch.equal(p_, q_)


def test_crystal_runner_rejects_small_boxes_and_fp64(ctx):
    mo, mg = md_pair()
    x = torch.zeros((128, 3), dtype=torch.float64, device=DEV)
    Wd = torch.zeros((1, 2), dtype=torch.float64, device=DEV)
    with pytest.raises(ne.NeError, match="NE_EINVAL"):
        ne.ne_crystal_run_segment(ctx, [mg], [(O.BCC, 2.87, 4, 4, 4)], x, x.clone(), Wd, 0, 10)
    mg.prec = ne.NE_FP64
    x = torch.zeros((250, 3), dtype=torch.float64, device=DEV)
    with pytest.raises(ne.NeError, match="NE_EINVAL"):
        ne.ne_crystal_run_segment(ctx, [mg], [(O.BCC, 2.87, 5, 5, 5)], x, x.clone(), Wd, 0, 10)


def test_uneven_batch_size_classes_match_multikernel_path(ctx):
    """Replicas of 432 to 4000 atoms (bcc, fcc and hcp; cluster sizes 2 to 11
    CTAs, launched per size class on separate streams) against the
    multi-kernel mixed path."""
    systems = [(O.BCC, 6, 1500.0, 1), (O.FCC, 10, 600.0, 2), (O.BCC, 9, 1100.0, 3), (O.FCC, 5, 300.0, 4),
               (O.BCC, 12, 900.0, 5), (O.FCC, 7, 1300.0, 6), (O.BCC, 6, 400.0, 7), (O.HCP, 6, 1000.0, 8)]
    x, v, Wd, x0s, vs = run_crystals(ctx, systems, 0, 60, t_eq=10, t_s=25, k_spring=3.0)
    offs = np.cumsum([0] + [len(a) for a in x0s])
    mgs = [md_pair(T=Tk, seed=seed, replica=r, t_eq=10, t_s=25, k_spring=3.0)[1]
           for r, (lat, n, Tk, seed) in enumerate(systems)]
    boxes = [O.create_crystal(lat, lat_a(lat), n, n, n)[1] for (lat, n, Tk, seed) in systems]
    X0 = T(np.concatenate(x0s))
    x2, v2 = X0.clone(), T(np.concatenate(vs))
    W2 = torch.zeros((len(systems), 2), dtype=torch.float64, device=DEV)
    for m in mgs:
        m.skin = 1.5
    ne.ne_switch_run_segment(ctx, mgs, list(offs), x2, v2, X0, boxes, W2, 0, 60)
    assert torch.abs(x - x2).max().item() < 2e-5
    assert torch.allclose(Wd, W2, rtol=1e-5, atol=1e-4)


def test_cluster_size_changes_rounding_only(ctx):
    """The same batch on clusters of 3 (the fewest CTAs that hold 1024
    atoms), 5 and 16 CTAs and on the size chosen from the device's cluster
    occupancy: the CTA sums regroup, nothing else changes."""
    systems = [(O.BCC, 8, 1000.0, 3), (O.BCC, 8, 1000.0, 4)]
    out = []
    try:
        for C in (0, 3, 5, 16):
            ne.ne_ctx_set_cluster_size(ctx, C)
            x, v, Wd, _, _ = run_crystals(ctx, systems, 0, 100)
            out.append((x, Wd))
        ne.ne_ctx_set_cluster_size(ctx, 2)
        with pytest.raises(ne.NeError, match="NE_EINVAL"):
            run_crystals(ctx, systems, 0, 10)
    finally:
        ne.ne_ctx_set_cluster_size(ctx, 0)
    for x, Wd in out[1:]:
        assert torch.abs(x - out[0][0]).max().item() < 2e-5
        assert torch.allclose(Wd, out[0][1], rtol=1e-5, atol=1e-4)
    with pytest.raises(ne.NeError, match="NE_EINVAL"):
        ne.ne_ctx_set_cluster_size(ctx, 17)


def test_free_energy_estimators_and_convergence_workflow(ctx, pot):
    """Two-sided FL estimate and the one-sided Jarzynski estimates from the
    same works agree to within the dissipation; dissipation falls with the
    switching time (Sec. III.B); and every F(t_s) point, with its Jarzynski
    estimates and dissipation, equals the one assembled from the oracle's
    runs of the same seeds (Philox replica indices 0-3) to 1e-5 eV/atom."""
    from paper_2201_04622_gb300 import workflow as WF
    seeds, t_s_list = [1, 2, 3, 4], [500, 2000]
    rows = WF.fl_convergence(ctx, O.BCC, W.A_BCC, 5, 800.0, MASS, 2.8, t_s_list, seeds, 300, runner="crystal")
    p, th = pot
    x0, box = O.create_crystal(O.BCC, W.A_BCC, 5, 5, 5)
    for r, ts in zip(rows, t_s_list):
        wf, wb = [], []
        for q, seed in enumerate(seeds):
            mo = O.md(mass=MASS, T=800.0, k_spring=2.8, t_eq=300, t_s=ts, seed=seed, replica=q, fix_cm=1)
            ro = O.switch_run(p, th, mo, x0, O.init_velocities(mo, len(x0)), x0, box)
            wf.append(ro["W_f"])
            wb.append(ro["W_b"])
        fo = WF.fl_free_energies(O.BCC, W.A_BCC, 5, 800.0, MASS, 2.8, wf, wb)
        for key in ("F", "F_jarzynski_fwd", "F_jarzynski_bwd", "Ediss"):
            assert abs(r[key] - fo[key]) < 1e-5, (ts, key)
    for r in rows:
        tol = 3 * abs(r["Ediss"]) + 6 * r["stderr"] + 1e-4
        assert abs(r["F_jarzynski_fwd"] - r["F"]) < tol
        assert abs(r["F_jarzynski_bwd"] - r["F"]) < tol
    assert rows[1]["Ediss"] < rows[0]["Ediss"]
    assert abs(rows[1]["F"] - rows[0]["F"]) < 5 * (rows[0]["stderr"] + rows[1]["stderr"]) + 2 * rows[0]["Ediss"]


def test_size_scaling_workflow_against_the_oracle():
    """The finite-size study of Sec. IV.A from 250 to 11,664 atoms (bcc 5^3
    .. 18^3, the paper's size) in one batch, four seeds each at 1000 K: a
    batch with cells above 4096 atoms (14^3, 18^3) runs on the brick runner
    (the multi-kernel path takes them only if the batch's CTAs do not fit
    the device at once).  The two smallest sizes equal the
    oracle's stored runs (tests/golden/size_scaling_works.json, same seeds
    and Philox replica indices): every work within 1e-6 eV per atom and F
    within 1 meV/atom; the larger cells give finite F and the 1/N fit."""
    import json
    import os
    from paper_2201_04622_gb300 import workflow as WF
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "size_scaling_works.json")))
    sizes = g["sizes"]
    cells = [s["cells"] for s in sizes] + [10, 14, 18]
    big = ne.ne_ctx_create(ne.eam_params(**W.EAM_FE_LIKE), 90000, 32)
    try:
        rows, (F_inf, slope) = WF.size_scaling(big, O.BCC, g["a"], cells, g["T"], MASS, g["k"], g["seeds"],
                                               g["t_eq"], g["t_s"], runner="auto", chunk=3000)
    finally:
        ne.ne_ctx_destroy(big)
    assert [r["atoms"] for r in rows] == [2 * c ** 3 for c in cells]
    for q, ref in enumerate(sizes):
        r = rows[q]
        want = [w for w in g["rows"] if w["cells"] == ref["cells"]]
        assert np.abs(np.array(r["W_f"]) - [w["W_f"] for w in want]).max() / r["atoms"] < 1e-6
        assert np.abs(np.array(r["W_b"]) - [w["W_b"] for w in want]).max() / r["atoms"] < 1e-6
        assert abs(r["F"] - ref["F_per_atom"]) < 1e-3
    assert all(np.isfinite([r["F"] for r in rows])) and np.isfinite(F_inf) and np.isfinite(slope)
    # F(N) flattens with size: the largest cells agree within their error bars
    assert abs(rows[-1]["F"] - rows[-2]["F"]) < 4 * (rows[-1]["stderr"] + rows[-2]["stderr"]) + 1e-3


def test_crystal_runner_reports_atoms_beyond_the_stencil_range(ctx):
    """Three bcc 6^3 replicas; the middle one starts with an atom 2.2 A from
    its site (D = 2 A; along [110], 1.45 A from its nearest neighbours, far
    from overlap): NE_ERANGE, and ne_ctx_replica_status names that replica
    alone; it keeps its x, v and W of the first step while the other two are
    advanced.  The same start 1.8 A out runs."""
    mo, mg = md_pair(T=300.0)
    x0, box = O.create_crystal(O.BCC, W.A_BCC, 6, 6, 6)
    mgs = [md_pair(T=300.0, replica=r)[1] for r in range(3)]
    crs = [(O.BCC, W.A_BCC, 6, 6, 6)] * 3
    for shift, ok in ((2.2, False), (1.8, True)):
        x = np.concatenate([x0] * 3)
        x[len(x0), :2] += shift / np.sqrt(2.0)
        xt, vt = T(x), T(np.zeros_like(x))
        Wd = torch.full((3, 2), 1.5, dtype=torch.float64, device=DEV)
        if ok:
            ne.ne_crystal_run_segment(ctx, mgs, crs, xt, vt, Wd, 0, 10)
            assert list(ne.ne_ctx_replica_status(ctx, 3)) == [ne.NE_OK] * 3
        else:
            xin, vin = xt.clone(), vt.clone()
            with pytest.raises(ne.NeError, match="NE_ERANGE"):
                ne.ne_crystal_run_segment(ctx, mgs, crs, xt, vt, Wd, 0, 10)
            assert list(ne.ne_ctx_replica_status(ctx, 3)) == [ne.NE_OK, ne.NE_ERANGE, ne.NE_OK]
            n1 = len(x0)
            assert torch.equal(xt[n1:2 * n1], xin[n1:2 * n1]) and torch.equal(vt[n1:2 * n1], vin[n1:2 * n1])
            assert Wd[1].tolist() == [1.5, 1.5]
            assert not torch.equal(xt[:n1], xin[:n1]) and not torch.equal(xt[2 * n1:], xin[2 * n1:])


@pytest.mark.parametrize("lat,n", [(O.BCC, 5), (O.FCC, 4)])
def test_crystal_runner_small_hot_boxes_track_oracle(ctx, pot, lat, n):
    """bcc 5^3 and fcc 4^3 (L ~ 14.5 A < 2 (r_c + 2D)): the stencil holds two
    periodic images of some sites.  At 1400 K over 100 steps the runner
    follows the FP64 oracle as closely as on large boxes."""
    p, th = pot
    x, v, Wd, x0s, vs = run_crystals(ctx, [(lat, n, 1400.0, 7)], 0, 100, k_spring=2.5)
    mo, _ = md_pair(T=1400.0, seed=7, replica=0, k_spring=2.5)
    x0, box = O.create_crystal(lat, lat_a(lat), n, n, n)
    ro = O.switch_run(p, th, mo, x0, vs[0], x0, box)
    assert np.abs(x.cpu().numpy() - ro["x"]).max() < 2e-4
    Wg = Wd.cpu().numpy()[0]
    assert Wg[0] == pytest.approx(ro["W_f"], rel=1e-5, abs=1e-3)
    assert Wg[1] == pytest.approx(ro["W_b"], rel=1e-5, abs=1e-3)


def test_auto_runner_moves_out_of_range_replicas_to_the_multikernel_path(ctx, monkeypatch):
    """fl_batch(runner='auto') on the BatchAdvancer, chunks of 40 steps: when
    the crystal runner reports NE_ERANGE for replica 1 in the second chunk (a
    stand-in raises it after the real call and ne_ctx_replica_status names
    replica 1, since a crystal that stays solid never leaves the range),
    replica 1 goes back to its state before that chunk and continues on the
    multi-kernel mixed path (second context, concurrent with the crystal
    runner for the others).  With the cluster size fixed, replicas 0 and 2
    equal a plain crystal-runner run bit for bit, and replica 1 equals 40
    crystal-runner steps followed by the multi-kernel path to rounding."""
    from paper_2201_04622_gb300 import workflow as WF
    real = ne.ne_crystal_run_segment
    calls = []

    def fake(c, mds, crs, x, v, W, s0, ns, stream=None):
        n_rep = mds.n_rep if isinstance(mds, ne.CrystalBatch) else len(mds)
        fail = s0 == 40 and n_rep == 3
        if fail:  # the runner's contract: a replica that raised keeps its state of s0
            keep = (x[432:864].clone(), v[432:864].clone(), W[1].clone())
        real(c, mds, crs, x, v, W, s0, ns, stream=stream)
        calls.append((s0, n_rep))
        if fail:
            x[432:864], v[432:864], W[1] = keep
            raise ne.NeError(ne.NE_ERANGE, "ne_crystal_run_segment", "stand-in")

    crystals = [(O.BCC, W.A_BCC, 6)] * 3
    args = (ctx, crystals, 1400.0, [2.38] * 3, [1, 2, 3], 20, 40, MASS)
    ne.ne_ctx_set_cluster_size(ctx, 2)
    try:
        monkeypatch.setattr(ne, "ne_crystal_run_segment", fake)
        monkeypatch.setattr(ne, "ne_ctx_replica_status",
                            lambda c, n: np.array([ne.NE_OK, ne.NE_ERANGE, ne.NE_OK][:n], dtype=np.int32))
        with pytest.warns(UserWarning):
            Wf, Wb, x = WF.fl_batch(*args, runner="auto", skin=1.0, chunk=40)
        monkeypatch.undo()
        assert calls == [(0, 3), (40, 3), (80, 2)]
        # reference: the crystal runner for all three, in one call
        Wc, Wbc, xc = WF.fl_batch(*args, runner="crystal")
        # reference for replica 1: 40 crystal-runner steps, then the multi-kernel path
        mass = MASS
        mds, crs, x0s, offs = [], [], [], [0]
        for r, (lat, a, n) in enumerate(crystals):
            mds.append(ne.md_params(T=1400.0, mass=mass, k_spring=2.38, skin=1.0, prec=ne.NE_MIXED, t_eq=20,
                                    t_s=40, seed=r + 1, replica=r, fix_cm=1))
            x0, box = WF.crystal_sites(lat, a, n)
            x0s.append(x0)
            crs.append((lat, a, n, n, n))
            offs.append(offs[-1] + len(x0))
        X0 = T(np.concatenate(x0s))
        xr, vr = X0.clone(), torch.zeros_like(X0)
        for r, m in enumerate(mds):
            ne.ne_init_velocities(ctx, m, vr[offs[r]:offs[r + 1]])
        Wr = torch.zeros((3, 2), dtype=torch.float64, device=DEV)
        ne.ne_crystal_run_segment(ctx, mds, crs, xr, vr, Wr, 0, 40)
        a1, b1 = offs[1], offs[2]
        x1, v1, W1 = xr[a1:b1].clone(), vr[a1:b1].clone(), Wr[1:2].clone()
        ne.ne_switch_run_segment(ctx, [mds[1]], [0, b1 - a1], x1, v1, X0[a1:b1].contiguous(),
                                 [WF.crystal_sites(*crystals[1])[1]], W1, 40, 80)
    finally:
        ne.ne_ctx_set_cluster_size(ctx, 0)
    assert Wf[0] == Wc[0] and Wf[2] == Wc[2] and Wb[0] == Wbc[0] and Wb[2] == Wbc[2]
    assert torch.equal(x[:a1], xc[:a1]) and torch.equal(x[b1:], xc[b1:])
    # the multi-kernel path resumes bit for bit only while no atom has strayed
    # skin/2 from its site (its list is rebuilt from positions after that), so
    # replica 1 (split at step 80 there, not in the reference) agrees to rounding
    assert abs(Wf[1] - float(W1[0, 0])) < 1e-6 * (b1 - a1) and abs(Wb[1] - float(W1[0, 1])) < 1e-6 * (b1 - a1)
    assert float((x[a1:b1] - x1).abs().max()) < 1e-5


def test_fl1400_full_length_works_vs_oracle(ctx):
    """The 1400 K batch (10 x bcc 10^3 + 10 x fcc 8^3) at full length
    (t_eq 10 ps, t_s 50 ps, 120,000 steps per replica) in the crystal
    runner's benchmark launch configuration: the forward and backward works
    of the eight replicas stored from the FP64 oracle
    (tests/golden/fl1400_works.json, same seeds and replica indices).  With
    the same Philox noise and 0.1 ps damping the mixed and FP64 trajectories
    stay synchronised, so each work agrees to FP32 pair-energy rounding:
    |U|/N ~ 4.3 eV carries 2^-24 * 4.3 ~ 2.6e-7 eV per atom of systematic
    rounding, and the test allows 1e-6 eV per atom (1 ueV/atom in F)."""
    import json
    import os
    from paper_2201_04622_gb300 import workflow as WF
    with open(os.path.join(os.path.dirname(__file__), "golden", "fl1400_works.json")) as f:
        doc = json.load(f)
    crystals = [(O.BCC, W.A_BCC, 10)] * 10 + [(O.FCC, W.A_FCC, 8)] * 10
    ks = [W.K_BCC_1400] * 10 + [W.K_FCC_1400] * 10
    seeds = list(range(1, 11)) * 2
    Wf, Wb, _ = WF.fl_batch(ctx, crystals, doc["T"], ks, seeds, doc["t_eq"], doc["t_s"], MASS,
                            prec=ne.NE_MIXED, runner="crystal", chunk=20000)
    assert len(doc["rows"]) == 8
    for row in doc["rows"]:
        q = row["replica"]
        lat, a, n = crystals[q]
        assert (lat, a, n, ks[q], seeds[q]) == (row["lattice"], row["a"], row["n"], row["k"], row["seed"])
        tol = 1e-6 * row["natoms"]
        assert abs(Wf[q] - row["W_f"]) < tol, (q, Wf[q], row["W_f"])
        assert abs(Wb[q] - row["W_b"]) < tol, (q, Wb[q], row["W_b"])
        dF = 0.5 * ((Wf[q] - row["W_f"]) - (Wb[q] - row["W_b"])) / row["natoms"]
        assert abs(dF) < 1e-6


@pytest.mark.parametrize("set_name", ["rs_bcc6", "fl_hcp6"])
def test_runner_rs_and_hcp_full_length_works_vs_oracle(ctx, set_name):
    """The crystal runner's other paths at lengths where the trajectories have
    long decorrelated from their start (22,000 steps): reversible scaling on
    bcc 6^3 from 300 to 1200 K, and Frenkel-Ladd on ideal hcp 6^3 at 1000 K.
    Forward and backward works equal the stored FP64 oracle works
    (tests/golden/runner_paths_works.json, same seeds and replica indices) to
    the FP32 pair-energy rounding bound of the 1400 K test, 1e-6 eV per atom."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "runner_paths_works.json")) as f:
        doc = json.load(f)
    rows = [r for r in doc["rows"] if r["set"] == set_name]
    assert len(rows) == 2
    mgs, crs, x0s, vs = [], [], [], []
    for r in rows:
        m = ne.md_params(dt=1e-3, T=r["T"], damp=0.1, mass=MASS, k_spring=r["k"], skin=1.0, lambda_fn=2,
                         path=r["path"], t_eq=doc["t_eq"], t_s=doc["t_s"], lambda_f=r["lambda_f"],
                         seed=r["seed"], replica=r["replica"], fix_cm=1, prec=ne.NE_MIXED)
        x0, box = O.create_crystal(r["lattice"], r["a"], r["n"], r["n"], r["n"])
        v = torch.zeros((len(x0), 3), dtype=torch.float64, device=DEV)
        ne.ne_init_velocities(ctx, m, v)
        mgs.append(m)
        crs.append((r["lattice"], r["a"], r["n"], r["n"], r["n"]))
        x0s.append(x0)
        vs.append(v)
    x, v = T(np.concatenate(x0s)), torch.cat(vs)
    Wd = torch.zeros((len(rows), 2), dtype=torch.float64, device=DEV)
    ne.ne_crystal_run_segment(ctx, mgs, crs, x, v, Wd, 0, 2 * doc["t_eq"] + 2 * doc["t_s"])
    Wg = Wd.cpu().numpy()
    for q, r in enumerate(rows):
        tol = 1e-6 * r["natoms"]
        assert abs(Wg[q, 0] - r["W_f"]) < tol, (set_name, q, Wg[q, 0], r["W_f"])
        assert abs(Wg[q, 1] - r["W_b"]) < tol, (set_name, q, Wg[q, 1], r["W_b"])


def test_crystal_runner_cumulative_works_track_oracle(ctx, pot):
    """Reversible scaling (Sec. III.C, eq. rs) in the crystal runner with the
    cumulative works of both switches (ne_crystal_run_segment_cum, cut into
    two segments inside the forward switch): equal to the oracle's cumulative
    works over 100 steps to the tolerance of the 100-step tracking test, and
    the last entries equal the totals."""
    p, th = pot
    mo, mg = md_pair(T=300.0, seed=5, replica=0, path=O.PATH_RS)
    x0, box = O.create_crystal(O.BCC, W.A_BCC, 6, 6, 6)
    v0 = O.init_velocities(mo, len(x0))
    ro = O.switch_run(p, th, mo, x0, v0, x0, box, cumulative=True)
    x, v = T(x0), T(v0)
    Wd = torch.zeros((1, 2), dtype=torch.float64, device=DEV)
    t_s = mg.t_s
    Wc = torch.zeros(2 * (t_s + 1), dtype=torch.float64, device=DEV)
    S = 2 * mg.t_eq + 2 * t_s
    cut = mg.t_eq + 7
    crs = [(O.BCC, W.A_BCC, 6, 6, 6)]
    ne.ne_crystal_run_segment_cum(ctx, [mg], crs, x, v, Wd, Wc, 0, cut)
    ne.ne_crystal_run_segment_cum(ctx, [mg], crs, x, v, Wd, Wc, cut, S - cut)
    wc = Wc.cpu().numpy().reshape(2, t_s + 1)
    assert np.allclose(wc[0], ro["Wcum_f"], rtol=1e-5, atol=1e-4)
    assert np.allclose(wc[1], ro["Wcum_b"], rtol=1e-5, atol=1e-4)
    assert wc[0, -1] == float(Wd[0, 0]) and wc[1, -1] == float(Wd[0, 1])
    assert np.abs(x.cpu().numpy() - ro["x"]).max() < 2e-5


def test_rs_batch_on_the_crystal_runner_matches_the_multikernel_path(ctx):
    """eq. rs from workflow.rs_batch (crystal runner, cumulative works of two
    seeds in one batch) against workflow.rs_works (multi-kernel mixed path, the
    same seeds and noise streams): F(T) on a 300-600 K grid agrees to 1e-5 eV
    per atom (the trajectories stay synchronised over 4,400 steps)."""
    from paper_2201_04622_gb300 import workflow as WF
    lam_f, t_eq, t_s, T0 = 0.5, 200, 2000, 300.0
    cf, cb, _ = WF.rs_batch(ctx, [(O.BCC, W.A_BCC, 6)] * 2, T0, [1, 2], lam_f, t_eq, t_s, MASS, replica_ids=[0, 0])
    gf, gb, _ = WF.rs_works(ctx, O.BCC, W.A_BCC, 6, T0, MASS, lam_f, t_eq, t_s, [1, 2])
    grid = np.linspace(300.0, 600.0, 7)
    Fc = WF.rs_free_energy(O.BCC, W.A_BCC, 6, T0, -4.2, lam_f, t_s, cf, cb, grid)
    Fg = WF.rs_free_energy(O.BCC, W.A_BCC, 6, T0, -4.2, lam_f, t_s, gf, gb, grid)
    assert np.abs(np.asarray(Fc) - np.asarray(Fg)).max() < 1e-5


def test_uneven_campaign_fits_one_spring_per_replica():
    """The uneven-batch workload with one spring per replica at its own size
    and temperature (eq. msd in one batched fit): each batched spring equals
    the single-replica fit of the same replica (FP64 path, same noise), the
    springs stiffen as T falls, and the campaign gives a finite F for every
    replica."""
    from paper_2201_04622_gb300 import workflow as WF
    reps = [r for r in W.batched_replicas(64, seed=1) if r["n"] <= 7][:5]
    big = ne.ne_ctx_create(ne.eam_params(**W.EAM_FE_LIKE), 20000, 8)
    try:
        crystals = [(r["lattice"], W.A_BCC if r["lattice"] == W.BCC else W.A_FCC, r["n"]) for r in reps]
        Ts = [r["T"] for r in reps]
        fit = dict(n_eq=200, n_samples=40, stride=5)
        k, msd = WF.fit_spring_constants(big, crystals, Ts, MASS, prec=ne.NE_FP64,
                                         replica_ids=[r["replica"] for r in reps], **fit)
        for q, ((lat, a, n), Tr) in enumerate(zip(crystals, Ts)):
            x0_np, box = WF.crystal_sites(lat, a, n)
            md = ne.md_params(T=Tr, mass=MASS, skin=1.0, prec=ne.NE_FP64, seed=1, replica=reps[q]["replica"],
                              fix_cm=1)
            x0 = torch.tensor(x0_np, dtype=torch.float64, device=DEV)
            x, v = x0.clone(), torch.zeros_like(x0)
            ne.ne_init_velocities(big, md, v)
            m1, k1 = ne.ne_msd_fit(big, md, x, v, x0, box, fit["n_eq"], fit["n_samples"], fit["stride"])
            assert k[q] == pytest.approx(k1, rel=1e-9) and msd[q] == pytest.approx(m1, rel=1e-9)
        order = np.argsort(Ts)
        assert k[order[0]] > k[order[-1]]  # colder replicas are stiffer
        rows = WF.uneven_campaign(big, reps, MASS, 100, 300, fit=fit, chunk=400)
        assert len(rows) == len(reps) and all(np.isfinite(r["F"]) for r in rows)
    finally:
        ne.ne_ctx_destroy(big)


@pytest.mark.parametrize("runner", [1, 2], ids=["cluster", "brick"])
def test_runner_pairs_past_the_tmem_visits(ctx, pot, runner):
    """The cluster runner keeps the neighbour slot and f'(r)/r of 56 stencil
    visits a thread in tensor memory, the brick runner f'(r)/r of 80; later
    visits take their neighbour from the wrapped-cell tables and are
    recomputed in pass 2.  Two atoms of the (2,2,0)a shell of bcc (stencil
    entries 168-179: visits 84-89 at 2 threads per atom), each moved 1.55 A
    towards the other (within the 2 A range), are 5.02 A apart: inside r_c,
    with their embedding force from that recomputation.  10 steps at 10 K
    against the oracle."""
    p, th = pot
    x0, box = O.create_crystal(O.BCC, W.A_BCC, 6, 6, 6)
    tgt = x0[0] + W.A_BCC * np.array([2.0, 2.0, 0.0])
    j = int(np.argmin(np.linalg.norm(x0 - tgt, axis=1)))
    nrm = np.array([1.0, 1.0, 0.0]) / np.sqrt(2.0)
    xs = x0.copy()
    xs[0] += 1.55 * nrm
    xs[j] -= 1.55 * nrm
    mo, mg = md_pair(T=10.0, t_eq=2, t_s=3, k_spring=3.0, seed=3, replica=0)
    v0 = O.init_velocities(mo, len(x0))
    ro = O.switch_run(p, th, mo, xs, v0, x0, box)
    ne.ne_ctx_set_runner(ctx, runner)
    try:
        x, v = T(xs), T(v0)
        Wd = torch.zeros((1, 2), dtype=torch.float64, device=DEV)
        ne.ne_crystal_run_segment(ctx, [mg], [(O.BCC, W.A_BCC, 6, 6, 6)], x, v, Wd, 0, 10)
        plan = ne.ne_ctx_crystal_plan(ctx)
    finally:
        ne.ne_ctx_set_runner(ctx, 0)
    assert plan["runner"] == ("cluster" if runner == 1 else "brick")
    if runner == 1:  # 432 atoms: two CTAs of 384 slots, two threads per atom
        assert plan["threads_per_atom"] == 2 and plan["cluster_ctas"] >= 2 and plan["ctas"] == plan["cluster_ctas"]
    assert np.abs(x.cpu().numpy() - ro["x"]).max() < 2e-5
    assert np.abs(v.cpu().numpy() - ro["v"]).max() < 1e-3  # that force alone changes v by ~4e-3 A/ps a step
    assert float(Wd[0, 0]) == pytest.approx(ro["W_f"], rel=1e-5)
    assert float(Wd[0, 1]) == pytest.approx(ro["W_b"], rel=1e-5)
