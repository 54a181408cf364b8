"""The brick runner (ne_ctx_set_runner 2, and automatically for replicas
above 4096 atoms): every CTA owns a block of cells of one replica and the
CTAs exchange displacements and F'(rho) through global memory between grid
barriers.  Against the oracle (FP64) on small cells at 1400 K and on a
config-4-sized bcc 16^3 cell, against the cluster runner on the same batch,
with one threads-per-atom choice per batch size (8, 4, 3, 2 or 1), species tables,
the cumulative works of eq. rs, a replica that leaves the stencil range, and
segment resume.  The reversible-scaling prefix of bcc 16^3 against the stored
oracle works is in test_zz_workloads_vs_oracle.py."""
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
MASS = W.MASS_FE_AMU / 9648.5332


@pytest.fixture(scope="module")
def pot():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    p = O.eam(**W.EAM_FE_LIKE)
    return p, O.eam_theta(p)


@pytest.fixture(scope="module")
def ctx():
    c = ne.ne_ctx_create(ne.eam_params(**W.EAM_FE_LIKE), 70000, 64)
    yield c
    ne.ne_ctx_destroy(c)


def T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device=DEV)


def lat_a(lat):
    return W.A_BCC if lat == O.BCC else (W.A_FCC if lat == O.FCC else W.A_HCP)


def md_pair(**kw):
    base = dict(dt=1e-3, T=300.0, damp=0.1, k_spring=6.0, lambda_fn=2, t_eq=20, t_s=30, lambda_f=0.5, seed=11,
                replica=2, fix_cm=1)
    base.update(kw)
    path = base.pop("path", O.PATH_FL)
    mo = O.md(mass=MASS, path=path, **base)
    mg = ne.md_params(mass=MASS, skin=1.0, prec=ne.NE_MIXED, path=path, **base)
    return mo, mg


def batch(systems, **kw):
    mgs, mos, crs, x0s, vs = [], [], [], [], []
    for r, (lat, n, Tk, seed) in enumerate(systems):
        mo, mg = md_pair(T=Tk, seed=seed, replica=r, **kw)
        x0, box = O.create_crystal(lat, lat_a(lat), n, n, n)
        mos.append(mo)
        mgs.append(mg)
        x0s.append(x0)
        vs.append(O.init_velocities(mo, len(x0)))
        crs.append((lat, lat_a(lat), n, n, n))
    return mgs, mos, crs, x0s, vs


def run(ctx, runner, mgs, crs, x0s, vs, s0, ns, x=None, v=None, Wd=None, cum=False):
    ne.ne_ctx_set_runner(ctx, runner)
    try:
        if x is None:
            x, v = T(np.concatenate(x0s)), T(np.concatenate(vs))
            Wd = torch.zeros((len(mgs), 2), dtype=torch.float64, device=DEV)
        if cum:
            Wc = torch.zeros(len(mgs) * 2 * (mgs[0].t_s + 1), dtype=torch.float64, device=DEV)
            ne.ne_crystal_run_segment_cum(ctx, mgs, crs, x, v, Wd, Wc, s0, ns)
            return x, v, Wd, Wc
        ne.ne_crystal_run_segment(ctx, mgs, crs, x, v, Wd, s0, ns)
        return x, v, Wd
    finally:
        ne.ne_ctx_set_runner(ctx, 0)


@pytest.mark.parametrize("lat,n,path", [(O.BCC, 5, O.PATH_FL), (O.FCC, 4, O.PATH_FL), (O.BCC, 6, O.PATH_RS),
                                        (O.HCP, 5, O.PATH_FL)])
def test_brick_runner_tracks_oracle_100_steps(ctx, pot, lat, n, path):
    p, th = pot
    mgs, mos, crs, x0s, vs = batch([(lat, n, 1400.0 if path == O.PATH_FL else 300.0, 5)], path=path,
                                   k_spring=2.5)
    x, v, Wd = run(ctx, 2, mgs, crs, x0s, vs, 0, 100)
    box = O.create_crystal(lat, lat_a(lat), n, n, n)[1]
    ro = O.switch_run(p, th, mos[0], x0s[0], vs[0], x0s[0], box)
    assert np.abs(x.cpu().numpy() - ro["x"]).max() < 2e-4
    Wg = Wd.cpu().numpy()[0]
    assert Wg[0] == pytest.approx(ro["W_f"], rel=1e-5, abs=1e-3)
    assert Wg[1] == pytest.approx(ro["W_b"], rel=1e-5, abs=1e-3)


def test_brick_runner_matches_the_cluster_runner(ctx):
    """An uneven batch (threads per atom 8 or 4 for it) on both runners:
    the same trajectories to the rounding of the replica sums."""
    systems = [(O.BCC, 6, 800.0, 3), (O.FCC, 5, 1200.0, 4), (O.BCC, 8, 400.0, 9), (O.FCC, 6, 300.0, 2)]
    mgs, mos, crs, x0s, vs = batch(systems)
    xb, vb, Wb = run(ctx, 2, mgs, crs, x0s, vs, 0, 100)
    xc, vc, Wc = run(ctx, 1, mgs, crs, x0s, vs, 0, 100)
    assert torch.abs(xb - xc).max().item() < 2e-5
    assert torch.allclose(Wb, Wc, rtol=1e-5, atol=1e-4)


def test_brick_runner_two_threads_per_atom_matches_the_cluster_runner(ctx):
    """The 20-replica benchmark batch (10 x bcc 10^3 + 10 x fcc 8^3 at
    1400 K) forced onto the brick runner: 3 threads per atom would need 160
    CTAs on a 152-SM device, so it takes 2 (120 CTAs; 24 neighbour indices a
    thread in tensor memory beside 56 visits of f'(r)/r); the 100-step
    schedule against the cluster runner on the same batch."""
    systems = [(O.BCC, 10, 1400.0, s) for s in range(1, 11)] + [(O.FCC, 8, 1400.0, s) for s in range(11, 21)]
    mgs, mos, crs, x0s, vs = batch(systems, k_spring=2.4)
    xb, vb, Wb = run(ctx, 2, mgs, crs, x0s, vs, 0, 100)
    plan = ne.ne_ctx_crystal_plan(ctx)
    xc, vc, Wc = run(ctx, 1, mgs, crs, x0s, vs, 0, 100)
    assert plan["runner"] == "brick"
    sms = torch.cuda.get_device_properties(DEV).multi_processor_count
    if 120 <= sms < 160:
        assert plan["threads_per_atom"] == 2 and plan["ctas"] == 120
    assert torch.abs(xb - xc).max().item() < 2e-5
    assert torch.allclose(Wb, Wc, rtol=1e-5, atol=1e-4)


def test_brick_runner_large_replica_against_oracle(ctx, pot):
    """bcc 16^3 (8192 atoms, the reversible-scaling cell): too large for a
    cluster, so the default setting runs it on the brick runner; 60 steps
    of the FL schedule at 1400 K against the oracle, atom by atom."""
    p, th = pot
    mgs, mos, crs, x0s, vs = batch([(O.BCC, 16, 1400.0, 7)], t_eq=10, t_s=20, k_spring=2.4)
    x, v, Wd = run(ctx, 0, mgs, crs, x0s, vs, 0, 60)
    box = O.create_crystal(O.BCC, W.A_BCC, 16, 16, 16)[1]
    ro = O.switch_run(p, th, mos[0], x0s[0], vs[0], x0s[0], box)
    assert np.abs(x.cpu().numpy() - ro["x"]).max() < 2e-4
    Wg = Wd.cpu().numpy()[0]
    assert Wg[0] == pytest.approx(ro["W_f"], rel=1e-5, abs=1e-2)
    assert Wg[1] == pytest.approx(ro["W_b"], rel=1e-5, abs=1e-2)


def test_brick_runner_one_thread_per_atom_on_bcc32(ctx, pot):
    """bcc 32^3 (65,536 atoms, the gradient workload's cell): 2 threads per
    atom would need 171 CTAs, more than the device holds, so the brick
    runner takes 1 thread per atom (86 CTAs of 768 atoms); 10 steps of the
    FL schedule at 300 K against the oracle, atom by atom."""
    p, th = pot
    mgs, mos, crs, x0s, vs = batch([(O.BCC, 32, 300.0, 7)], t_eq=3, t_s=2, k_spring=4.0)
    x, v, Wd = run(ctx, 0, mgs, crs, x0s, vs, 0, 10)
    box = O.create_crystal(O.BCC, W.A_BCC, 32, 32, 32)[1]
    ro = O.switch_run(p, th, mos[0], x0s[0], vs[0], x0s[0], box)
    assert np.abs(x.cpu().numpy() - ro["x"]).max() < 2e-5
    dv = np.abs(v.cpu().numpy() - ro["v"])
    # the runners draw their normals with an FP32 Box-Muller: among 2e6
    # draws the extreme tails differ from the oracle's FP64 ones enough to
    # move a velocity by a few 1e-3 A/ps through c2 ~ 0.3 A/ps (2.6e-3 seen);
    # the bulk agrees to ~1e-7
    assert np.median(dv) < 1e-6 and dv.max() < 1e-2
    Wg = Wd.cpu().numpy()[0]
    assert Wg[0] == pytest.approx(ro["W_f"], rel=1e-6)
    assert Wg[1] == pytest.approx(ro["W_b"], rel=1e-6)


def test_brick_runner_three_threads_per_atom_on_four_bcc16(ctx, pot):
    """Four bcc 16^3 replicas (32,768 atoms, the reversible-scaling bench
    batch): 4 threads per atom would need 172 CTAs, more than a 152-SM device
    holds, so the brick runner takes 3 (128 CTAs of 256 atoms), as
    ne_ctx_crystal_plan reports; the 60-step FL schedule at 1400 K,
    replica 2 against the oracle atom by atom."""
    p, th = pot
    mgs, mos, crs, x0s, vs = batch([(O.BCC, 16, 1400.0, s) for s in (3, 5, 7, 9)], t_eq=10, t_s=20,
                                   k_spring=2.4)
    x, v, Wd = run(ctx, 0, mgs, crs, x0s, vs, 0, 60)
    plan = ne.ne_ctx_crystal_plan(ctx)
    assert plan["runner"] == "brick" and plan["cluster_ctas"] == 0
    sms = torch.cuda.get_device_properties(DEV).multi_processor_count
    if 128 <= sms < 172:
        assert plan["threads_per_atom"] == 3 and plan["ctas"] == 128
    q, n = 2, len(x0s[0])
    box = O.create_crystal(O.BCC, W.A_BCC, 16, 16, 16)[1]
    ro = O.switch_run(p, th, mos[q], x0s[q], vs[q], x0s[q], box)
    assert np.abs(x.cpu().numpy()[q * n:(q + 1) * n] - ro["x"]).max() < 2e-4
    Wg = Wd.cpu().numpy()[q]
    assert Wg[0] == pytest.approx(ro["W_f"], rel=1e-5, abs=1e-2)
    assert Wg[1] == pytest.approx(ro["W_b"], rel=1e-5, abs=1e-2)


def test_brick_runner_cumulative_works_resume_and_species(ctx, pot):
    """The cumulative works of eq. rs over two segments equal one call's
    (resume bit for bit: the plan and sums depend only on the batch), and a
    B2 replica with species tables follows the oracle."""
    p, th = pot
    mgs, mos, crs, x0s, vs = batch([(O.BCC, 6, 600.0, 3), (O.BCC, 7, 900.0, 4)], path=O.PATH_RS)
    S = 2 * mgs[0].t_eq + 2 * mgs[0].t_s
    x1, v1, W1, C1 = run(ctx, 2, mgs, crs, x0s, vs, 0, S, cum=True)
    x2, v2, W2, C2 = run(ctx, 2, mgs, crs, x0s, vs, 0, 37, cum=True)
    x2, v2, W2, C3 = run(ctx, 2, mgs, crs, x0s, vs, 37, S - 37, x=x2, v=v2, Wd=W2, cum=True)
    assert torch.equal(x1, x2) and torch.equal(W1, W2)
    assert torch.equal(C1.view(2, 2, -1)[:, :, 20:], C3.view(2, 2, -1)[:, :, 20:])
    # species: B2 bcc 5^3, masses 55.845 and 26.98 u
    x0, box = O.create_crystal(O.BCC, W.A_BCC, 5, 5, 5)
    sp = np.arange(len(x0)) % 2
    ms, ks = [55.845 / 9648.5332, 26.98 / 9648.5332], [4.2, 3.1]
    base = dict(dt=1e-3, T=600.0, damp=0.1, lambda_fn=2, t_eq=20, t_s=30, seed=5, replica=3, fix_cm=1)
    mo = O.md(mass=ms[0], k_spring=ks[0], species=sp, mass_s=ms, k_s=ks, **base)
    spt = torch.tensor(sp, dtype=torch.uint8, device=DEV)
    mg = ne.md_params(mass=ms[0], k_spring=ks[0], skin=1.0, prec=ne.NE_MIXED, species=spt, mass_s=ms, k_s=ks,
                      **base)
    v0 = O.init_velocities(mo, len(x0))
    ro = O.switch_run(p, th, mo, x0, v0, x0, box)
    x, v, Wd = run(ctx, 2, [mg], [(O.BCC, W.A_BCC, 5, 5, 5)], [x0], [v0], 0, 100)
    assert np.abs(x.cpu().numpy() - ro["x"]).max() < 2e-4
    assert float(Wd[0, 0]) == pytest.approx(ro["W_f"], rel=1e-5, abs=1e-3)


def test_brick_runner_replica_beyond_the_stencil_keeps_its_state(ctx):
    """Three bcc 6^3 replicas, the middle one with an atom 2.2 A from its site
    (D = 2 A): NE_ERANGE naming that replica alone; it keeps its state and
    work while the others advance."""
    x0, box = O.create_crystal(O.BCC, W.A_BCC, 6, 6, 6)
    mgs = [md_pair(T=300.0, replica=r)[1] for r in range(3)]
    crs = [(O.BCC, W.A_BCC, 6, 6, 6)] * 3
    x = np.concatenate([x0] * 3)
    x[len(x0), :2] += 2.2 / np.sqrt(2.0)
    xt, vt = T(x), T(np.zeros_like(x))
    Wd = torch.full((3, 2), 1.5, dtype=torch.float64, device=DEV)
    xin, vin = xt.clone(), vt.clone()
    ne.ne_ctx_set_runner(ctx, 2)
    try:
        with pytest.raises(ne.NeError, match="NE_ERANGE"):
            ne.ne_crystal_run_segment(ctx, mgs, crs, xt, vt, Wd, 0, 10)
        assert list(ne.ne_ctx_replica_status(ctx, 3)) == [ne.NE_OK, ne.NE_ERANGE, ne.NE_OK]
    finally:
        ne.ne_ctx_set_runner(ctx, 0)
    n1 = len(x0)
    assert torch.equal(xt[n1:2 * n1], xin[n1:2 * n1]) and Wd[1].tolist() == [1.5, 1.5]
    assert not torch.equal(xt[:n1], xin[:n1]) and not torch.equal(xt[2 * n1:], xin[2 * n1:])
