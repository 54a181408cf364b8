"""The barostat of the reversible-scaling path (Sec. III.C at P = 0; reading
A23) on the persistent crystal runners (the cluster runner, and the brick
runner whose CTAs exchange the virial through global memory behind a grid
barrier): the box and the lattice sites scale
with the overdamped Langevin step of ln V (isotropic) or of each ln L_a (per
axis, the paper's fix nph aniso), positions stay in fixed point about the
scaled sites.  Against the oracle's NPT_ISO and NPT_ANISO runs (same noise),
against the multi-kernel path, and across a segment boundary."""
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
NPT = dict(path=O.PATH_RS, T=300.0, t_eq=30, t_s=35, lambda_f=0.5, P0=0.0, beta_T=1.2, tau_p=0.05, damp=0.1,
           dt=1e-3, k_spring=1.0, lambda_fn=2, fix_cm=1, seed=11, replica=2)


@pytest.fixture(scope="module")
def pot():
    p = O.eam(**W.EAM_FE_LIKE)
    return p, O.eam_theta(p)


@pytest.fixture(scope="module")
def ctx():
    c = ne.ne_ctx_create(ne.eam_params(**W.EAM_FE_LIKE), 20000, 16)
    yield c
    ne.ne_ctx_destroy(c)


def T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device=DEV)


def pair(npt, **kw):
    base = dict(NPT, **kw)
    mo = O.md(mass=MASS, npt=npt, **base)
    mg = ne.md_params(mass=MASS, skin=1.0, prec=ne.NE_MIXED, npt=npt, **base)
    return mo, mg


@pytest.fixture(params=[1, 2], ids=["cluster", "brick"])
def runner(request, ctx):
    ne.ne_ctx_set_runner(ctx, request.param)
    yield request.param
    ne.ne_ctx_set_runner(ctx, 0)


@pytest.mark.parametrize("npt,lat,a,cells", [(1, O.BCC, 2.90, (5, 5, 5)), (2, O.HCP, W.A_HCP, (5, 3, 3))])
def test_runner_barostat_follows_the_oracle(ctx, pot, runner, npt, lat, a, cells):
    """bcc under tension (isotropic) and hcp at the ideal c/a (per axis), 130
    steps of the RS schedule on either runner: box, positions and works
    follow the oracle."""
    p, th = pot
    x0, box = O.create_crystal(lat, a, *cells)
    mo, mg = pair(npt)
    v0 = O.init_velocities(mo, len(x0))
    ro = O.switch_run(p, th, mo, x0, v0, x0, box)
    x, v = T(x0), T(v0)
    Wd = torch.zeros((1, 2), dtype=torch.float64, device=DEV)
    S = 2 * NPT["t_eq"] + 2 * NPT["t_s"]
    ne.ne_crystal_run_segment(ctx, [mg], [(lat, a) + cells], x, v, Wd, 0, S)
    bg = ne.ne_ctx_boxes(ctx, 1)[0]
    assert np.abs(np.asarray(bg) / box - 1.0).max() > 1e-3  # the box moved
    assert np.allclose(bg, ro["box"], rtol=2e-6, atol=0)
    assert np.abs(x.cpu().numpy() - ro["x"]).max() < 5e-5
    assert float(Wd[0, 0]) == pytest.approx(ro["W_f"], rel=1e-5, abs=1e-4)
    assert float(Wd[0, 1]) == pytest.approx(ro["W_b"], rel=1e-5, abs=1e-4)
    if npt == 2:  # hcp: the shape changed, not only the volume
        assert abs((bg[2] / bg[0]) / (box[2] / box[0]) - 1.0) > 1e-4


def test_runner_barostat_matches_the_multikernel_path_and_resumes(ctx, runner):
    """Two bcc replicas with the isotropic barostat: either runner and the
    mixed multi-kernel path agree; a run split in two segments, the second
    started at the lattice parameter the first reached (box / cells), gives
    the single call's state to rounding."""
    systems = [(O.BCC, 2.90, 5, 3), (O.BCC, 2.86, 6, 4)]
    mgs, x0s, vs, boxes, crs = [], [], [], [], []
    for r, (lat, a, n, seed) in enumerate(systems):
        mo, mg = pair(1, seed=seed, replica=r)
        x0, box = O.create_crystal(lat, a, n, n, n)
        mgs.append(mg)
        x0s.append(x0)
        vs.append(O.init_velocities(mo, len(x0)))
        boxes.append(box)
        crs.append((lat, a, n, n, n))
    offs = list(np.cumsum([0] + [len(q) for q in x0s]))
    S = 2 * NPT["t_eq"] + 2 * NPT["t_s"]
    x, v = T(np.concatenate(x0s)), T(np.concatenate(vs))
    Wd = torch.zeros((2, 2), dtype=torch.float64, device=DEV)
    ne.ne_crystal_run_segment(ctx, mgs, crs, x, v, Wd, 0, S)
    b_run = np.array(ne.ne_ctx_boxes(ctx, 2))
    X0 = T(np.concatenate(x0s))
    x2, v2 = X0.clone(), T(np.concatenate(vs))
    W2 = torch.zeros((2, 2), dtype=torch.float64, device=DEV)
    ne.ne_switch_run_segment(ctx, mgs, offs, x2, v2, X0, boxes, W2, 0, S)
    b_mk = np.array(ne.ne_ctx_boxes(ctx, 2))
    assert np.allclose(b_run, b_mk, rtol=2e-6, atol=0)
    assert torch.abs(x - x2).max().item() < 5e-5
    assert torch.allclose(Wd, W2, rtol=1e-5, atol=1e-4)
    # two segments: the second from the lattice parameter the first reached
    cut = 47
    x3, v3 = T(np.concatenate(x0s)), T(np.concatenate(vs))
    W3 = torch.zeros((2, 2), dtype=torch.float64, device=DEV)
    ne.ne_crystal_run_segment(ctx, mgs, crs, x3, v3, W3, 0, cut)
    b1 = np.array(ne.ne_ctx_boxes(ctx, 2))
    crs2 = [(lat, b1[r][0] / n, n, n, n) for r, (lat, a, n, seed) in enumerate(systems)]
    ne.ne_crystal_run_segment(ctx, mgs, crs2, x3, v3, W3, cut, S - cut)
    assert np.allclose(np.array(ne.ne_ctx_boxes(ctx, 2)), b_run, rtol=1e-6, atol=0)
    assert torch.abs(x3 - x).max().item() < 2e-5
    assert torch.allclose(W3, Wd, rtol=1e-6, atol=1e-5)


def test_brick_barostat_on_a_cell_above_the_cluster_limit(ctx, pot):
    """bcc 14^3 (5488 atoms, more than a cluster holds, so the brick runner
    takes it with many CTAs whose virial sums meet in global memory) under
    the isotropic barostat: box, positions and works follow the oracle."""
    p, th = pot
    x0, box = O.create_crystal(O.BCC, 2.90, 14, 14, 14)
    mo, mg = pair(1, t_eq=10, t_s=20)
    v0 = O.init_velocities(mo, len(x0))
    ro = O.switch_run(p, th, mo, x0, v0, x0, box)
    x, v = T(x0), T(v0)
    Wd = torch.zeros((1, 2), dtype=torch.float64, device=DEV)
    ne.ne_crystal_run_segment(ctx, [mg], [(O.BCC, 2.90, 14, 14, 14)], x, v, Wd, 0, 60)
    bg = ne.ne_ctx_boxes(ctx, 1)[0]
    assert np.abs(np.asarray(bg) / box - 1.0).max() > 1e-4  # the box moved
    assert np.allclose(bg, ro["box"], rtol=2e-6, atol=0)
    assert np.abs(x.cpu().numpy() - ro["x"]).max() < 5e-5
    assert float(Wd[0, 0]) == pytest.approx(ro["W_f"], rel=1e-5, abs=1e-3)
    assert float(Wd[0, 1]) == pytest.approx(ro["W_b"], rel=1e-5, abs=1e-3)


def test_rs_batch_at_zero_pressure_matches_rs_works(ctx):
    """Reversible scaling at P = 0 (Sec. III.C with the isotropic barostat)
    from workflow.rs_batch on the crystal runner, in chunks that restart from
    the lattice parameter reached, against workflow.rs_works on the
    multi-kernel path (the same seeds and noise streams): F(T) on a 300-600 K
    grid and the final lattice parameters agree."""
    from paper_2201_04622_gb300 import workflow as WF
    lam_f, t_eq, t_s, T0 = 0.5, 200, 2000, 300.0
    cf, cb, a_c = WF.rs_batch(ctx, [(O.BCC, W.A_BCC, 6)] * 2, T0, [1, 2], lam_f, t_eq, t_s, MASS,
                              replica_ids=[0, 0], chunk=1500, npt=True)
    gf, gb, a_g = WF.rs_works(ctx, O.BCC, W.A_BCC, 6, T0, MASS, lam_f, t_eq, t_s, [1, 2], npt=True)
    assert np.abs(a_c / W.A_BCC - 1.0).max() > 1e-4  # the lattice moved
    assert np.allclose(a_c, a_g, rtol=1e-4, atol=0)
    grid = np.linspace(300.0, 600.0, 7)
    Fc = WF.rs_free_energy(O.BCC, W.A_BCC, 6, T0, -4.2, lam_f, t_s, cf, cb, grid)
    Fg = WF.rs_free_energy(O.BCC, W.A_BCC, 6, T0, -4.2, lam_f, t_s, gf, gb, grid)
    assert np.abs(np.asarray(Fc) - np.asarray(Fg)).max() < 1e-4
