"""Several species on the GPU (Sec. V: one Einstein spring per species, for
an A-B solid; reading A24: the fixed centre of mass is the mass-weighted
one).  A B2 (CsCl) cell -- the bcc lattice with species A on the corner and B
on the centre site, masses 55.845 u and 26.98 u -- run through the C ABI
against the oracle's species tables: initial velocities, 100-step switching
trajectories on the multi-kernel path (FP64 to 1e-8 A, mixed) and on the
crystal runner, the per-species msd fit, and a short Frenkel-Ladd campaign
whose free energy, assembled by ne_free_energy_species from the GPU works,
equals the oracle's within 1 meV/atom."""
import numpy as np
import pytest

import oracle as O
from paper_2201_04622_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2201_04622_gb300 import ne  # noqa: E402

DEV = torch.device("cuda:0")
AMU = 1.0 / 9648.5332
MASS_S = [55.845 * AMU, 26.98 * AMU]
K_S = [4.2, 3.1]


@pytest.fixture(scope="module")
def pot():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    p = O.eam(**W.EAM_FE_LIKE)
    return p, O.eam_theta(p)


@pytest.fixture(scope="module")
def ctx():
    c = ne.ne_ctx_create(ne.eam_params(**W.EAM_FE_LIKE), 8192, 16)
    yield c
    ne.ne_ctx_destroy(c)


def b2(n):
    x0, box = O.create_crystal(O.BCC, W.A_BCC, n, n, n)
    species = np.arange(len(x0)) % 2  # basis site 0: A, 1: B
    return x0, box, species


def pair(species, **kw):
    base = dict(dt=1e-3, T=300.0, damp=0.1, lambda_fn=2, t_eq=20, t_s=30, seed=5, replica=3, fix_cm=1)
    base.update(kw)
    prec = base.pop("prec", ne.NE_FP64)
    skin = base.pop("skin", 0.3)
    mo = O.md(mass=MASS_S[0], k_spring=K_S[0], species=species, mass_s=MASS_S, k_s=K_S, **base)
    sp = torch.tensor(species, dtype=torch.uint8, device=DEV)
    mg = ne.md_params(mass=MASS_S[0], k_spring=K_S[0], skin=skin, prec=prec, species=sp, mass_s=MASS_S,
                      k_s=K_S, **base)
    return mo, mg


def T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device=DEV)


def test_species_initial_velocities_match_oracle(ctx, pot):
    x0, box, sp = b2(4)
    mo, mg = pair(sp)
    vo = O.init_velocities(mo, len(x0))
    v = torch.zeros((len(x0), 3), dtype=torch.float64, device=DEV)
    ne.ne_init_velocities(ctx, mg, v)
    torch.cuda.synchronize()
    assert np.abs(v.cpu().numpy() - vo).max() < 1e-12
    m = np.array(MASS_S)[sp]
    assert np.abs((m[:, None] * vo).sum(0)).max() < 1e-12  # the mass-weighted momentum is zero


@pytest.mark.parametrize("prec,tol_x,tol_w", [(ne.NE_FP64, 1e-8, 1e-10), (ne.NE_MIXED, 5e-5, 2e-6)])
def test_species_switch_run_tracks_oracle(ctx, pot, prec, tol_x, tol_w):
    """100 steps of the four-phase FL schedule on bcc 4^3 B2 at 300 K."""
    p, th = pot
    x0, box, sp = b2(4)
    mo, mg = pair(sp, prec=prec)
    v0 = O.init_velocities(mo, len(x0))
    ro = O.switch_run(p, th, mo, x0, v0, x0, box)
    x, v = T(x0), T(v0)
    wf = torch.zeros(1, dtype=torch.float64, device=DEV)
    wb = torch.zeros(1, dtype=torch.float64, device=DEV)
    ne.ne_switch_run(ctx, mg, x, v, T(x0), box, wf, wb)
    torch.cuda.synchronize()
    assert np.abs(x.cpu().numpy() - ro["x"]).max() < tol_x
    assert float(wf.item()) == pytest.approx(ro["W_f"], rel=tol_w)
    assert float(wb.item()) == pytest.approx(ro["W_b"], rel=tol_w)
    # the mass-weighted centre stays where it started (to rounding)
    m = np.array(MASS_S)[sp]
    dR = (m[:, None] * (x.cpu().numpy() - x0)).sum(0) / m.sum()
    assert np.abs(dR).max() < (1e-12 if prec == ne.NE_FP64 else 1e-6)


def test_species_crystal_runner_tracks_oracle(ctx, pot):
    """The persistent crystal runner with species tables: bcc 5^3 B2 at
    600 K, 100 steps, beside a one-species replica in the same launch."""
    p, th = pot
    x0, box, sp = b2(5)
    mo, mg = pair(sp, T=600.0, prec=ne.NE_MIXED, skin=1.0)
    v0 = O.init_velocities(mo, len(x0))
    ro = O.switch_run(p, th, mo, x0, v0, x0, box)
    one = ne.md_params(mass=MASS_S[0], k_spring=K_S[0], prec=ne.NE_MIXED, T=600.0, t_eq=20, t_s=30, seed=9,
                       replica=4, fix_cm=1, skin=1.0)
    mo1 = O.md(mass=MASS_S[0], k_spring=K_S[0], T=600.0, t_eq=20, t_s=30, seed=9, replica=4, fix_cm=1)
    v1 = O.init_velocities(mo1, len(x0))
    ro1 = O.switch_run(p, th, mo1, x0, v1, x0, box)
    x = T(np.concatenate([x0, x0]))
    v = T(np.concatenate([v0, v1]))
    Wd = torch.zeros((2, 2), dtype=torch.float64, device=DEV)
    cr = [(O.BCC, W.A_BCC, 5, 5, 5)] * 2
    ne.ne_crystal_run_segment(ctx, [mg, one], cr, x, v, Wd, 0, 100)
    torch.cuda.synchronize()
    xs = x.cpu().numpy()
    n = len(x0)
    assert np.abs(xs[:n] - ro["x"]).max() < 2e-4
    assert np.abs(xs[n:] - ro1["x"]).max() < 2e-4
    Wg = Wd.cpu().numpy()
    for r, ref in ((0, ro), (1, ro1)):
        assert Wg[r, 0] == pytest.approx(ref["W_f"], rel=1e-5, abs=1e-3)
        assert Wg[r, 1] == pytest.approx(ref["W_b"], rel=1e-5, abs=1e-3)


def test_species_msd_fit_matches_oracle(ctx, pot):
    p, th = pot
    x0, box, sp = b2(4)
    mo, mg = pair(sp, T=400.0)
    v0 = O.init_velocities(mo, len(x0))
    msd_o, k_o = O.msd_fit_species(p, th, mo, x0, v0, x0, box, 20, 10, 5)
    msd, k = ne.ne_msd_fit_species(ctx, mg, T(x0), T(v0), T(x0), box, 20, 10, 5)
    assert np.allclose(msd, msd_o, rtol=1e-9) and np.allclose(k, k_o, rtol=1e-9)


def test_species_free_energy_within_1meV_of_oracle(ctx, pot):
    """Four seeds of a short FL switch (t_eq 200, t_s 500 steps) of bcc 5^3
    B2 at 300 K on the crystal runner (mixed) and in the oracle (FP64):
    every work within 1e-6 eV per atom, and the free energy of eq. fl + eq.
    cm with one spring per species within 1 meV/atom."""
    p, th = pot
    x0, box, sp = b2(5)
    n, seeds = len(x0), [1, 2, 3, 4]
    kw = dict(T=300.0, t_eq=200, t_s=500)
    wo_f, wo_b, mgs, vs = [], [], [], []
    for r, seed in enumerate(seeds):
        mo, mg = pair(sp, seed=seed, replica=r, prec=ne.NE_MIXED, skin=1.0, **kw)
        v0 = O.init_velocities(mo, n)
        ro = O.switch_run(p, th, mo, x0, v0, x0, box)
        wo_f.append(ro["W_f"])
        wo_b.append(ro["W_b"])
        mgs.append(mg)
        vs.append(v0)
    x = T(np.concatenate([x0] * len(seeds)))
    v = T(np.concatenate(vs))
    Wd = torch.zeros((len(seeds), 2), dtype=torch.float64, device=DEV)
    ne.ne_crystal_run_segment(ctx, mgs, [(O.BCC, W.A_BCC, 5, 5, 5)] * len(seeds), x, v, Wd, 0,
                              2 * kw["t_eq"] + 2 * kw["t_s"])
    Wg = Wd.cpu().numpy()
    assert np.abs(Wg[:, 0] - wo_f).max() / n < 1e-6 and np.abs(Wg[:, 1] - wo_b).max() / n < 1e-6
    V = float(np.prod(box))
    F, se, _ = ne.ne_free_energy_species(sp, MASS_S, K_S, V, 300.0, Wg[:, 0], Wg[:, 1])
    Fo, seo, _ = O.free_energy_species(sp, MASS_S, K_S, V, 300.0, wo_f, wo_b)
    assert abs(F - Fo) < 1e-3 and abs(F - Fo) < 2 * (se + seo) + 1e-5
