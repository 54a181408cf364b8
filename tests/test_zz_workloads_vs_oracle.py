"""Full-length and edge-case comparisons of the GPU path with stored oracle
results, on the workloads' own sizes:

- the small case (bcc 4^3 at 100 K: the msd fit and ten seeds at full length);
- the 1400 K campaign, all twenty replicas on the crystal runner;
- the 256-replica uneven set through the chunked runner with its
  multi-kernel fallback, against the oracle's 24-replica subset;
- the reversible-scaling workload (bcc 16^3) on a stated 12,000-step prefix;
- the degenerate one-step schedule on both GPU paths.
- a potential read from a tabulated setfl file.

The stored values come from tests/golden/make_*.py, which call only
oracle/.  Collected after the other GPU tests.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2201_04622_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
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


def N(t):
    return t.detach().cpu().numpy()


def md_pair(**kw):
    """Matching oracle and library parameter blocks."""
    base = dict(dt=1e-3, T=100.0, damp=0.1, k_spring=6.0, lambda_fn=2, t_eq=20, t_s=30,
                lambda_f=0.5, seed=11, replica=2, fix_cm=1)
    base.update(kw)
    skin = base.pop("skin", 0.3)
    prec = base.pop("prec", ne.NE_FP64)
    path = base.pop("path", O.PATH_FL)
    mo = O.md(mass=MASS, path=path, **base)
    mg = ne.md_params(mass=MASS, skin=skin, prec=prec, path=path, **base)
    return mo, mg


def test_fl1400_campaign_all_twenty_replicas_against_the_oracle(ctx):
    """The 1400 K batch (10 x bcc 10^3 + 10 x fcc 8^3, t_eq 10 ps, t_s 50 ps,
    120,000 steps per replica) on the crystal runner in the benchmark's
    launch configuration, against the works of all twenty replicas stored
    from the oracle (tests/golden/fl1400_all_works.json; same seeds and
    replica indices): each work to 1e-6 eV per atom, as for the first eight
    in test_gpu_crystal."""
    import json
    import os
    from paper_2201_04622_gb300 import workflow as WF
    with open(os.path.join(os.path.dirname(__file__), "golden", "fl1400_all_works.json")) as f:
        doc = json.load(f)
    crystals = [(O.BCC, W.A_BCC, 10)] * 10 + [(O.FCC, W.A_FCC, 8)] * 10
    ks = [W.K_BCC_1400] * 10 + [W.K_FCC_1400] * 10
    seeds = list(range(1, 11)) * 2
    Wf, Wb, _ = WF.fl_batch(ctx, crystals, doc["T"], ks, seeds, doc["t_eq"], doc["t_s"], MASS,
                            prec=ne.NE_MIXED, runner="crystal", chunk=20000)
    assert len(doc["rows"]) == 20
    for row in doc["rows"]:
        q = row["replica"]
        lat, a, n = crystals[q]
        assert (lat, a, n, ks[q], seeds[q]) == (row["lattice"], row["a"], row["n"], row["k"], row["seed"])
        tol = 1e-6 * row["natoms"]
        assert abs(Wf[q] - row["W_f"]) < tol, (q, Wf[q], row["W_f"])
        assert abs(Wb[q] - row["W_b"]) < tol, (q, Wb[q], row["W_b"])


def test_small_case_at_full_length_against_the_oracle(ctx):
    """bcc 4x4x4 (128 atoms, a = 2.87 A) at 100 K at full length against the
    oracle's stored results (tests/golden/c1_works.json, written by
    make_c1_works.py from oracle/ alone): the spring from eq. msd (2000 + 2000
    x 5 steps), then ten seeds of 2000 + 5000 + 2000 + 5000 steps as one
    batch.  FP64: the fit and every work equal the oracle's to rounding;
    mixed: F within 1 meV/atom of the oracle's, and within two combined
    standard errors."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c1_works.json")))
    x0, box = O.create_crystal(O.BCC, g["a"], g["cells"], g["cells"], g["cells"])
    n, V, Tk, k = len(x0), float(np.prod(box)), g["T"], g["k"]
    fit = g["fit"]
    mo, mg = md_pair(T=Tk, k_spring=1.0, seed=fit["seed"], replica=fit["replica"])
    x, v = T(x0), T(O.init_velocities(mo, n))
    msd, kf = ne.ne_msd_fit(ctx, mg, x, v, T(x0), box, fit["n_eq"], fit["n_samples"], fit["stride"])
    assert kf == pytest.approx(k, rel=1e-6) and msd == pytest.approx(g["msd"], rel=1e-6)
    rows = g["rows"]
    offs = [r * n for r in range(len(rows) + 1)]
    F = {}
    for name, prec in (("fp64", ne.NE_FP64), ("mixed", ne.NE_MIXED)):
        mos, mgs, vs = [], [], []
        for row in rows:
            mo, mg = md_pair(T=Tk, k_spring=k, t_eq=g["t_eq"], t_s=g["t_s"], seed=row["seed"],
                             replica=row["replica"], prec=prec)
            mgs.append(mg)
            vs.append(O.init_velocities(mo, n))
        X0 = T(np.concatenate([x0] * len(rows)))
        x, v = X0.clone(), T(np.concatenate(vs))
        wf = torch.zeros(len(rows), dtype=torch.float64, device=DEV)
        wb = torch.zeros_like(wf)
        ne.ne_switch_run_batched(ctx, mgs, offs, x, v, X0, [box] * len(rows), wf, wb)
        wf, wb = N(wf), N(wb)
        if prec == ne.NE_FP64:
            assert np.abs(wf - [r["W_f"] for r in rows]).max() < 1e-4
            assert np.abs(wb - [r["W_b"] for r in rows]).max() < 1e-4
        F[name] = ne.ne_free_energy(n, V, Tk, MASS, k, wf, wb)
    assert F["fp64"][0] == pytest.approx(g["F_per_atom"], abs=1e-8)
    assert abs(F["mixed"][0] - g["F_per_atom"]) < 1e-3
    assert abs(F["mixed"][0] - g["F_per_atom"]) < 2 * math.hypot(F["mixed"][1], g["stderr_per_atom"]) + 1e-4


def test_uneven_256_replica_set_at_full_length_against_the_oracle():
    """The 256-replica uneven set (bcc 6-12^3 / fcc 5-10^3, 300-1600 K, t_eq =
    10 ps, t_s = 20 ps) through workflow.fl_batch(runner="auto") -- the
    crystal runner in 20,000-step chunks, a replica that leaves its range
    continuing on the multi-kernel path -- against the oracle's works for a
    stated subset (the 16 smallest replicas and 8 drawn by PCG64(3);
    tests/golden/config3_subset_works.json from make_config3_subset_works.py):
    each replica's F within 1 meV/atom of the oracle's."""
    import json
    import os
    import warnings
    from paper_2201_04622_gb300 import workflow as WF
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "config3_subset_works.json")))
    reps = W.batched_replicas(256, seed=1)
    a = {W.BCC: W.A_BCC, W.FCC: W.A_FCC}
    k = {W.BCC: W.K_BCC_1400, W.FCC: W.K_FCC_1400}
    crystals = [(r["lattice"], a[r["lattice"]], r["n"]) for r in reps]
    big = ne.ne_ctx_create(ne.eam_params(**W.EAM_FE_LIKE), 500000, 256)
    try:
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")  # a hop at high T moves its replica to the multi-kernel path
            Wf, Wb, _ = WF.fl_batch(big, crystals, [r["T"] for r in reps], [k[r["lattice"]] for r in reps],
                                    [r["seed"] for r in reps], g["t_eq"], g["t_s"], MASS, runner="auto",
                                    chunk=20000)
    finally:
        ne.ne_ctx_destroy(big)
    dF = []
    for row in g["rows"]:
        q = row["replica"]
        assert reps[q]["lattice"] == row["lattice"] and reps[q]["n"] == row["n"]
        x0, box = O.create_crystal(row["lattice"], row["a"], row["n"], row["n"], row["n"])
        F = ne.ne_free_energy(len(x0), float(np.prod(box)), row["T"], MASS, row["k"], [Wf[q]], [Wb[q]])[0]
        dF.append(F - row["F_per_atom"])
    assert len(dF) == 24 and np.abs(dF).max() < 1e-3, np.abs(dF).max()


def test_one_step_schedule_edge_case(ctx, pot):
    """Degenerate schedule: no equilibration and a one-step switch (t_eq = 0,
    t_s = 1) from the lattice sites.  The forward work is then
    U_EAM(x_0) - U_E(x_0) = U_EAM(x_0), taken before the step (Sec. II.A):
    the oracle's exactly, the multi-kernel path's to 1e-9 (FP64) and 1e-6
    (mixed) relative, and the crystal runner's to 1e-6 relative."""
    p, th = pot
    x0, box = O.create_crystal(O.BCC, W.A_BCC, 5, 5, 5)
    U0 = O.eam_energy_forces(p, th, x0, box)[0]
    for prec, tol in ((ne.NE_FP64, 1e-9), (ne.NE_MIXED, 1e-6)):
        mo, mg = md_pair(T=300.0, k_spring=4.0, t_eq=0, t_s=1, seed=2, replica=0, prec=prec)
        v0 = O.init_velocities(mo, len(x0))
        ro = O.switch_run(p, th, mo, x0, v0, x0, box)
        assert ro["W_f"] == U0
        x, v = T(x0), T(v0)
        wf = torch.zeros(1, dtype=torch.float64, device=DEV)
        wb = torch.zeros(1, dtype=torch.float64, device=DEV)
        ne.ne_switch_run(ctx, mg, x, v, T(x0), box, wf, wb)
        assert float(wf.item()) == pytest.approx(U0, rel=tol)
        if prec == ne.NE_MIXED:
            x, v = T(x0), T(v0)
            Wd = torch.zeros((1, 2), dtype=torch.float64, device=DEV)
            ne.ne_crystal_run_segment(ctx, [mg], [(O.BCC, W.A_BCC, 5, 5, 5)], x, v, Wd, 0, 2)
            assert float(Wd[0, 0].item()) == pytest.approx(U0, rel=1e-6)


def test_reversible_scaling_workload_prefix_against_the_oracle(ctx):
    """The reversible-scaling workload (bcc 16^3, 8192 atoms, T0 = 100 K,
    lambda 1 -> 0.0625 over 100 ps after 10 ps at lambda = 1) on a stated
    prefix -- its first 12,000 steps, the equilibration and 2000 switching
    steps -- against the oracle's works (tests/golden/config4_prefix_works.json,
    written by make_config4_prefix_works.py from oracle/ alone): the work
    after the prefix to 1e-8 (FP64) and 1e-6 (mixed) relative."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "config4_prefix_works.json")))
    x0, box = O.create_crystal(O.BCC, g["a"], g["cells"], g["cells"], g["cells"])
    n = len(x0)
    for row in g["rows"]:
        for prec, tol in ((ne.NE_FP64, 1e-8), (ne.NE_MIXED, 1e-6)):
            mo, mg = md_pair(T=g["T0"], k_spring=1.0, path=O.PATH_RS, lambda_f=g["lambda_f"], t_eq=g["t_eq"],
                             t_s=g["t_s"], seed=row["seed"], replica=row["replica"], prec=prec)
            x, v = T(x0), T(O.init_velocities(mo, n))
            Wd = torch.zeros((1, 2), dtype=torch.float64, device=DEV)
            ne.ne_switch_run_segment(ctx, [mg], [0, n], x, v, T(x0), [box], Wd, 0, g["prefix_steps"])
            assert float(Wd[0, 0].item()) == pytest.approx(row["W_f"], rel=tol)
            assert float(Wd[0, 1].item()) == 0.0


def test_reversible_scaling_workload_prefix_on_the_brick_runner(ctx):
    """The same prefix of the reversible-scaling workload on the brick runner
    (bcc 16^3 is too large for one thread-block cluster, so the crystal
    runner call takes it there), both seeds in one launch: each work after
    the prefix within 1e-6 relative of the oracle's, as on the mixed
    multi-kernel path."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "config4_prefix_works.json")))
    x0, box = O.create_crystal(O.BCC, g["a"], g["cells"], g["cells"], g["cells"])
    n = len(x0)
    mgs, vs = [], []
    for row in g["rows"]:
        mo, mg = md_pair(T=g["T0"], k_spring=1.0, path=O.PATH_RS, lambda_f=g["lambda_f"], t_eq=g["t_eq"],
                         t_s=g["t_s"], seed=row["seed"], replica=row["replica"], prec=ne.NE_MIXED, skin=1.0)
        mgs.append(mg)
        vs.append(O.init_velocities(mo, n))
    nr = len(mgs)
    x, v = T(np.concatenate([x0] * nr)), T(np.concatenate(vs))
    Wd = torch.zeros((nr, 2), dtype=torch.float64, device=DEV)
    crs = [(O.BCC, g["a"], g["cells"], g["cells"], g["cells"])] * nr
    ne.ne_crystal_run_segment(ctx, mgs, crs, x, v, Wd, 0, g["prefix_steps"])
    for q, row in enumerate(g["rows"]):
        assert float(Wd[q, 0].item()) == pytest.approx(row["W_f"], rel=1e-6)
        assert float(Wd[q, 1].item()) == 0.0


def test_potential_from_a_setfl_file_matches_the_oracle(tmp_path):
    """A tabulated single-element setfl file (written here from the analytic
    Fe-like potential) loaded with potentials.load_eam: a context created
    from its parameters and knots gives the oracle's FP64 energy, forces and
    densities under the same knots to the FP64 parity tolerance."""
    from paper_2201_04622_gb300 import potentials as P
    nr = nrho = 20000
    r_c, rho_max = W.EAM_FE_LIKE["r_c"], W.EAM_FE_LIKE["rho_max"]
    p = O.eam(**W.EAM_FE_LIKE)
    dr, drho = r_c / (nr - 1), rho_max / (nrho - 1)
    r, rho = dr * np.arange(nr), drho * np.arange(nrho)
    F = [O.eam_analytic(p, 2, float(t))[0] for t in rho]
    f = [O.eam_analytic(p, 1, float(t))[0] for t in r]
    rphi = [float(t) * O.eam_analytic(p, 0, float(t))[0] for t in r]
    path = tmp_path / "fe.setfl"
    with open(path, "w") as fh:
        fh.write("c\nc\nc\n1 Fe\n%d %.16e %d %.16e %.16e\n26 55.845 2.87 bcc\n" % (nrho, drho, nr, dr, r_c))
        fh.write("\n".join("%.16e" % v for v in F + f + rphi) + "\n")
    params, theta, _ = P.load_eam(str(path))
    x0, box = O.create_crystal(O.BCC, W.A_BCC, 6, 6, 6)
    x = W.displaced(x0, 0.2, 41)
    Eo, fo, rho_o = O.eam_energy_forces(O.eam(**params), theta.reshape(-1), x, box)
    c = ne.ne_ctx_create(ne.eam_params(**params), 5000, 1)
    try:
        ne.ne_ctx_set_theta(c, T(theta.reshape(-1)))
        xt = T(x)
        fg = torch.zeros_like(xt)
        e = torch.zeros(1, dtype=torch.float64, device=DEV)
        rho_g = torch.zeros(len(x), dtype=torch.float64, device=DEV)
        ne.ne_eam_energy_forces(c, ne.NE_FP64, xt, box, f=fg, e=e, rho=rho_g)
        torch.cuda.synchronize()
    finally:
        ne.ne_ctx_destroy(c)
    assert float(e.item()) == pytest.approx(Eo, rel=1e-10)
    assert np.linalg.norm(N(fg) - fo) < 1e-10 * np.linalg.norm(fo)
    assert np.abs(N(rho_g) - rho_o).max() < 1e-10 * np.abs(rho_o).max()
