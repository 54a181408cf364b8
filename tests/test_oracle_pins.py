"""Pins of the CPU oracle to things other than itself (CPU only, no GPU).

Each test fixes a part of the oracle against a closed form, an invariant, a
brute-force or library computation, or a value the paper states, chosen so a
dropped term, a wrong sign or a swapped index in the oracle fails one of them.
"""
import json
import math
import os
from concurrent.futures import ThreadPoolExecutor
from fractions import Fraction

import numpy as np
import pytest
import scipy.constants as sc
import scipy.stats

import oracle as O
from paper_2201_04622_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.fixture(scope="module")
def pot():
    p = O.eam(**W.EAM_FE_LIKE)
    return p, O.eam_theta(p)


def mass():
    return W.MASS_FE_AMU * O.amu()


# --------------------------------------------------------------- constants
def test_constants_match_codata():
    assert O.kB() == pytest.approx(sc.k / sc.e, rel=1e-12)
    assert O.hbar() == pytest.approx(sc.hbar / sc.e * 1e12, rel=1e-12)
    # 1 u in eV ps^2 / A^2
    assert O.amu() == pytest.approx(sc.atomic_mass / (sc.e * 1e-24 / 1e-20), rel=1e-12)


# ----------------------------------------------------------------- crystal
@pytest.mark.parametrize("lat,a,nb,shells", [
    (O.BCC, 2.87, 2, [(2.87 * math.sqrt(3) / 2, 8), (2.87, 6), (2.87 * math.sqrt(2), 12)]),
    (O.FCC, 3.65, 4, [(3.65 / math.sqrt(2), 12), (3.65, 6)]),
])
def test_crystal_sites_and_shells(lat, a, nb, shells):
    x0, box = O.create_crystal(lat, a, 4, 4, 4)
    assert x0.shape == (nb * 64, 3)
    assert np.allclose(box, 4 * a)
    assert x0.min() >= 0 and x0.max() < 4 * a
    # every site distinct modulo the box
    keys = {tuple(np.round(r / a * 2).astype(int) % (8)) for r in x0}
    assert len(keys) == len(x0)
    d = x0[None] - x0[:, None]
    d -= box * np.rint(d / box)
    r = np.sqrt((d ** 2).sum(-1))[0]
    for dist, count in shells:
        assert np.sum(np.abs(r - dist) < 1e-9) == count
    # atom order ((ix*ny+iy)*nz+iz)*nb+b
    assert np.allclose(x0[nb * ((1 * 4 + 2) * 4 + 3)], a * np.array([1, 2, 3]))


def test_hcp_sites_and_shells():
    """The orthohexagonal hcp cell: with the ideal axial ratio every site has
    the textbook coordination shells (12 at a, 6 at sqrt(2) a, 2 at
    sqrt(8/3) a, 18 at sqrt(3) a, 12 at sqrt(11/3) a, 6 at 2a); with c/a = 1.6
    the twelve nearest split into 6 in-plane at a and 6 at sqrt(a^2/3 + c^2/4)."""
    a = 2.58
    x0, box = O.create_crystal(O.HCP, a, 6, 3, 3)
    assert x0.shape == (4 * 54, 3)
    assert np.allclose(box, [6 * a, 3 * math.sqrt(3) * a, 3 * math.sqrt(8 / 3) * a])
    d = x0[None] - x0[:, None]
    d -= box * np.rint(d / box)
    r = np.sqrt((d ** 2).sum(-1))
    shells = [(1.0, 12), (math.sqrt(2), 6), (math.sqrt(8 / 3), 2), (math.sqrt(3), 18), (math.sqrt(11 / 3), 12),
              (2.0, 6)]
    for i in (0, 1, 2, 3, 101):
        for dist, count in shells:
            assert np.sum(np.abs(r[i] - dist * a) < 1e-9) == count
    x1, b1 = O.create_crystal(O.HCP, a, 6, 3, 3, c_over_a=1.6)
    d = x1[None] - x1[:, None]
    d -= b1 * np.rint(d / b1)
    r1 = np.sqrt((d ** 2).sum(-1))[2]
    assert np.sum(np.abs(r1 - a) < 1e-9) == 6
    assert np.sum(np.abs(r1 - a * math.sqrt(1 / 3 + 1.6 ** 2 / 4)) < 1e-9) == 6


# --------------------------------------------------------- analytic EAM
def _phi_f_numpy(r, which):
    q = W.EAM_FE_LIKE
    x = np.clip((r - q["r_s"]) / (q["r_c"] - q["r_s"]), 0, 1)
    s = np.where(r <= q["r_s"], 1.0, np.where(r >= q["r_c"], 0.0,
                 (1 - x) ** 3 * (1 + 3 * x + 6 * x * x)))
    if which == 0:
        return q["A"] * np.exp(-q["alpha"] * (r / q["r_e"] - 1)) * s
    return np.exp(-q["beta"] * (r / q["r_e"] - 1)) * s


def test_analytic_potential_and_taper(pot):
    p, _ = pot
    for which in (0, 1):
        for r in [1.3, 2.4855, 3.7, 4.6, 4.9, 5.2999, 5.3, 6.0]:
            y, dy = O.eam_analytic(p, which, r)
            assert y == pytest.approx(_phi_f_numpy(np.array(r), which), rel=1e-13, abs=1e-15)
            h = 1e-6
            fd = (_phi_f_numpy(np.array(r + h), which) - _phi_f_numpy(np.array(r - h), which)) / (2 * h)
            if abs(r - 5.3) > 1e-3 and abs(r - 4.6) > 1e-3:
                assert dy == pytest.approx(fd, rel=1e-6, abs=1e-9)
    # taper is C2 at both ends: second differences match across r_s and r_c
    for rb in (4.6, 5.3):
        h = 1e-4
        for which in (0, 1):
            lo = [O.eam_analytic(p, which, rb - k * h)[0] for k in (0, 1, 2)]
            hi = [O.eam_analytic(p, which, rb + k * h)[0] for k in (0, 1, 2)]
            d2lo = (lo[0] - 2 * lo[1] + lo[2]) / h ** 2
            d2hi = (hi[0] - 2 * hi[1] + hi[2]) / h ** 2
            assert abs(d2lo - d2hi) < 2e-2 * (1 + abs(d2lo))
    y, dy = O.eam_analytic(p, 2, 12.25)
    assert y == pytest.approx(-W.EAM_FE_LIKE["B"] * 3.5)
    assert dy == pytest.approx(-W.EAM_FE_LIKE["B"] / 7.0)


# ----------------------------------------------------------------- Hermite
def test_hermite_reproduces_cubics_and_knots():
    n, xmax = 11, 2.0
    c = [0.3, -1.2, 0.7, 0.25]
    xs = np.linspace(0, xmax, n)
    th = np.stack([c[0] + c[1] * xs + c[2] * xs ** 2 + c[3] * xs ** 3,
                   c[1] + 2 * c[2] * xs + 3 * c[3] * xs ** 2], axis=1)
    for x in np.linspace(0, xmax, 97):
        y, dy = O.hermite(th, xmax, x)
        assert y == pytest.approx(c[0] + c[1] * x + c[2] * x ** 2 + c[3] * x ** 3, abs=1e-13)
        assert dy == pytest.approx(c[1] + 2 * c[2] * x + 3 * c[3] * x ** 2, abs=1e-12)
    g = np.random.default_rng(5)
    th = g.normal(size=(n, 2))
    h = xmax / (n - 1)
    for k in range(n):
        y, dy = O.hermite(th, xmax, k * h)
        assert y == pytest.approx(th[k, 0], abs=1e-14)
        assert dy == pytest.approx(th[k, 1], abs=1e-12)
    # C1 across an interior knot
    for k in range(1, n - 1):
        a = O.hermite(th, xmax, k * h - 1e-9)
        b = O.hermite(th, xmax, k * h + 1e-9)
        assert a[0] == pytest.approx(b[0], abs=1e-7)
        assert a[1] == pytest.approx(b[1], abs=1e-6)
    with pytest.raises(O.OracleError):
        O.hermite(th, xmax, xmax + 0.1)


def test_tables_interpolate_analytic_potential(pot):
    p, th = pot
    for which, xmax, xs in [(0, 5.3, np.linspace(1.5, 5.29, 50)),
                            (1, 5.3, np.linspace(1.5, 5.29, 50)),
                            (2, W.EAM_FE_LIKE["rho_max"], np.linspace(2.0, 29.0, 50))]:
        for x in xs:
            ya, _ = O.eam_analytic(p, which, x)
            yt, _ = O.hermite(th[which], xmax, x)
            assert yt == pytest.approx(ya, rel=1e-9, abs=1e-12)


# -------------------------------------------------------------- neighbours
def _pairset(pi, pj):
    return set(zip(pi.tolist(), pj.tolist()))


@pytest.mark.parametrize("lat,a,n,rcut,amp,seed", [
    (O.BCC, 2.87, 2, 2.6, 0.0, 0),
    (O.FCC, 3.65, 2, 2.7, 0.1, 1),
    (O.BCC, 2.87, 4, 5.6, 0.2, 2),
    (O.BCC, 2.87, 6, 5.3, 0.3, 3),
    (O.FCC, 3.65, 5, 5.8, 0.4, 4),
])
def test_cell_pairs_equal_brute_force(lat, a, n, rcut, amp, seed):
    x0, box = O.create_crystal(lat, a, n, n, n)
    x = W.displaced(x0, amp, seed)
    g = np.random.default_rng(seed)
    x += box * g.integers(-2, 3, size=x.shape)  # unwrapped images
    A = _pairset(*O.pairs_cells(x, box, rcut))
    B = _pairset(*O.pairs_brute(x, box, rcut))
    assert A == B and len(A) > 0


# -------------------------------------------------------------------- EAM
def _eam_numpy_analytic(x, box):
    q = W.EAM_FE_LIKE
    d = x[None] - x[:, None]
    d -= box * np.rint(d / box)
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, 1e9)
    rho = _phi_f_numpy(r, 1).sum(1)
    return 0.5 * _phi_f_numpy(r, 0).sum() - q["B"] * np.sqrt(rho).sum()


def test_eam_energy_against_independent_evaluation(pot):
    p, th = pot
    x0, box = O.create_crystal(O.BCC, 2.87, 4, 4, 4)
    E, f, rho = O.eam_energy_forces(p, th, x0, box)
    assert E / 128 == pytest.approx(-4.28, abs=1e-9)
    assert np.abs(f).max() < 1e-10
    for lat, a, seed in [(O.BCC, 2.87, 11), (O.FCC, 3.65, 12)]:
        x0, box = O.create_crystal(lat, a, 4, 4, 4)
        x = W.displaced(x0, 0.1, seed)
        E, f, rho = O.eam_energy_forces(p, th, x, box)
        assert E == pytest.approx(_eam_numpy_analytic(x, box), rel=1e-9)
        assert np.abs(f.sum(0)).max() < 1e-10  # Newton's third law
        E2, _, _ = O.eam_energy_forces(p, th, x + np.array([0.3, -1.7, 12.0]), box)
        assert E2 == pytest.approx(E, rel=1e-12)


def test_eam_forces_are_minus_gradient(pot):
    p, th = pot
    x0, box = O.create_crystal(O.BCC, 2.87, 4, 4, 4)
    x = W.displaced(x0, 0.08, 21)
    E, f, _ = O.eam_energy_forces(p, th, x, box)
    h = 1e-5
    g = np.random.default_rng(0)
    fd = np.zeros((12, ))
    an = np.zeros((12, ))
    for q, (i, c) in enumerate(zip(g.integers(0, 128, 12), g.integers(0, 3, 12))):
        xp, xm = x.copy(), x.copy()
        xp[i, c] += h
        xm[i, c] -= h
        fd[q] = -(O.eam_energy_forces(p, th, xp, box)[0] - O.eam_energy_forces(p, th, xm, box)[0]) / (2 * h)
        an[q] = f[i, c]
    assert np.linalg.norm(fd - an) / np.linalg.norm(an) < 1e-7


def test_eam_range_errors(pot):
    p, th = pot
    x0, box = O.create_crystal(O.BCC, 2.87, 4, 4, 4)
    x = x0.copy()
    x[1] = x[0] + np.array([0.1, 0.0, 0.0])
    with pytest.raises(O.OracleError, match="ERANGE"):
        O.eam_energy_forces(p, th, x, box)
    x0, box = O.create_crystal(O.BCC, 2.87, 3, 3, 3)  # r_c >= L/2
    with pytest.raises(O.OracleError, match="EINVAL"):
        O.eam_energy_forces(p, th, x0, box)


def test_eam_grad_theta_central_differences(pot):
    p, th = pot
    x0, box = O.create_crystal(O.BCC, 2.87, 4, 4, 4)
    x = W.displaced(x0, 0.1, 31)
    g = O.eam_grad_theta(p, th, x, box)
    E0 = O.eam_energy_forces(p, th, x, box)[0]
    active = [np.flatnonzero(np.abs(g[w]).sum(1) > 0) for w in range(3)]
    rng = np.random.default_rng(1)
    for w in range(3):
        for k in rng.choice(active[w], 6, replace=False):
            for s in (0, 1):
                h = 1e-6 if s == 0 else 1e-6
                tp, tm = th.copy(), th.copy()
                tp[w, k, s] += h
                tm[w, k, s] -= h
                fd = (O.eam_energy_forces(p, tp, x, box)[0] - O.eam_energy_forces(p, tm, x, box)[0]) / (2 * h)
                assert fd == pytest.approx(g[w, k, s], rel=2e-6, abs=2e-6)
    # the energy is linear in the phi and F knots: E = sum g * theta for phi
    # (F enters through knots only, pair term exactly)
    assert np.all(np.isfinite(g))
    assert E0 < 0


# --------------------------------------------------------------- schedules
@pytest.mark.parametrize("lat,a,n,amp,seed", [(O.BCC, 2.80, 5, 0.10, 2), (O.BCC, 2.95, 5, 0.20, 3),
                                                (O.FCC, 3.65, 4, 0.15, 4)])
def test_virial_is_minus_the_scaling_derivative_of_the_energy(pot, lat, a, n, amp, seed):
    """W = sum_{i<j} r_ij . F_ij (the configurational virial behind the
    zero-pressure lattice parameter of Sec. III.A) equals -dU/d(eps) when
    positions and box are scaled by (1 + eps): U depends on the coordinates
    only through the pair distances, each of which scales by (1 + eps)."""
    p, th = pot
    x0, box = O.create_crystal(lat, a, n, n, n)
    x = W.displaced(x0, amp, seed)
    w = O.eam_virial(p, th, x, box)
    eps = 1e-6
    Ep = O.eam_energy_forces(p, th, x * (1 + eps), np.asarray(box) * (1 + eps))[0]
    Em = O.eam_energy_forces(p, th, x * (1 - eps), np.asarray(box) * (1 - eps))[0]
    assert w == pytest.approx(-(Ep - Em) / (2 * eps), rel=1e-6, abs=1e-5)


def test_virial_sign_and_zero_pressure_lattice(pot):
    """The analytic potential's A and B were fixed so that the perfect bcc
    crystal at a = 2.87 A is at zero static pressure: W vanishes there,
    is positive under compression and negative under tension."""
    p, th = pot
    ws = {}
    for a in (2.84, 2.87, 2.90):
        x0, box = O.create_crystal(O.BCC, a, 6, 6, 6)
        ws[a] = O.eam_virial(p, th, x0, box) / len(x0)
    assert abs(ws[2.87]) < 1e-8
    assert ws[2.84] > 1e-3 and ws[2.90] < -1e-3


def test_fl_lambda_function2_pins():
    coef = GOLDEN["fl_function2_coefficients"]["value"]
    for t in [Fraction(0), Fraction(1, 4), Fraction(1, 2), Fraction(3, 4), Fraction(1)]:
        exact = t ** 5 * sum(c * t ** (4 - i) for i, c in enumerate(coef))
        assert O.lambda_fl(2, float(t)) == pytest.approx(float(exact), abs=1e-15)
    assert O.lambda_fl(2, 0.0) == 0.0 and O.lambda_fl(2, 1.0) == 1.0
    assert O.lambda_fl(2, 0.5) == pytest.approx(0.5, abs=1e-15)
    assert O.lambda_fl(2, 0.25) == pytest.approx(0.0489273, abs=5e-8)
    assert O.lambda_fl(2, 0.75) == pytest.approx(0.9510727, abs=5e-8)
    for t in np.linspace(0, 1, 41):
        assert O.lambda_fl(2, 1 - t) == pytest.approx(1 - O.lambda_fl(2, t), abs=1e-13)
        h = 1e-6
        if 0 < t < 1:
            d = (O.lambda_fl(2, t + h) - O.lambda_fl(2, t - h)) / (2 * h)
            assert d == pytest.approx(630 * t ** 4 * (1 - t) ** 4, abs=1e-7)
    # vanishing end slopes (Sec. III.B)
    assert O.lambda_fl(2, 1e-3) < 1e-12 and 1 - O.lambda_fl(2, 1 - 1e-3) < 1e-12
    assert O.lambda_fl(1, 0.37) == 0.37


def test_rs_lambda_pins():
    g = GOLDEN["rs_endpoints"]
    lf = g["lambda_f"]
    assert O.lambda_rs(lf, 0.0) == 1.0
    assert O.lambda_rs(lf, 1.0) == pytest.approx(lf, rel=1e-15)
    assert g["T0"] / O.lambda_rs(lf, 1.0) == pytest.approx(g["T_end"])
    Ts = [g["T0"] / O.lambda_rs(lf, t) for t in np.linspace(0, 1, 21)]
    assert np.allclose(np.diff(Ts), (g["T_end"] - g["T0"]) / 20, rtol=1e-12)


def test_schedule_lambda_pins():
    """The four phases of Sec. III.B / III.C: lambda_i for the first t_eq
    steps, the switch over t_s steps (tau = elapsed steps / t_s), lambda_f for
    t_eq steps, the switch back (FL: 1 - lambda(tau); RS: lambda(1 - tau)),
    lambda_i at the end; the work weights of a switch telescope to
    lambda_f - lambda_i."""
    t_eq, t_s = 7, 10
    fl = O.md(mass=mass(), path=O.PATH_FL, lambda_fn=2, t_eq=t_eq, t_s=t_s)
    lam = [O.sched_lambda(fl, s) for s in range(2 * t_eq + 2 * t_s + 1)]
    assert lam[:t_eq + 1] == [0.0] * (t_eq + 1)
    assert lam[t_eq + t_s:2 * t_eq + t_s + 1] == [1.0] * (t_eq + 1)
    assert lam[-1] == 0.0
    assert lam[t_eq + 5] == pytest.approx(0.5, abs=1e-15)
    for q in range(t_s + 1):
        assert lam[t_eq + q] == pytest.approx(float(Fraction(q, t_s) ** 5 * sum(
            c * Fraction(q, t_s) ** (4 - i) for i, c in enumerate(GOLDEN["fl_function2_coefficients"]["value"]))),
            abs=1e-14)
        assert lam[2 * t_eq + t_s + q] == pytest.approx(1.0 - lam[t_eq + q], abs=1e-14)
    assert sum(lam[s + 1] - lam[s] for s in range(t_eq, t_eq + t_s)) == pytest.approx(1.0, abs=1e-15)
    g = GOLDEN["rs_endpoints"]
    rs = O.md(mass=mass(), path=O.PATH_RS, lambda_f=g["lambda_f"], t_eq=t_eq, t_s=t_s)
    lam = [O.sched_lambda(rs, s) for s in range(2 * t_eq + 2 * t_s + 1)]
    assert lam[:t_eq + 1] == [1.0] * (t_eq + 1) and lam[-1] == 1.0
    assert lam[t_eq + t_s] == pytest.approx(g["lambda_f"], rel=1e-15)
    Ts = [g["T0"] / lam[t_eq + q] for q in range(t_s + 1)]  # T = T0 / lambda, linear in time
    assert np.allclose(np.diff(Ts), (g["T_end"] - g["T0"]) / t_s, rtol=1e-12)
    for q in range(t_s + 1):
        assert lam[2 * t_eq + t_s + q] == pytest.approx(lam[t_eq + t_s - q], rel=1e-15)


def test_pressure_pins(pot):
    """P = (N_dof k_B T + <W>) / (3V) (Sec. III.A's zero-pressure condition):
    with W = 0 the ideal gas of the thermostat's 3N - 3 degrees of freedom,
    P V = (N - 1) k_B T (k_B from CODATA); at 0 K the static lattice's
    pressure equals -dE/dV by central differences in a, vanishing at the
    fitted a = 2.87 A; the error is the standard error of the samples."""
    p, th = pot
    kB = sc.k / sc.e
    P, err = O.pressure(3 * 128 - 3, 300.0, 1234.5, [0.0, 0.0, 0.0])
    assert P * 1234.5 == pytest.approx(127 * kB * 300.0, rel=1e-9) and err == 0.0
    n = 5
    for a in (2.84, 2.87, 2.90):
        x0, box = O.create_crystal(O.BCC, a, n, n, n)
        P0, _ = O.pressure(3 * len(x0) - 3, 0.0, float(np.prod(box)), [O.eam_virial(p, th, x0, box)])
        h = 1e-5
        E = {}
        for s in (-1, 1):
            xs, bs = O.create_crystal(O.BCC, a + s * h, n, n, n)
            E[s] = O.eam_energy_forces(p, th, xs, bs)[0]
        dEdV = (E[1] - E[-1]) / ((n * (a + h)) ** 3 - (n * (a - h)) ** 3)
        assert P0 == pytest.approx(-dEdV, rel=1e-6, abs=1e-9)
        if a == 2.87:
            assert abs(P0) < 1e-9
    w = np.array([1.0, 2.0, 4.0, 7.0])
    P, err = O.pressure(30, 100.0, 50.0, w)
    assert err == pytest.approx(w.std(ddof=1) / 2.0 / 150.0, rel=1e-14)


# ------------------------------------------------------------------ Philox
def test_philox_normals_statistics():
    z = np.array([O.normals(7, 3, O.STREAM_FL, a, s) for a in range(200) for s in range(150)])
    z = z.ravel()
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    assert abs(scipy.stats.kurtosis(z)) < 0.1
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3
    # streams, replicas, atoms and steps give distinct blocks
    a = O.normals(7, 3, 0, 5, 9)
    for other in [O.normals(7, 3, 1, 5, 9), O.normals(7, 4, 0, 5, 9), O.normals(7, 3, 0, 6, 9),
                  O.normals(7, 3, 0, 5, 10), O.normals(8, 3, 0, 5, 9),
                  O.normals(7, 3, 0, 5, 9 + (1 << 32))]:
        assert not np.allclose(a, other)


def test_philox_avalanche_and_uniform_words():
    g = np.random.default_rng(3)
    flips = []
    words = []
    for _ in range(300):
        ctr = g.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
        key = g.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
        out = O.philox(ctr, key)
        words.extend(out.tolist())
        c2 = ctr.copy()
        bit = g.integers(0, 128)
        c2[bit // 32] ^= np.uint32(1 << (bit % 32))
        out2 = O.philox(c2, key)
        flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(out, out2)))
    assert abs(np.mean(flips) - 64) < 2.0
    u = (np.array(words, dtype=np.float64) + 0.5) / 2 ** 32
    assert scipy.stats.kstest(u, "uniform").pvalue > 1e-3


# --------------------------------------------------------------- assembly
def test_einstein_and_cm_closed_forms():
    m = mass()
    n = 128
    V = 64 * 2.87 ** 3
    # sanity scale: k = 5.787 eV/A^2 at 100 K (the paper's spring constant, Sec. III.A)
    k = GOLDEN["spring_constant_bcc_Fe_100K"]["k_eV_per_A2"]
    FE = O.einstein_F(n, 100.0, m, k) / n
    assert FE * 1e3 == pytest.approx(22.796, abs=2e-3)
    assert math.sqrt(k / m) == pytest.approx(31.620, abs=2e-3)
    dcm = O.cm_correction(n, V, 100.0, m, k) / n
    assert dcm * 1e3 == pytest.approx(-1.128, abs=2e-3)
    n2 = 8192
    assert O.cm_correction(n2, 4096 * 2.87 ** 3, 100.0, m, k) / n2 * 1e3 == pytest.approx(-0.0242, abs=2e-4)
    # ln(N)/N decay at fixed density (Sec. III.B)
    vals = [abs(O.cm_correction(nn, nn * 2.87 ** 3 / 2, 100.0, m, k) / nn) for nn in (1000, 10000, 100000)]
    assert vals[0] > vals[1] > vals[2]
    # assembly and its standard error
    Wf = np.array([-10.0, -10.2, -9.9])
    Wb = np.array([9.0, 9.3, 9.1])
    F, se, ed = O.free_energy(n, V, 100.0, m, k, Wf, Wb)
    assert F == pytest.approx((O.einstein_F(n, 100.0, m, k) + 0.5 * (Wf.mean() - Wb.mean())
                               + O.cm_correction(n, V, 100.0, m, k)) / n)
    assert se == pytest.approx(scipy.stats.sem(0.5 * (Wf - Wb) / n))
    assert ed == pytest.approx(-0.5 * (Wf.mean() + Wb.mean()) / n)


# --------------------------------------------------------------- dynamics
def _harmonic_md(**kw):
    base = dict(T=100.0, damp=0.1, k_spring=6.0, h0=O.H0_HARMONIC, k_h0=6.0, fix_cm=1)
    base.update(kw)
    return O.md(**base)


def test_self_switch_gives_zero_work_bitwise():
    x0, box = O.create_crystal(O.BCC, 2.87, 3, 3, 3)
    m = _harmonic_md(k_h0=5.0, k_spring=5.0, t_eq=50, t_s=200, seed=4)
    v = O.init_velocities(m, len(x0))
    r = O.switch_run(None, np.zeros((3, 2, 2)), m, x0, v, x0, box, cumulative=True)
    assert r["W_f"] == 0.0 and r["W_b"] == 0.0
    assert np.all(r["Wcum_f"] == 0.0) and np.all(r["Wcum_b"] == 0.0)


def _run_fl(args):
    m, x0, box, p, th = args
    v = O.init_velocities(m, len(x0))
    r = O.switch_run(p, th, m, x0, v, x0, box)
    return r["W_f"], r["W_b"]


def test_harmonic_to_harmonic_exact_free_energy():
    """dF between Einstein crystals k1 -> k2 with fixed CM is (3N-3)/2 kT ln(k2/k1);
    in the sign convention of eq. fl, (W_f - W_b)/2 = F_0 - F_E = -that."""
    x0, box = O.create_crystal(O.BCC, 2.87, 3, 3, 3)
    n, T, k1, k2 = len(x0), 300.0, 3.0, 9.0
    jobs = [(_harmonic_md(T=T, k_h0=k1, k_spring=k2, t_eq=500, t_s=2000, seed=s), x0, box, None,
             np.zeros((3, 2, 2))) for s in range(1, 9)]
    with ThreadPoolExecutor(8) as ex:
        res = np.array(list(ex.map(_run_fl, jobs)))
    est = 0.5 * (res[:, 0] - res[:, 1])
    exact = -(3 * n - 3) / 2 * O.kB() * T * math.log(k2 / k1)
    se = est.std(ddof=1) / math.sqrt(len(est))
    assert abs(est.mean() - exact) < max(4 * se, 2e-4 * abs(exact))
    # dissipation is non-negative in this sign convention (eq. Ediss)
    assert -0.5 * (res[:, 0] + res[:, 1]).mean() > -3 * se


def test_rs_on_harmonic_crystal_reproduces_einstein_F():
    """With U harmonic and a free centre of mass, eq. rs must give
    3 N kT ln(hbar w / kT) at every T of the grid (within the seed scatter)."""
    x0, box = O.create_crystal(O.BCC, 2.87, 4, 4, 4)
    n, T0, lf, k, ts = len(x0), 100.0, 0.25, 6.0, 3000
    m_list = [O.md(T=T0, damp=0.1, k_spring=k, h0=O.H0_HARMONIC, k_h0=k, fix_cm=0,
                   path=O.PATH_RS, lambda_f=lf, t_eq=500, t_s=ts, seed=s) for s in range(1, 9)]

    def run(m):
        v = O.init_velocities(m, n)
        return O.switch_run(None, np.zeros((3, 2, 2)), m, x0, v, x0, box, cumulative=True)

    with ThreadPoolExecutor(8) as ex:
        res = list(ex.map(run, m_list))
    Ts = np.arange(100.0, 401.0, 25.0)
    F0 = O.einstein_F(n, T0, mass(), k)
    exact = np.array([O.einstein_F(n, T, mass(), k) / n for T in Ts])
    per_seed = np.array([O.rs_free_energy(n, T0, F0, lf, ts, r["Wcum_f"], r["Wcum_b"], Ts) - exact
                         for r in res])
    assert np.all(per_seed[:, 0] == pytest.approx(0.0, abs=1e-12))
    mean = per_seed.mean(0)
    se = per_seed.std(0, ddof=1) / math.sqrt(len(res))
    assert np.all(np.abs(mean) < 4 * se + 1e-5)
    assert se.max() < 1e-3  # the check has teeth: a wrong term shifts F by > 0.05 eV/atom
    # the seed-averaged assembly agrees with the per-seed mean at T0 and is finite elsewhere
    cf = np.array([r["Wcum_f"] for r in res])
    cb = np.array([r["Wcum_b"] for r in res])
    F = O.rs_free_energy(n, T0, F0, lf, ts, cf, cb, Ts)
    assert np.all(np.abs(F - exact) < 4 * se * math.sqrt(len(res)) + 1e-5)


def test_nve_energy_conservation(pot):
    """gamma = 0 gives velocity Verlet (Sec. III.A NVE check): total energy
    conserved, fluctuations scaling as dt^2."""
    p, th = pot
    x0, box = O.create_crystal(O.BCC, 2.87, 4, 4, 4)
    n = len(x0)
    v0 = W.gaussian_velocities(n, math.sqrt(O.kB() * 300 / mass()), 9)
    fl = []
    for dt, nsteps in [(1e-3, 400), (0.5e-3, 800)]:
        m = O.md(T=300.0, damp=0.0, dt=dt, k_spring=5.0, fix_cm=1)
        x, v = x0.copy(), v0.copy()
        es = []
        for blk in range(20):
            x, v = O.langevin_steps(p, th, m, 0.0, x, v, x0, box, blk * nsteps // 20, nsteps // 20)
            E = O.eam_energy_forces(p, th, x, box)[0] + 0.5 * mass() * (v ** 2).sum()
            es.append(E)
        es = np.array(es)
        assert abs(es[-1] - es[0]) / n < 1e-5
        fl.append(es.std())
    assert 2.5 < fl[0] / fl[1] < 6.0


def test_thermostat_equipartition_and_fixed_cm():
    x0, box = O.create_crystal(O.BCC, 2.87, 3, 3, 3)
    n, T = len(x0), 500.0
    m = _harmonic_md(T=T, k_h0=6.0, k_spring=6.0, fix_cm=1, seed=3)
    x, v = x0.copy(), O.init_velocities(m, n)
    assert np.abs(v.sum(0)).max() < 1e-12
    kes, ues = [], []
    for blk in range(400):
        x, v = O.langevin_steps(None, np.zeros((3, 2, 2)), m, 0.0, x, v, x0, box, blk * 10, 10)
        if blk >= 40:
            kes.append(0.5 * mass() * (v ** 2).sum())
            ues.append(0.5 * 6.0 * ((x - x0) ** 2).sum())
    dof = 3 * n - 3
    assert np.mean(kes) == pytest.approx(dof / 2 * O.kB() * T, rel=0.03)
    assert np.mean(ues) == pytest.approx(dof / 2 * O.kB() * T, rel=0.03)
    assert np.abs(v.sum(0)).max() < 1e-10
    assert np.abs((x - x0).mean(0)).max() < 1e-12


def test_msd_fit_on_einstein_crystal():
    """Eq. msd on a harmonic crystal: the CM-corrected msd is (3N-3) kT / (N k1)."""
    x0, box = O.create_crystal(O.BCC, 2.87, 3, 3, 3)
    n, k1 = len(x0), 4.0
    m = _harmonic_md(T=200.0, k_h0=k1, fix_cm=1, seed=2)
    v = O.init_velocities(m, n)
    msd, k = O.msd_fit(None, np.zeros((3, 2, 2)), m, x0, v, x0, box, 500, 2000, 5)
    assert k == pytest.approx(k1 * 3 * n / (3 * n - 3), rel=0.03)


# ------------------------------------------------- low-T quasi-harmonic (P4)
def _hessian(p, th, x0, box):
    n = len(x0)
    H = np.zeros((3 * n, 3 * n))
    h = 1e-4
    for q in range(3 * n):
        xp, xm = x0.copy().ravel(), x0.copy().ravel()
        xp[q] += h
        xm[q] -= h
        fp = O.eam_energy_forces(p, th, xp.reshape(-1, 3), box)[1].ravel()
        fm = O.eam_energy_forces(p, th, xm.reshape(-1, 3), box)[1].ravel()
        H[:, q] = -(fp - fm) / (2 * h)
    return 0.5 * (H + H.T)


@pytest.mark.slow
def test_fl_approaches_quasi_harmonic_limit(pot):
    """Frenkel-Ladd (eq. fl + eq. cm) at low T against the harmonic free energy
    of the same tabulated crystal from its Hessian (numpy eigvalsh):
    F_harm = U0 + kT sum_s ln(hbar w_s / kT) - kT ln(N^{1/2} V / Lambda^3),
    the classical harmonic crystal with the centre-of-mass convention of eq. cm.
    The anharmonic remainder grows like T^2."""
    p, th = pot
    x0, box = O.create_crystal(O.BCC, 2.87, 4, 4, 4)
    n = len(x0)
    V = float(np.prod(box))
    U0 = O.eam_energy_forces(p, th, x0, box)[0]
    H = _hessian(p, th, x0, box)
    w2 = np.linalg.eigvalsh(H / mass())
    w2 = np.sort(w2)
    assert np.all(np.abs(w2[:3]) < 1e-6 * w2[-1]) and np.all(w2[3:] > 0)
    w = np.sqrt(w2[3:])
    kB, hb = O.kB(), O.hbar()

    def F_harm(T):
        kT = kB * T
        lam = 2 * math.pi * hb / math.sqrt(2 * math.pi * mass() * kT)
        return (U0 + kT * np.sum(np.log(hb * w / kT)) - kT * math.log(math.sqrt(n) * V / lam ** 3)) / n

    k = 7.0
    temps = [10.0, 40.0, 80.0]
    jobs = [(O.md(T=T, k_spring=k, t_eq=1000, t_s=4000, seed=s), x0, box, p, th)
            for T in temps for s in (1, 2)]
    with ThreadPoolExecutor(8) as ex:
        res = np.array(list(ex.map(_run_fl, jobs))).reshape(len(temps), 2, 2)
    dev = []
    for q, T in enumerate(temps):
        F, se, ed = O.free_energy(n, V, T, mass(), k, res[q, :, 0], res[q, :, 1])
        dev.append(F - F_harm(T))
    dev = np.array(dev)
    assert abs(dev[0]) < 2e-5           # eV/atom at 10 K
    assert abs(dev[1]) < 2e-4
    assert abs(dev[2]) < 1e-3
    assert abs(dev[2]) > abs(dev[0])


@pytest.mark.slow
def test_forward_backward_cancels_dissipation(pot):
    """Sec. II, eq. W12 / Ediss: longer switching lowers the dissipation
    roughly as 1/t_s, while (W_f - W_b)/2 stays put."""
    p, th = pot
    x0, box = O.create_crystal(O.BCC, 2.87, 4, 4, 4)
    n = len(x0)
    out = {}
    for ts in (300, 3000):
        jobs = [(O.md(T=100.0, k_spring=7.0, t_eq=500, t_s=ts, seed=s), x0, box, p, th)
                for s in (1, 2, 3, 4)]
        with ThreadPoolExecutor(8) as ex:
            res = np.array(list(ex.map(_run_fl, jobs)))
        est = 0.5 * (res[:, 0] - res[:, 1]) / n
        out[ts] = (est.mean(), est.std(ddof=1) / math.sqrt(len(est)),
                   -0.5 * (res[:, 0] + res[:, 1]).mean() / n)
    se = math.hypot(out[300][1], out[3000][1])
    assert abs(out[300][0] - out[3000][0]) < 4 * se + 2e-5
    assert out[300][2] > out[3000][2] > -1e-5
    assert out[300][2] > 3 * out[3000][2]


def test_jarzynski_estimator_pins():
    """Eq. jarz on work samples with known exponential averages: a Gaussian
    work distribution N(mu, s^2) gives exactly dF = mu - s^2 / (2 k_B T)
    (sampled here by 200,001 equally spaced normal quantiles); one sample or
    equal samples give W itself; Jensen's inequality bounds dF by mean W."""
    T = 1400.0
    kT = O.kB() * T
    mu, s = -3.7, 0.2
    z = scipy.stats.norm.ppf((np.arange(200001) + 0.5) / 200001)
    dF = O.jarzynski(T, mu + s * z)
    assert dF == pytest.approx(mu - s * s / (2 * kT), abs=2e-3 * s * s / (2 * kT))
    assert O.jarzynski(T, [2.5]) == pytest.approx(2.5, rel=1e-15)
    assert O.jarzynski(T, [1e4] * 7) == pytest.approx(1e4, rel=1e-15)
    w = np.random.default_rng(3).normal(50.0, 1.0, 40)
    assert O.jarzynski(T, w) <= w.mean()
    assert O.jarzynski(T, w) >= w.min()


def test_barostat_samples_the_ideal_gas_volume_distribution():
    """Isothermal-isobaric ideal gas (U = 0) with the centre of mass fixed:
    the N - 1 free positions give p(V) ~ V^(N-1) exp(-P0 V / kT), a Gamma
    distribution with mean N kT / P0 and variance N (kT / P0)^2.  The final
    volumes of independent runs (each many barostat relaxation times long)
    sample it; a wrong Jacobian term would shift the mean by 1/N = 12.5 %."""
    n, T = 8, 300.0
    kT = O.kB() * T
    P0 = 2.585e-5
    V0 = n * kT / P0
    L = V0 ** (1 / 3)
    g = np.random.default_rng(8)
    x0 = g.uniform(0, L, (n, 3))
    box = np.array([L, L, L])
    p, th = O.eam(**W.EAM_FE_LIKE), None
    th = np.zeros(3 * 2 * W.EAM_FE_LIKE["n_knots"])

    def one(seed):
        m = O.md(T=T, mass=mass(), path=O.PATH_RS, lambda_f=0.5, t_eq=1500, t_s=1, seed=seed,
                 h0=O.H0_HARMONIC, k_h0=0.0, npt=1, P0=P0, beta_T=1.0 / P0, tau_p=0.5)
        v = O.init_velocities(m, n)
        r = O.switch_run(p, th, m, x0, v, x0, box)
        return float(np.prod(r["box"]))

    with ThreadPoolExecutor(8) as ex:
        Vs = np.array(list(ex.map(one, range(1, 801))))
    se = Vs.std(ddof=1) / np.sqrt(len(Vs))
    assert abs(Vs.mean() - V0) < max(4 * se, 0.02 * V0)
    assert abs(Vs.mean() - V0) < 0.06 * V0
    assert Vs.var(ddof=1) == pytest.approx(n * (kT / P0) ** 2, rel=0.3)


def test_barostat_relaxes_a_cold_crystal_to_zero_pressure(pot):
    """At 20 K and P0 = 0, bcc started under tension (a = 2.90 A) contracts to
    the potential's static zero-pressure lattice parameter, 2.87 A (thermal
    expansion at 20 K is ~1e-3 A)."""
    p, th = pot
    x0, box = O.create_crystal(O.BCC, 2.90, 4, 4, 4)
    m = O.md(T=20.0, mass=mass(), path=O.PATH_RS, lambda_f=0.9, t_eq=2000, t_s=1, seed=3,
             npt=1, P0=0.0, beta_T=1.2, tau_p=0.2)
    v = O.init_velocities(m, len(x0))
    r = O.switch_run(p, th, m, x0, v, x0, box)
    assert r["box"][0] / 4 == pytest.approx(2.8705, abs=2.5e-3)
    assert np.allclose(r["box"], r["box"][0])


# ------------------------------------------- per-axis virial and barostat
@pytest.mark.parametrize("lat,a,dims,ca,amp,seed", [(O.BCC, 2.87, (5, 5, 5), None, 0.1, 12),
                                                   (O.HCP, 2.60, (5, 3, 3), 1.58, 0.12, 13)])
def test_virial_axes_are_single_axis_scaling_derivatives(pot, lat, a, dims, ca, amp, seed):
    """W_a = -dU/d eps_a with axis a (coordinates and edge) scaled by e^eps_a
    alone, by central differences; the three sum to the scalar virial."""
    p, th = pot
    x0, box = O.create_crystal(lat, a, *dims, c_over_a=ca)
    x = x0 + np.random.default_rng(seed).uniform(-amp, amp, x0.shape)
    Wa = O.eam_virial_axes(p, th, x, box)
    assert Wa.sum() == pytest.approx(O.eam_virial(p, th, x, box), rel=1e-12)
    h = 1e-5
    for ax in range(3):
        s = np.ones(3)
        s[ax] = math.exp(h)
        Up = O.eam_energy_forces(p, th, x * s, box * s)[0]
        s[ax] = math.exp(-h)
        Um = O.eam_energy_forces(p, th, x * s, box * s)[0]
        assert Wa[ax] == pytest.approx(-(Up - Um) / (2 * h), rel=2e-6, abs=1e-6)


def test_virial_axes_on_perfect_hcp_are_equal_in_the_basal_plane(pot):
    """Hexagonal symmetry: the two in-plane components of the stress of a
    perfect hcp cell are equal; off the zero-stress c/a the axial one is not."""
    p, th = pot
    x0, box = O.create_crystal(O.HCP, W.A_HCP, 5, 3, 3)
    Wa = O.eam_virial_axes(p, th, x0, box)
    assert Wa[0] == pytest.approx(Wa[1], rel=1e-12)
    assert abs(Wa[2] - Wa[0]) > 0.1 * abs(Wa).max()


def test_anisotropic_barostat_samples_the_ideal_gas_volume_distribution():
    """Per-axis barostat, ideal gas: the box shape is free but the volume of
    the N - 1 free positions must follow the same Gamma distribution as with
    the isotropic barostat (mean N kT / P0, variance N (kT / P0)^2); a
    kinetic drive of dof kT instead of N' kT per axis would triple it."""
    n, T = 8, 300.0
    kT = O.kB() * T
    P0 = 2.585e-5
    V0 = n * kT / P0
    L = V0 ** (1 / 3)
    x0 = np.random.default_rng(18).uniform(0, L, (n, 3))
    box = np.array([L, L, L])
    p = O.eam(**W.EAM_FE_LIKE)
    th = np.zeros(3 * 2 * W.EAM_FE_LIKE["n_knots"])

    def one(seed):
        m = O.md(T=T, mass=mass(), path=O.PATH_RS, lambda_f=0.5, t_eq=1500, t_s=1, seed=seed,
                 h0=O.H0_HARMONIC, k_h0=0.0, npt=O.NPT_ANISO, P0=P0, beta_T=1.0 / P0, tau_p=0.5)
        r = O.switch_run(p, th, m, x0, O.init_velocities(m, n), x0, box)
        return float(np.prod(r["box"])), r["box"]

    with ThreadPoolExecutor(8) as ex:
        out = list(ex.map(one, range(1, 801)))
    Vs = np.array([o[0] for o in out])
    se = Vs.std(ddof=1) / np.sqrt(len(Vs))
    assert abs(Vs.mean() - V0) < max(4 * se, 0.02 * V0)
    assert abs(Vs.mean() - V0) < 0.06 * V0
    assert Vs.var(ddof=1) == pytest.approx(n * (kT / P0) ** 2, rel=0.3)
    shapes = np.array([o[1][2] / o[1][0] for o in out])
    assert shapes.std() > 0.05  # the edges did move independently


def test_anisotropic_barostat_relaxes_hcp_to_the_static_zero_stress_cell(pot):
    """fix nph aniso (Sec. III.A): hcp started at the ideal c/a under 4 GPa
    of axial tension relaxes at 5 K, P0 = 0, to the cell whose static stress
    vanishes on every axis (a, c from eam_virial_axes by root finding; the
    kinetic pressure at 5 K moves them by ~1e-4 A).  The isotropic barostat
    cannot change c/a."""
    import scipy.optimize
    p, th = pot

    def stress(v):
        x0, box = O.create_crystal(O.HCP, v[0], 5, 3, 3, c_over_a=v[1] / v[0])
        Wa = O.eam_virial_axes(p, th, x0, box)
        return [Wa[0] / np.prod(box), Wa[2] / np.prod(box)]

    a_s, c_s = scipy.optimize.fsolve(stress, [W.A_HCP, W.A_HCP * math.sqrt(8 / 3)], xtol=1e-12)
    x0, box = O.create_crystal(O.HCP, W.A_HCP, 5, 3, 3)
    n, cells = len(x0), np.array([5.0, 3.0 * math.sqrt(3.0), 3.0])

    def one(args):
        seed, npt = args
        m = O.md(T=5.0, mass=mass(), path=O.PATH_RS, lambda_f=0.9, t_eq=1000, t_s=1, seed=seed,
                 npt=npt, P0=0.0, beta_T=1.2, tau_p=0.2)
        return O.switch_run(p, th, m, x0, O.init_velocities(m, n), x0, box)["box"] / cells

    with ThreadPoolExecutor(8) as ex:
        got = np.array(list(ex.map(one, [(s, O.NPT_ANISO) for s in range(1, 9)])))
    mean = got.mean(0)
    assert mean[0] == pytest.approx(a_s, abs=3e-3)
    assert mean[1] == pytest.approx(a_s, abs=3e-3)
    assert mean[2] == pytest.approx(c_s, abs=3e-3)
    assert abs(W.A_HCP - a_s) > 0.03 and abs(W.A_HCP * math.sqrt(8 / 3) - c_s) > 0.1
    iso = one((1, O.NPT_ISO))
    assert iso[2] / iso[0] == pytest.approx(math.sqrt(8 / 3), rel=1e-12)


def test_anisotropic_barostat_moves_the_lattice_with_the_box(pot):
    """Each barostat move scales coordinate a with edge a (fixed scaled
    coordinates): a perfect bcc lattice at rest, without thermostat, stays
    the perfect lattice of the new box, whose edges changed by different
    factors (every site of a Bravais lattice is an inversion centre, so the
    forces vanish under any homogeneous strain and only the barostat moves
    the atoms)."""
    p, th = pot
    x0, box = O.create_crystal(O.BCC, 2.87, 5, 5, 5)
    m = O.md(T=300.0, damp=0.0, mass=mass(), path=O.PATH_RS, lambda_f=0.9, t_eq=0, t_s=1, seed=21,
             npt=O.NPT_ANISO, P0=0.0, beta_T=1.2, tau_p=0.2)
    r = O.switch_run(p, th, m, x0, np.zeros_like(x0), x0, box)
    ratio = r["box"] / box
    assert np.ptp(ratio) > 1e-4
    assert np.abs(r["x"] / r["box"] - x0 / box).max() < 1e-12


def test_two_sided_estimate_removes_the_dissipation_bias_of_short_switches(pot):
    """Sec. III.B (fig. fl_convergence): a short switch biases each one-sided
    estimate by the dissipation, and the forward/backward combination of
    eq. fl cancels it.  On the 4x4x4 bcc cell at 100 K, 16 seeds of a
    300-step switch give a two-sided F within 4 combined standard errors of
    the 5000-step result stored in tests/golden/c1_works.json (same cell,
    spring and potential), while the one-sided estimates are off by more than
    1 meV/atom on opposite sides of it."""
    p, th = pot
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c1_works.json")))
    x0, box = O.create_crystal(O.BCC, g["a"], g["cells"], g["cells"], g["cells"])
    n, V, T, k = len(x0), float(np.prod(box)), g["T"], g["k"]

    def one(seed):
        m = O.md(T=T, mass=mass(), k_spring=k, t_eq=1000, t_s=300, seed=seed, replica=seed - 1)
        r = O.switch_run(p, th, m, x0, O.init_velocities(m, n), x0, box)
        return r["W_f"], r["W_b"]

    with ThreadPoolExecutor(8) as ex:
        res = np.array(list(ex.map(one, range(101, 117))))
    F2, se, ed = O.free_energy(n, V, T, mass(), k, res[:, 0], res[:, 1])
    ref, se_ref = g["F_per_atom"], g["stderr_per_atom"]
    base = (O.einstein_F(n, T, mass(), k) + O.cm_correction(n, V, T, mass(), k)) / n
    F_fwd = base + res[:, 0].mean() / n   # eq. fl with the backward work replaced by -W_f
    F_bwd = base - res[:, 1].mean() / n
    assert abs(F2 - ref) < 4 * math.hypot(se, se_ref)
    assert F_fwd - ref < -1e-3 and F_bwd - ref > 1e-3
    assert ed > 1e-3


@pytest.mark.slow
def test_rs_of_the_eam_crystal_matches_an_independent_fl_point(pot):
    """The check of Sec. III.C (fig. bcc) on the anharmonic crystal: eq. rs
    from the 100 K Frenkel-Ladd reference of the 4x4x4 bcc cell
    (tests/golden/c1_works.json) up to 400 K (lambda_f = 0.25, 20,000-step
    switches, 8 seeds) equals a separate Frenkel-Ladd calculation at 400 K
    (spring from eq. msd at 400 K, 8 seeds), both at the cell's fixed
    volume, within 4 combined standard errors (~1 meV/atom).  Dropping the
    kinetic term of eq. rs would move F by 72 meV/atom; a wrong sign or
    mapping of the works, by eV."""
    p, th = pot
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c1_works.json")))
    x0, box = O.create_crystal(O.BCC, g["a"], g["cells"], g["cells"], g["cells"])
    n, V = len(x0), float(np.prod(box))
    T0, T1, lf, ts = g["T"], 400.0, 0.25, 20000

    def rs(seed):
        m = O.md(T=T0, mass=mass(), path=O.PATH_RS, lambda_f=lf, t_eq=2000, t_s=ts, seed=seed, replica=seed)
        r = O.switch_run(p, th, m, x0, O.init_velocities(m, n), x0, box, cumulative=True)
        return r["Wcum_f"], r["Wcum_b"]

    mf = O.md(T=T1, mass=mass(), k_spring=1.0, seed=1, replica=0)
    _, k = O.msd_fit(p, th, mf, x0, O.init_velocities(mf, n), x0, box, 2000, 2000, 5)

    def fl(seed):
        m = O.md(T=T1, mass=mass(), k_spring=k, t_eq=2000, t_s=5000, seed=seed, replica=seed)
        r = O.switch_run(p, th, m, x0, O.init_velocities(m, n), x0, box)
        return r["W_f"], r["W_b"]

    with ThreadPoolExecutor(8) as ex:
        res = list(ex.map(rs, range(1, 9)))
        w = np.array(list(ex.map(fl, range(1, 9))))
    cf, cb = np.array([r[0] for r in res]), np.array([r[1] for r in res])
    F0 = g["F_per_atom"] * n
    per = [O.rs_free_energy(n, T0, F0, lf, ts, cf[i], cb[i], [T1])[0] for i in range(len(res))]
    F_rs = O.rs_free_energy(n, T0, F0, lf, ts, cf, cb, [T1])[0]
    se_rs = math.hypot(np.std(per, ddof=1) / math.sqrt(len(per)), g["stderr_per_atom"] * T1 / T0)
    F_fl, se_fl, _ = O.free_energy(n, V, T1, mass(), k, w[:, 0], w[:, 1])
    assert abs(F_rs - F_fl) < 4 * math.hypot(se_rs, se_fl)
    assert math.hypot(se_rs, se_fl) < 5e-4  # a dropped or wrong term of eq. rs is far larger


def test_one_step_switch_takes_the_work_at_the_start_of_the_step(pot):
    """Sec. II.A's discrete work sum with the Hamiltonian jumping at fixed x:
    a one-step switch (t_eq = 0, t_s = 1) from the lattice sites does work
    (lambda_1 - lambda_0) dH/dlambda(x_0) = U_EAM(x_0) - U_E(x_0) = U_EAM(x_0)
    on the Frenkel-Ladd path (function 2 reaches 1 in one step) and
    (lambda_f - 1) U_EAM(x_0) on the reversible-scaling path -- exactly, since
    the state after the step plays no part."""
    p, th = pot
    x0, box = O.create_crystal(O.BCC, W.A_BCC, 4, 4, 4)
    U0 = O.eam_energy_forces(p, th, x0, box)[0]
    for path, want in ((O.PATH_FL, U0), (O.PATH_RS, (0.3 - 1.0) * U0)):
        m = O.md(T=300.0, mass=mass(), k_spring=4.0, path=path, lambda_f=0.3, t_eq=0, t_s=1, seed=2)
        r = O.switch_run(p, th, m, x0, O.init_velocities(m, len(x0)), x0, box, cumulative=True)
        assert r["W_f"] == want
        assert r["Wcum_f"][0] == 0.0 and r["Wcum_f"][1] == want
        assert r["W_b"] != 0.0 and abs(r["W_b"] + want) < 0.05 * abs(want)  # back from x_1, near x_0


def test_prefix_runs_are_the_full_run_cut_short(pot):
    """The first n steps of the schedule are the full run's first n steps:
    positions, velocities and cumulative works equal bit for bit, the works
    so far equal the cumulative work at that point, and a prefix covering
    the whole schedule is the full run."""
    p, th = pot
    x0, box = O.create_crystal(O.BCC, W.A_BCC, 4, 4, 4)
    for path in (O.PATH_FL, O.PATH_RS):
        m = O.md(T=600.0, mass=mass(), k_spring=4.0, path=path, lambda_f=0.5, t_eq=15, t_s=40, seed=7)
        v0 = O.init_velocities(m, len(x0))
        full = O.switch_run(p, th, m, x0, v0, x0, box, cumulative=True)
        cut = 15 + 23  # inside the forward switch
        pre = O.switch_run_prefix(p, th, m, x0, v0, x0, box, cut, cumulative=True)
        assert pre["W_f"] == full["Wcum_f"][23] and pre["W_b"] == 0.0
        assert np.array_equal(pre["Wcum_f"][:24], full["Wcum_f"][:24]) and not pre["Wcum_f"][24:].any()
        whole = O.switch_run_prefix(p, th, m, x0, v0, x0, box, 10 ** 6, cumulative=True)
        for key in ("W_f", "W_b"):
            assert whole[key] == full[key]
        assert np.array_equal(whole["x"], full["x"]) and np.array_equal(whole["Wcum_b"], full["Wcum_b"])
        # the state after the prefix is the state after that many steps of the full schedule
        pre2 = O.switch_run_prefix(p, th, m, x0, v0, x0, box, cut + 1)
        assert not np.array_equal(pre2["x"], pre["x"])
