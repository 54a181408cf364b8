"""Pins of the oracle's several-species extension (CPU only, no GPU).

Sec. V of the paper proposes one Einstein spring per species (k_A, k_B) for
A-B solids, each spring from the msd of its own atoms.  With several masses,
the centre of mass that the dynamics holds fixed is the mass-weighted one:
forces and noise are projected in the mass metric, eq. cm's variance becomes
that of the mass-weighted centre, and the Einstein free energy sums one
oscillator frequency per species.  These tests pin each of those against
one-species reductions, sampling, and Gaussian closed forms of the
constrained harmonic crystal.
"""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as O
from paper_2201_04622_gb300 import workloads as W

AMU = None


def amu():
    global AMU
    if AMU is None:
        AMU = O.amu()
    return AMU


def b2(nx):
    """B2 (CsCl) order on a bcc supercell: corner sites species 0, body centres species 1."""
    x0, box = O.create_crystal(O.BCC, 2.87, nx, nx, nx)
    return x0, box, np.arange(len(x0)) % 2


ZERO_THETA = np.zeros((3, 2, 2))


# ------------------------------------------------------ one-species reduction
def test_equal_species_entries_reduce_to_one_species():
    """A two-entry table with equal masses and springs is one species: eq.
    einstein, eq. cm and eq. fl give the printed single-species forms."""
    m, k, T, n = W.MASS_FE_AMU * amu(), 5.787, 100.0, 128
    sp = np.arange(n) % 2
    V = 64 * 2.87 ** 3
    assert O.einstein_F_species(sp, [m, m], [k, k], T) == pytest.approx(O.einstein_F(n, T, m, k), rel=1e-13)
    assert O.cm_correction_species(sp, [m, m], [k, k], V, T) == pytest.approx(
        O.cm_correction(n, V, T, m, k), rel=1e-12)
    Wf, Wb = np.array([-10.0, -10.2, -9.9]), np.array([9.0, 9.3, 9.1])
    a = O.free_energy_species(sp, [m, m], [k, k], V, T, Wf, Wb)
    b = O.free_energy(n, V, T, m, k, Wf, Wb)
    assert a == pytest.approx(b, rel=1e-13)


def test_equal_species_entries_reproduce_the_one_species_run():
    """The dynamics with a table of equal entries follows the one-species run
    to rounding (the mass-weighted projections become plain means)."""
    p = O.eam(**W.EAM_FE_LIKE)
    th = O.eam_theta(p)
    x0, box, sp = b2(4)
    n, m = len(x0), W.MASS_FE_AMU * amu()
    kw = dict(T=900.0, t_eq=20, t_s=40, seed=5, k_spring=3.0)
    m1 = O.md(**kw)
    m2 = O.md(**kw, species=sp, mass_s=[m, m], k_s=[3.0, 3.0])
    v1, v2 = O.init_velocities(m1, n), O.init_velocities(m2, n)
    assert np.abs(v1 - v2).max() < 1e-14
    r1 = O.switch_run(p, th, m1, x0 + 0.01, v1, x0, box, cumulative=True)
    r2 = O.switch_run(p, th, m2, x0 + 0.01, v2, x0, box, cumulative=True)
    for key in ("W_f", "W_b"):
        assert r2[key] == pytest.approx(r1[key], rel=1e-10, abs=1e-12)
    assert np.abs(r2["x"] - r1["x"]).max() < 1e-11
    assert np.abs(r2["Wcum_f"] - r1["Wcum_f"]).max() < 1e-10
    # per-species msd, count-weighted, is the one-species msd
    mh = dict(T=300.0, h0=O.H0_HARMONIC, k_h0=4.0, seed=2)
    msd1, _ = O.msd_fit(None, ZERO_THETA, O.md(**mh), x0, v1, x0, box, 20, 50, 3)
    msd2, _ = O.msd_fit_species(None, ZERO_THETA, O.md(**mh, species=sp, mass_s=[m, m], k_s=[3.0, 3.0]),
                                x0, v1, x0, box, 20, 50, 3)
    assert msd2.mean() == pytest.approx(msd1, rel=1e-10)


# ------------------------------------------------------------ assembly forms
def test_einstein_F_is_additive_over_species():
    """Independent oscillators: F_E of a mixture is the sum of the one-species
    F_E of its parts, whatever the order of the atoms."""
    T, mA, mB, kA, kB = 700.0, 55.845 * amu(), 26.98 * amu(), 2.5, 6.0
    rng = np.random.default_rng(4)
    sp = rng.permutation(np.r_[np.zeros(37, int), np.ones(91, int)])
    F = O.einstein_F_species(sp, [mA, mB], [kA, kB], T)
    assert F == pytest.approx(O.einstein_F(37, T, mA, kA) + O.einstein_F(91, T, mB, kB), rel=1e-13)
    assert O.einstein_F_species(np.sort(sp), [mA, mB], [kA, kB], T) == pytest.approx(F, rel=1e-13)
    # swapping the labels together with the tables changes nothing
    assert O.einstein_F_species(1 - sp, [mB, mA], [kB, kA], T) == pytest.approx(F, rel=1e-13)


def test_cm_correction_variance_against_sampled_centre_of_mass():
    """Eq. cm's (2 pi kT / (N m w^2)) is 2 pi times the variance of the fixed
    centre of the Einstein crystal; with several species that centre is the
    mass-weighted mean of independent Gaussian displacements (variance kT/k_i
    per axis).  The variance inside the oracle's correction must match the one
    sampled here from that definition."""
    T, V = 500.0, 1234.5
    kT = O.kB() * T
    rng = np.random.default_rng(11)
    n = 24
    sp = rng.integers(0, 3, n)
    mass_s = np.array([55.845, 26.98, 200.0]) * amu()
    k_s = np.array([3.0, 8.0, 1.5])
    mi, ki = mass_s[sp], k_s[sp]
    dcm = O.cm_correction_species(sp, mass_s, k_s, V, T)
    s2_oracle = math.exp((dcm / kT - math.log(n / V)) / 1.5) / (2 * math.pi)
    acc, cnt = 0.0, 0
    for _ in range(10):
        u = rng.standard_normal((100000, n)) * np.sqrt(kT / ki)
        R = u @ mi / mi.sum()
        acc += (R ** 2).sum()
        cnt += R.size
    s2_mc = acc / cnt
    assert s2_oracle == pytest.approx(s2_mc, rel=0.01)       # sampling error ~0.45 %
    # the plain (unweighted) centre would be 2x off here: the check has teeth
    s2_plain = kT * (1.0 / ki).sum() / n ** 2
    assert abs(s2_plain / s2_oracle - 1) > 0.3


# --------------------------------------------- dynamics under the constraint
def _constrained_gaussian(mi, ki, kT):
    """Per-axis variances of a harmonic crystal (springs ki, masses mi) at
    fixed sum_i m_i u_i = 0 and sum_i m_i v_i = 0: Gaussian conditioning."""
    var_u = kT / ki - (mi * kT / ki) ** 2 / (mi ** 2 * kT / ki).sum()
    mvar_v = kT * (1.0 - mi / mi.sum())
    return var_u, mvar_v


def test_species_equipartition_under_the_mass_weighted_constraint():
    """Einstein crystal of an FeAl-like B2 cell (16 atoms, springs 3 and 8
    eV/A^2) at lambda = 1: per species, <u^2> and <m v^2> equal the Gaussian
    closed forms conditioned on the fixed mass-weighted centre and momentum;
    the mass-weighted centre and the momentum stay zero, the plain mean
    displacement does not."""
    x0, box, sp = b2(2)
    n, T = len(x0), 300.0
    kT = O.kB() * T
    mass_s, k_s = np.array([55.845, 26.98]) * amu(), np.array([3.0, 8.0])
    mi, ki = mass_s[sp], k_s[sp]
    m = O.md(T=T, damp=0.1, h0=O.H0_HARMONIC, k_h0=0.0, fix_cm=1, seed=7,
             species=sp, mass_s=mass_s, k_s=k_s)
    x, v = x0.copy(), O.init_velocities(m, n)
    assert np.abs(mi @ v).max() < 1e-13
    assert 0.5 * (mi[:, None] * v ** 2).sum() == pytest.approx(0.5 * (3 * n - 3) * kT, rel=1e-12)
    nb, per, blk = 20, 2000, 10
    u2 = np.zeros((nb, 2))
    mv2 = np.zeros((nb, 2))
    plain_max = 0.0
    step = 0
    for _ in range(200):  # equilibrate
        x, v = O.langevin_steps(None, ZERO_THETA, m, 1.0, x, v, x0, box, step, blk)
        step += blk
    for b in range(nb):
        for _ in range(per):
            x, v = O.langevin_steps(None, ZERO_THETA, m, 1.0, x, v, x0, box, step, blk)
            step += blk
            d = x - x0
            for s in (0, 1):
                u2[b, s] += (d[sp == s] ** 2).sum() / (3 * (sp == s).sum())
                mv2[b, s] += (mi[sp == s, None] * v[sp == s] ** 2).sum() / (3 * (sp == s).sum())
            plain_max = max(plain_max, np.abs(d.mean(0)).max())
        assert np.abs(mi @ (x - x0)).max() < 1e-12
        assert np.abs(mi @ v).max() < 1e-12
    u2 /= per
    mv2 /= per
    var_u, mvar_v = _constrained_gaussian(mi, ki, kT)
    for s in (0, 1):
        for got, want in ((u2[:, s], var_u[sp == s][0]), (mv2[:, s], mvar_v[sp == s][0])):
            se = got.std(ddof=1) / math.sqrt(nb)
            assert se < 0.01 * want
            assert abs(got.mean() - want) < 4 * se
    # the unconstrained values differ by 11.5 % (A, <u^2>) and 8.4 % (A, <m v^2>)
    assert abs(u2[:, 0].mean() / (kT / 3.0) - 1) > 0.07
    assert abs(mv2[:, 0].mean() / kT - 1) > 0.05
    assert plain_max > 1e-3


def test_msd_fit_species_matches_the_constrained_gaussian():
    """Eq. msd per species on a harmonic crystal (one spring k_h for all
    atoms, FeAl-like masses): msd_s = 3 kT/k_h (1 - m_s^2 / sum_j m_j^2) under
    the fixed mass-weighted centre, so the fitted springs differ by species
    although the springs do not."""
    x0, box, sp = b2(2)
    n, T, kh = len(x0), 400.0, 4.0
    kT = O.kB() * T
    mass_s = np.array([55.845, 26.98]) * amu()
    mi = mass_s[sp]
    m = O.md(T=T, damp=0.1, h0=O.H0_HARMONIC, k_h0=kh, fix_cm=1, seed=9,
             species=sp, mass_s=mass_s, k_s=[1.0, 1.0])
    v = O.init_velocities(m, n)
    msd, k = O.msd_fit_species(None, ZERO_THETA, m, x0, v, x0, box, 1000, 40000, 10)
    want = 3 * kT / kh * (1 - mass_s ** 2 / (mi ** 2).sum())
    assert msd == pytest.approx(want, rel=0.025)
    assert k == pytest.approx(3 * kT / msd, rel=1e-14)
    assert k[0] / k[1] == pytest.approx((1 - mass_s[1] ** 2 / (mi ** 2).sum())
                                        / (1 - mass_s[0] ** 2 / (mi ** 2).sum()), rel=0.03)


def test_harmonic_to_species_einstein_switch_is_exact():
    """Frenkel-Ladd switch from springs k_h on every atom to k_A, k_B by
    species, with the mass-weighted centre fixed.  Exact constrained dF:
    sum_i (3/2) kT ln(k_i/k_h) + (3/2) kT ln(s_E^2 / s_h^2), s^2 the variance
    of the fixed centre, proportional to sum_i m_i^2 / k_i.  Masses 200 and
    20 u make that last term 0.053 eV, and 0.034 eV away from a mass-blind
    centre; (W_f - W_b)/2 must equal -dF (sign convention of eq. fl)."""
    x0, box, sp = b2(2)
    n, T, kh = len(x0), 300.0, 4.0
    kT = O.kB() * T
    mass_s, k_s = np.array([200.0, 20.0]) * amu(), np.array([16.0, 4.0])
    mi, ki = mass_s[sp], k_s[sp]

    def job(seed):
        m = O.md(T=T, damp=0.1, h0=O.H0_HARMONIC, k_h0=kh, fix_cm=1, t_eq=1000, t_s=10000,
                 seed=seed, species=sp, mass_s=mass_s, k_s=k_s)
        r = O.switch_run(None, ZERO_THETA, m, x0, O.init_velocities(m, n), x0, box)
        return r["W_f"], r["W_b"]

    with ThreadPoolExecutor(8) as ex:
        res = np.array(list(ex.map(job, range(1, 129))))
    est = 0.5 * (res[:, 0] - res[:, 1])
    cm_term = 1.5 * kT * math.log((mi ** 2 / ki).sum() / (mi ** 2 / kh).sum())
    exact = -(1.5 * kT * np.log(ki / kh).sum() + cm_term)
    se = est.std(ddof=1) / math.sqrt(len(est))
    assert se < 0.004
    assert abs(est.mean() - exact) < 4 * se + 1e-4
    assert abs(cm_term) > 10 * se


# ------------------------------------------------------------------- errors
def test_species_tables_are_validated():
    x0, box, sp = b2(2)
    n, m = len(x0), W.MASS_FE_AMU * amu()
    bad = sp.copy()
    bad[3] = 2
    with pytest.raises(O.OracleError):
        O.init_velocities(O.md(species=bad, mass_s=[m, m], k_s=[1.0, 1.0]), n)
    with pytest.raises(O.OracleError):
        O.init_velocities(O.md(species=sp, mass_s=[m, -m], k_s=[1.0, 1.0]), n)
    mt = O.md(species=sp, mass_s=[m, m], k_s=[1.0, -1.0], t_s=2)
    with pytest.raises(O.OracleError):
        O.switch_run(None, ZERO_THETA, mt, x0, np.zeros_like(x0), x0, box)
    with pytest.raises(O.OracleError):  # one-species fit refuses a species table
        O.msd_fit(None, ZERO_THETA, O.md(species=sp, mass_s=[m, m], k_s=[1.0, 1.0], h0=O.H0_HARMONIC),
                  x0, np.zeros_like(x0), x0, box, 1, 1, 1)
    with pytest.raises(O.OracleError):  # a species without atoms has no msd
        O.msd_fit_species(None, ZERO_THETA, O.md(species=sp, mass_s=[m, m, m], k_s=[1.0, 1.0, 1.0],
                                                 h0=O.H0_HARMONIC),
                          x0, np.zeros_like(x0), x0, box, 1, 1, 1)
    with pytest.raises(O.OracleError):
        O.free_energy_species(sp, [m, m], [1.0, 0.0], 100.0, 300.0, [1.0], [1.0])
