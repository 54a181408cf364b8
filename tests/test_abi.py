"""The C ABI without a GPU: libne.so builds for sm_103a, loads, exports every
entry point include/ne.h declares, and its host-only functions agree with the
oracle.  No kernel is launched here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2201_04622_gb300 import ne, workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ne.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^ne_status\s+(ne_\w+)\s*\(", text, re.M)))


def test_header_declares_the_binding_symbols():
    assert declared_symbols() == sorted(ne.SYMBOLS)


def test_library_exports_every_declared_symbol():
    L = ne.load()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_invalid_arguments_are_rejected_without_a_gpu():
    L = ne.load()
    assert L.ne_ctx_create(None, 10, 1, None) == ne.NE_EINVAL
    assert L.ne_ctx_destroy(None) == ne.NE_EINVAL
    box = (C.c_double * 3)()
    assert L.ne_create_crystal(7, 2.87, 2, 2, 2, None, box, None) == ne.NE_EINVAL
    assert L.ne_create_crystal(ne.NE_BCC, -1.0, 2, 2, 2, None, box, None) == ne.NE_EINVAL
    assert L.ne_noise(1, 0, 99, 0, 10, 0, None, None) == ne.NE_EINVAL


def test_every_entry_point_rejects_null_arguments_without_a_gpu():
    """Null context, null buffers, unit sizes: every entry point returns
    NE_EINVAL before touching the device (the crystal builder's outputs are
    all optional, so there a null call only counts sites)."""
    L = ne.load()
    for name in ne.SYMBOLS:
        f = getattr(L, name)
        args = [None if t is C.c_void_p else (1.0 if t is C.c_double else 1) for t in f.argtypes]
        want = ne.NE_OK if name.startswith("ne_create_crystal") else ne.NE_EINVAL
        assert f(*args) == want, name


@pytest.mark.parametrize("lat,a,n,ca", [(ne.NE_BCC, 2.87, (4, 4, 4), None), (ne.NE_FCC, 3.65, (3, 4, 5), None),
                                       (ne.NE_HCP, 2.58, (4, 3, 3), None), (ne.NE_HCP, 2.58, (3, 3, 4), 1.6)])
def test_crystal_matches_oracle(lat, a, n, ca):
    x0, box = ne.ne_create_crystal(lat, a, *n, c_over_a=ca)
    xo, bo = O.create_crystal(lat, a, *n, c_over_a=ca)
    assert np.allclose(x0, xo, rtol=0, atol=1e-13) and np.allclose(box, bo, rtol=0, atol=1e-13)


def test_free_energy_assembly_matches_oracle():
    g = np.random.default_rng(4)
    m = W.MASS_FE_AMU * O.amu()
    for n, T, k in [(128, 100.0, 5.787), (2000, 1400.0, 3.1), (8192, 400.0, 6.2)]:
        V = n * 11.82
        wf = g.normal(-4.0 * n, 0.01 * n, 10)
        wb = g.normal(4.0 * n, 0.01 * n, 10)
        a = ne.ne_free_energy(n, V, T, m, k, wf, wb)
        b = O.free_energy(n, V, T, m, k, wf, wb)
        assert np.allclose(a, b, rtol=1e-13, atol=1e-15)


def test_species_free_energy_assembly_matches_oracle():
    """Several species (Sec. V): the library's per-species sums against the
    oracle's per-atom loops, and the one-species assembly when the table has
    one entry."""
    g = np.random.default_rng(7)
    amu = O.amu()
    for n, T, nsp in [(16, 300.0, 2), (432, 900.0, 3), (2000, 1400.0, 2)]:
        sp = g.integers(0, nsp, n)
        sp[:nsp] = np.arange(nsp)
        ms = g.uniform(20.0, 200.0, nsp) * amu
        ks = g.uniform(1.0, 9.0, nsp)
        V = n * 11.82
        wf = g.normal(-4.0 * n, 0.01 * n, 7)
        wb = g.normal(4.0 * n, 0.01 * n, 7)
        a = ne.ne_free_energy_species(sp, ms, ks, V, T, wf, wb)
        b = O.free_energy_species(sp, ms, ks, V, T, wf, wb)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-15)
    m = W.MASS_FE_AMU * amu
    one = ne.ne_free_energy_species(np.zeros(128, int), [m], [5.787], 128 * 11.82, 100.0, wf[:3], wb[:3])
    assert np.allclose(one, ne.ne_free_energy(128, 128 * 11.82, 100.0, m, 5.787, wf[:3], wb[:3]),
                       rtol=1e-13, atol=1e-15)
    with pytest.raises(ne.NeError):
        ne.ne_free_energy_species([0, 2], [m, m], [1.0, 1.0], 100.0, 300.0, [1.0], [1.0])
    with pytest.raises(ne.NeError):
        ne.ne_free_energy_species([0, 1], [m, m], [1.0, 0.0], 100.0, 300.0, [1.0], [1.0])


def test_rs_assembly_matches_oracle():
    g = np.random.default_rng(5)
    n, T0, lf, ts = 128, 100.0, 0.0625, 400
    cf = np.cumsum(g.normal(0.5, 0.1, (3, ts + 1)), axis=1)
    cb = np.cumsum(g.normal(-0.5, 0.1, (3, ts + 1)), axis=1)
    cf[:, 0] = 0
    cb[:, 0] = 0
    Ts = np.arange(100.0, 1601.0, 1.0)
    a = ne.ne_rs_free_energy(n, T0, -550.0, lf, ts, cf, cb, Ts)
    b = O.rs_free_energy(n, T0, -550.0, lf, ts, cf, cb, Ts)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


def test_jarzynski_matches_oracle():
    g = np.random.default_rng(6)
    for T, n in [(100.0, 1), (1400.0, 10), (400.0, 257)]:
        w = g.normal(-8000.0, 0.5, n)
        assert ne.ne_jarzynski(T, w) == pytest.approx(O.jarzynski(T, w), rel=1e-13, abs=1e-10)
    with pytest.raises(ne.NeError):
        ne.ne_jarzynski(-1.0, [1.0])


def test_batched_entry_points_reject_an_empty_batch_without_a_gpu():
    """n_rep = 0 is NE_EINVAL at every batched entry point, decided from the
    arguments alone (the non-null pointers here are never followed)."""
    L = ne.load()
    dummy = C.c_void_p(16)
    for name in ("ne_switch_run_batched", "ne_switch_run_segment", "ne_switch_run_segment_grad",
                 "ne_profile_segment", "ne_crystal_run_segment", "ne_crystal_run_segment_cum"):
        f = getattr(L, name)
        args = []
        for q, t in enumerate(f.argtypes):
            if t is C.c_void_p:
                args.append(dummy)
            elif t is C.c_double:
                args.append(1.0)
            else:
                args.append(1)
        # the replica count: argument 2 of the md-array entry points, 3 of the crystal runner's
        args[3 if name.startswith("ne_crystal") else 2] = 0
        assert f(*args) == ne.NE_EINVAL, name


def test_noalloc_rejections_before_any_device_work():
    """Every documented refusal of ne_eam_energy_forces_noalloc (limits
    NE_NOALLOC_MAX_ATOMS = 2048, NE_NOALLOC_MAX_KNOTS = 5000) returns before
    the call touches the device (the pointers below are never dereferenced):
    sizes beyond the fixed scratch (NE_ENOMEM), boxes of edge <= 2 r_c, an
    unknown precision, null buffers and non-finite analytic parameters (the
    NaN placeholders of a file-loaded potential) (NE_EINVAL)."""
    L = ne.load()
    fake = C.c_void_p(256)  # stands for a device buffer; not dereferenced
    box = (C.c_double * 3)(30.0, 30.0, 30.0)
    small = (C.c_double * 3)(30.0, 30.0, 2.0 * W.EAM_FE_LIKE["r_c"])

    def call(eam=None, prec=ne.NE_FP64, x=fake, n=128, bx=box, f=fake, e=fake):
        e_ = ne.eam_params(**W.EAM_FE_LIKE) if eam is None else eam
        return L.ne_eam_energy_forces_noalloc(C.byref(e_), prec, x, n, bx, f, e, None)

    assert call(n=2048 + 1) == ne.NE_ENOMEM
    big = dict(W.EAM_FE_LIKE, n_knots=5000 + 1)
    assert call(eam=ne.eam_params(**big)) == ne.NE_ENOMEM
    assert call(bx=small) == ne.NE_EINVAL
    assert call(prec=7) == ne.NE_EINVAL
    assert call(x=None) == ne.NE_EINVAL
    assert call(f=None, e=None) == ne.NE_EINVAL
    assert call(n=1) == ne.NE_EINVAL
    for key in ("A", "alpha", "beta", "B"):
        assert call(eam=ne.eam_params(**dict(W.EAM_FE_LIKE, **{key: float("nan")}))) == ne.NE_EINVAL, key



@pytest.mark.parametrize("path,fn", [(ne.NE_PATH_FL, 2), (ne.NE_PATH_FL, 1), (ne.NE_PATH_RS, 2)])
def test_lambda_schedule_matches_oracle(path, fn):
    """ne_lambda (the schedule every run uses) against the oracle's schedule
    at every step of a small four-phase run, and its range check."""
    t_eq, t_s = 5, 13
    kw = dict(path=path, lambda_fn=fn, t_eq=t_eq, t_s=t_s, lambda_f=0.0625)
    md = ne.md_params(mass=1.0, **kw)
    mo = O.md(mass=1.0, **kw)
    for s in range(2 * t_eq + 2 * t_s + 1):
        assert ne.ne_lambda(md, s) == pytest.approx(O.sched_lambda(mo, s), abs=1e-13), s
    for bad in (-1, 2 * t_eq + 2 * t_s + 1):
        with pytest.raises(ne.NeError, match="NE_EINVAL"):
            ne.ne_lambda(md, bad)


def test_pressure_matches_oracle():
    """ne_pressure (P = (N_dof k_B T + <W>)/(3V) and its standard error)
    against the oracle's, on virial samples of either sign."""
    rng = np.random.default_rng(5)
    for n_dof, T, V, w in [(381, 1400.0, 2364.5, rng.normal(-40.0, 5.0, 50)), (5997, 300.0, 23645.0, [12.5]),
                           (0, 0.0, 10.0, [1.0, -3.0])]:
        P, se = ne.ne_pressure(n_dof, T, V, w)
        Po, seo = O.pressure(n_dof, T, V, w)
        assert P == pytest.approx(Po, rel=1e-13, abs=1e-18) and se == pytest.approx(seo, rel=1e-12, abs=1e-18)
