"""Plain FP64 CPU oracle of nonequilibrium free-energy switching MD.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
never does.  The arithmetic lives in ``ne_oracle.c`` (plain C, one loop per
definition of the paper); this module compiles it with gcc and marshals numpy
arrays through ctypes.  It shares no code with the CUDA library.

Parity status per function (what pins it, see tests/test_oracle_pins.py):
  create_crystal        site counts, nearest-neighbour shells, closed forms
  eam_theta / hermite   analytic values at knots, cubic exactness, continuity
  pairs_cells           brute-force all-pairs on tiny and wrapped cells
  eam_energy_forces     -grad E by central differences; perfect-lattice energy
                        against an independent numpy evaluation of the
                        analytic potential; Newton's third law
  eam_grad_theta        central differences in theta
  lambda_fl / lambda_rs end conditions, symmetry, printed values, T linear
  sched_lambda          the four phases' end values, telescoping work weights,
                        the backward switch mirrors the forward one
  pressure              ideal-gas limit P V = (N - 1) k_B T with the centre
                        fixed; at 0 K equals -dE/dV of the static lattice
                        by central differences (zero at the fitted a)
  philox4x32_10         normal moments, KS and avalanche tests (CPU); bit
                        for bit against cuRAND's Philox4_32_10 (NVIDIA's
                        implementation, run through its device API on the
                        GPU) over >= 1e6 counters (tests/test_gpu_philox_curand.py)
  switch_run (FL)       harmonic->harmonic exact dF, self-switch W == 0,
                        NVE energy conservation, equipartition
  switch_run (RS)       harmonic F(T) = 3NkT ln(hbar w/kT) at every T
                        and an independent FL point on the EAM crystal
  switch_run_prefix     the full run's first n steps bit for bit
  free_energy           F_E and dF_CM closed forms; low-T quasi-harmonic limit
  msd_fit               equipartition on a harmonic crystal
  eam_virial_axes       sums to the virial; -dU/d eps_a by central differences;
                        equal in-plane components on perfect hcp
  barostat (aniso)      ideal-gas volume distribution; relaxes hcp to the
                        static zero-stress a and c found from eam_virial_axes
  species tables        one species in a two-entry table reproduces the
                        single-species run; Einstein F additive over species;
                        eq. cm's centre-of-mass variance against sampling;
                        per-species equipartition and msd under the
                        mass-weighted constraint against Gaussian closed
                        forms; harmonic -> per-species Einstein switch exact
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ne_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libne_oracle.so")
_lock = threading.Lock()
_lib = None

BCC, FCC, HCP = 0, 1, 2
PATH_FL, PATH_RS = 0, 1
H0_EAM, H0_HARMONIC = 0, 1
NPT_OFF, NPT_ISO, NPT_ANISO = 0, 1, 2
STREAM_FL, STREAM_INITV, STREAM_RS, STREAM_MSD, STREAM_STEP = 0, 1, 2, 3, 4
ERRORS = {0: "ok", -1: "EINVAL", -4: "ERANGE", -6: "ENAN"}


class OracleError(RuntimeError):
    pass


class EAM(C.Structure):
    _fields_ = [("A", C.c_double), ("alpha", C.c_double), ("beta", C.c_double),
                ("B", C.c_double), ("r_e", C.c_double), ("r_s", C.c_double),
                ("r_c", C.c_double), ("rho_max", C.c_double), ("n_knots", C.c_int)]


class MD(C.Structure):
    _fields_ = [("dt", C.c_double), ("T", C.c_double), ("damp", C.c_double),
                ("mass", C.c_double), ("k_spring", C.c_double),
                ("lambda_fn", C.c_int), ("path", C.c_int),
                ("t_eq", C.c_long), ("t_s", C.c_long), ("lambda_f", C.c_double),
                ("seed", C.c_uint64), ("replica", C.c_uint32),
                ("fix_cm", C.c_int), ("h0", C.c_int), ("k_h0", C.c_double),
                ("npt", C.c_int), ("P0", C.c_double), ("beta_T", C.c_double), ("tau_p", C.c_double),
                ("n_species", C.c_int), ("species", C.c_void_p), ("mass_s", C.c_void_p),
                ("k_s", C.c_void_p)]


def build(force: bool = False) -> str:
    """Compile ne_oracle.c into a shared library (gcc, -O2, IEEE FP64)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB) >= os.path.getmtime(os.path.join(_HERE, "ne_oracle.h"))):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i, p = C.c_double, C.c_int, C.c_void_p
            L.ora_kB.restype = d
            L.ora_hbar.restype = d
            L.ora_amu.restype = d
            L.ora_lambda_fl.restype = d
            L.ora_lambda_fl.argtypes = [i, d]
            L.ora_lambda_rs.restype = d
            L.ora_lambda_rs.argtypes = [d, d]
            L.ora_einstein_F.restype = d
            L.ora_einstein_F.argtypes = [i, d, d, d]
            L.ora_cm_correction.restype = d
            L.ora_cm_correction.argtypes = [i, d, d, d, d]
            L.ora_eam_analytic.argtypes = [p, i, d, p, p]
            L.ora_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                      C.c_uint64, p]
            L.ora_hermite.argtypes = [p, i, d, d, p, p]
            L.ora_create_crystal.argtypes = [i, d, i, i, i, p, p, p]
            L.ora_pairs_brute.argtypes = [p, i, p, d, p, p, i, p]
            L.ora_pairs_cells.argtypes = [p, i, p, d, p, p, i, p]
            L.ora_eam_energy_forces.argtypes = [p, p, p, i, p, p, p, p]
            L.ora_eam_grad_theta.argtypes = [p, p, p, i, p, p]
            L.ora_eam_virial_axes.argtypes = [p, p, p, i, p, p]
            L.ora_spring.argtypes = [p, p, i, d, p, p]
            L.ora_init_velocities.argtypes = [p, i, p]
            L.ora_switch_run.argtypes = [p, p, p, p, p, p, i, p, p, p, p, p, p, i, i]
            L.ora_langevin_steps.argtypes = [p, p, p, d, p, p, p, i, p, C.c_long, C.c_long]
            L.ora_switch_run_prefix.argtypes = [p, p, p, p, p, p, i, p, C.c_long, p, p, p, p]
            L.ora_msd_fit.argtypes = [p, p, p, p, p, p, i, p, C.c_long, C.c_long, i, p, p]
            L.ora_msd_fit_species.argtypes = [p, p, p, p, p, p, i, p, C.c_long, C.c_long, i, p, p]
            L.ora_einstein_F_species.restype = d
            L.ora_einstein_F_species.argtypes = [i, p, p, p, d]
            L.ora_cm_correction_species.restype = d
            L.ora_cm_correction_species.argtypes = [i, p, p, p, d, d]
            L.ora_free_energy_species.argtypes = [i, p, i, p, p, d, d, p, p, i, p, p, p]
            L.ora_free_energy.argtypes = [i, d, d, d, d, p, p, i, p, p, p]
            L.ora_rs_free_energy.argtypes = [i, d, d, d, C.c_long, p, p, i, p, i, p]
            L.ora_philox4x32_10.argtypes = [p, p, p]
            L.ora_philox_many.argtypes = [i, p, p, p]
            L.ora_sched_lambda.restype = d
            L.ora_sched_lambda.argtypes = [p, C.c_long]
            L.ora_pressure.argtypes = [i, d, d, p, i, p, p]
            L.ora_normals_many.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, i, p]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _pref(p):
    return None if p is None else C.byref(p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(st, what):
    if st != 0:
        raise OracleError("%s failed: %s" % (what, ERRORS.get(st, st)))


# ----------------------------------------------------------------- constants
def kB():
    return lib().ora_kB()


def hbar():
    return lib().ora_hbar()


def amu():
    return lib().ora_amu()


# ------------------------------------------------------------------- inputs
def eam(A, alpha, beta, B, r_e, r_s, r_c, rho_max, n_knots) -> EAM:
    return EAM(A, alpha, beta, B, r_e, r_s, r_c, rho_max, n_knots)


def md(dt=1e-3, T=100.0, damp=0.1, mass=None, k_spring=5.0, lambda_fn=2, path=PATH_FL,
       t_eq=0, t_s=1, lambda_f=0.5, seed=1, replica=0, fix_cm=1, h0=H0_EAM,
       k_h0=0.0, npt=0, P0=0.0, beta_T=0.0, tau_p=0.0, species=None, mass_s=None,
       k_s=None) -> MD:
    """npt = NPT_ISO: isotropic barostat at pressure P0 (eV/A^3) with coupling
    compressibility beta_T (A^3/eV) and time tau_p (ps); NPT_ANISO: the same
    on each box edge separately (non-cubic cells); RS path only.

    species ([n] ints), mass_s and k_s ([n_species]): one mass and one Einstein
    spring per species (Sec. V); mass and k_spring are then unused.  The
    returned struct keeps the three arrays alive."""
    if mass is None:
        mass = 55.845 * amu()
    m = MD(dt, T, damp, mass, k_spring, lambda_fn, path, t_eq, t_s, lambda_f,
           seed, replica, fix_cm, h0, k_h0, npt, P0, beta_T, tau_p)
    if species is not None:
        sp = np.ascontiguousarray(species, dtype=np.int32)
        ms, ks = _f64(mass_s).ravel().copy(), _f64(k_s).ravel().copy()
        if ms.size != ks.size:
            raise ValueError("mass_s and k_s need one entry per species")
        m._keep = (sp, ms, ks)
        m.n_species = ms.size
        m.species, m.mass_s, m.k_s = sp.ctypes.data, ms.ctypes.data, ks.ctypes.data
    return m


def create_crystal(lattice, a, nx, ny, nz, c_over_a=None):
    """Sites and box; hcp uses the orthohexagonal cell (a, sqrt(3) a, c) with
    c = c_over_a * a (default ideal, sqrt(8/3))."""
    n = (2 if lattice == BCC else 4) * nx * ny * nz
    x0 = np.zeros((n, 3))
    box = np.zeros(3)
    nout = C.c_int()
    if c_over_a is None:
        st = lib().ora_create_crystal(lattice, a, nx, ny, nz, _ptr(x0), _ptr(box), C.byref(nout))
    else:
        st = lib().ora_create_crystal_ca(lattice, C.c_double(a), C.c_double(c_over_a), nx, ny, nz, _ptr(x0),
                                         _ptr(box), C.byref(nout))
    _check(st, "create_crystal")
    return x0, box


def eam_analytic(p: EAM, which, x):
    y, dy = C.c_double(), C.c_double()
    lib().ora_eam_analytic(C.byref(p), which, x, C.byref(y), C.byref(dy))
    return y.value, dy.value


def eam_theta(p: EAM):
    th = np.zeros((3, p.n_knots, 2))
    lib().ora_eam_theta(C.byref(p), _ptr(th))
    return th


def hermite(th_one, xmax, x):
    th_one = _f64(th_one)
    y, dy = C.c_double(), C.c_double()
    _check(lib().ora_hermite(_ptr(th_one), th_one.shape[0], xmax, x, C.byref(y),
                             C.byref(dy)), "hermite")
    return y.value, dy.value


def _pairs(fn, x, box, rcut):
    x, box = _f64(x), _f64(box)
    n = x.shape[0]
    cap = 64 * n + 16
    while True:
        pi = np.zeros(cap, np.int32)
        pj = np.zeros(cap, np.int32)
        npairs = C.c_int()
        _check(fn(_ptr(x), n, _ptr(box), rcut, _ptr(pi), _ptr(pj), cap, C.byref(npairs)),
               "pairs")
        if npairs.value <= cap:
            return pi[:npairs.value].copy(), pj[:npairs.value].copy()
        cap = npairs.value + 16


def pairs_brute(x, box, rcut):
    return _pairs(lib().ora_pairs_brute, x, box, rcut)


def pairs_cells(x, box, rcut):
    return _pairs(lib().ora_pairs_cells, x, box, rcut)


def eam_energy_forces(p: EAM, theta, x, box):
    theta, x, box = _f64(theta), _f64(x), _f64(box)
    n = x.shape[0]
    f = np.zeros((n, 3))
    rho = np.zeros(n)
    E = C.c_double()
    _check(lib().ora_eam_energy_forces(C.byref(p), _ptr(theta), _ptr(x), n, _ptr(box),
                                       _ptr(f), C.byref(E), _ptr(rho)), "eam_energy_forces")
    return E.value, f, rho


def eam_virial(p: EAM, theta, x, box):
    """W = sum_{i<j} r_ij . F_ij = -sum_{i<j} r dU/dr (Sec. III.A zero pressure)."""
    theta, x, box = _f64(theta), _f64(x), _f64(box)
    W = C.c_double()
    _check(lib().ora_eam_virial(C.byref(p), _ptr(theta), _ptr(x), x.shape[0], _ptr(box), C.byref(W)),
           "eam_virial")
    return W.value


def eam_virial_axes(p: EAM, theta, x, box):
    """Diagonal of the virial tensor, W_a = -dU/d eps_a (axis a scaled alone)."""
    theta, x, box = _f64(theta), _f64(x), _f64(box)
    W = np.zeros(3)
    _check(lib().ora_eam_virial_axes(C.byref(p), _ptr(theta), _ptr(x), x.shape[0], _ptr(box), _ptr(W)),
           "eam_virial_axes")
    return W


def eam_grad_theta(p: EAM, theta, x, box):
    theta, x, box = _f64(theta), _f64(x), _f64(box)
    g = np.zeros_like(theta)
    _check(lib().ora_eam_grad_theta(C.byref(p), _ptr(theta), _ptr(x), x.shape[0],
                                    _ptr(box), _ptr(g)), "eam_grad_theta")
    return g


def spring(x, x0, k):
    x, x0 = _f64(x), _f64(x0)
    f = np.zeros_like(x)
    E = C.c_double()
    lib().ora_spring(_ptr(x), _ptr(x0), x.shape[0], k, _ptr(f), C.byref(E))
    return E.value, f


def lambda_fl(fn, tau):
    return lib().ora_lambda_fl(fn, tau)


def lambda_rs(lambda_f, tau):
    return lib().ora_lambda_rs(lambda_f, tau)


def sched_lambda(m: MD, step):
    """Lambda in force at the start of `step` of m's four-phase schedule."""
    return lib().ora_sched_lambda(C.byref(m), step)


def pressure(n_dof, T, V, W):
    """(P, standard error) = ((N_dof k_B T + <W>) / (3V), s(W)/sqrt(n)/(3V))."""
    w = _f64(np.atleast_1d(W))
    P, e = C.c_double(), C.c_double()
    lib().ora_pressure(n_dof, T, V, _ptr(w), w.size, C.byref(P), C.byref(e))
    return P.value, e.value


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().ora_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_many(ctr, key):
    """Philox4x32-10 blocks of many counters ([n][4] uint32) under one key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    lib().ora_philox_many(c.shape[0], _ptr(c), _ptr(k), _ptr(out))
    return out


def normals_many(seed, replica, stream, step, n):
    """normals() of atoms 0 .. n-1 at one (seed, replica, stream, step): [n][3]."""
    z = np.zeros((n, 3))
    lib().ora_normals_many(seed, replica, stream, step, n, _ptr(z))
    return z


def normals(seed, replica, stream, atom, step):
    z = np.zeros(3)
    lib().ora_normals(seed, replica, stream, atom, step, _ptr(z))
    return z


def init_velocities(m: MD, n):
    v = np.zeros((n, 3))
    _check(lib().ora_init_velocities(C.byref(m), n, _ptr(v)), "init_velocities")
    return v


def switch_run(p: EAM, theta, m: MD, x, v, x0, box, cumulative=False, trace_stride=0):
    """Run the four-phase schedule in place on copies of x, v.

    Returns dict with W_f, W_b, x, v and optionally Wcum_f/Wcum_b, trace."""
    theta, x0 = _f64(theta), _f64(x0)
    box = _f64(box).copy()  # the barostat updates it
    x, v = _f64(x).copy(), _f64(v).copy()
    n = x.shape[0]
    wf, wb = C.c_double(), C.c_double()
    cf = np.zeros(m.t_s + 1) if cumulative else None
    cb = np.zeros(m.t_s + 1) if cumulative else None
    ntr = 0
    tr = None
    if trace_stride > 0:
        ntr = (2 * m.t_eq + 2 * m.t_s) // trace_stride + 1
        tr = np.zeros((ntr, 8))
    _check(lib().ora_switch_run(_pref(p), _ptr(theta), C.byref(m), _ptr(x), _ptr(v),
                                _ptr(x0), n, _ptr(box), C.byref(wf), C.byref(wb),
                                _ptr(cf), _ptr(cb), _ptr(tr), trace_stride, ntr),
           "switch_run")
    out = dict(W_f=wf.value, W_b=wb.value, x=x, v=v, box=box)
    if cumulative:
        out.update(Wcum_f=cf, Wcum_b=cb)
    if tr is not None:
        out["trace"] = tr
    return out


def switch_run_prefix(p: EAM, theta, m: MD, x, v, x0, box, n_steps, cumulative=False):
    """The first n_steps steps of switch_run's schedule on copies of x, v:
    dict with W_f, W_b (works so far), x, v, box and optionally the
    cumulative works (zero beyond the last switching step reached)."""
    theta, x0 = _f64(theta), _f64(x0)
    box = _f64(box).copy()
    x, v = _f64(x).copy(), _f64(v).copy()
    wf, wb = C.c_double(), C.c_double()
    cf = np.zeros(m.t_s + 1) if cumulative else None
    cb = np.zeros(m.t_s + 1) if cumulative else None
    _check(lib().ora_switch_run_prefix(_pref(p), _ptr(theta), C.byref(m), _ptr(x), _ptr(v), _ptr(x0),
                                       x.shape[0], _ptr(box), int(n_steps), C.byref(wf), C.byref(wb),
                                       _ptr(cf), _ptr(cb)), "switch_run_prefix")
    out = dict(W_f=wf.value, W_b=wb.value, x=x, v=v, box=box)
    if cumulative:
        out.update(Wcum_f=cf, Wcum_b=cb)
    return out


def langevin_steps(p: EAM, theta, m: MD, lam, x, v, x0, box, step0, n_steps):
    theta, x0, box = _f64(theta), _f64(x0), _f64(box)
    x, v = _f64(x).copy(), _f64(v).copy()
    _check(lib().ora_langevin_steps(_pref(p), _ptr(theta), C.byref(m), lam, _ptr(x),
                                    _ptr(v), _ptr(x0), x.shape[0], _ptr(box), step0,
                                    n_steps), "langevin_steps")
    return x, v


def msd_fit(p: EAM, theta, m: MD, x, v, x0, box, n_eq, n_samples, stride):
    theta, x0, box = _f64(theta), _f64(x0), _f64(box)
    x, v = _f64(x).copy(), _f64(v).copy()
    msd, k = C.c_double(), C.c_double()
    _check(lib().ora_msd_fit(_pref(p), _ptr(theta), C.byref(m), _ptr(x), _ptr(v),
                             _ptr(x0), x.shape[0], _ptr(box), n_eq, n_samples, stride,
                             C.byref(msd), C.byref(k)), "msd_fit")
    return msd.value, k.value


def msd_fit_species(p: EAM, theta, m: MD, x, v, x0, box, n_eq, n_samples, stride):
    """Eq. msd per species (Sec. V): (msd_s, k_s) arrays over the species of m."""
    theta, x0, box = _f64(theta), _f64(x0), _f64(box)
    x, v = _f64(x).copy(), _f64(v).copy()
    msd = np.zeros(m.n_species)
    k = np.zeros(m.n_species)
    _check(lib().ora_msd_fit_species(_pref(p), _ptr(theta), C.byref(m), _ptr(x), _ptr(v),
                                     _ptr(x0), x.shape[0], _ptr(box), n_eq, n_samples, stride,
                                     _ptr(msd), _ptr(k)), "msd_fit_species")
    return msd, k


def _species_args(species, mass_s, k_s):
    sp = np.ascontiguousarray(species, dtype=np.int32)
    return sp, _f64(mass_s).ravel(), _f64(k_s).ravel()


def einstein_F_species(species, mass_s, k_s, T):
    sp, ms, ks = _species_args(species, mass_s, k_s)
    return lib().ora_einstein_F_species(sp.size, _ptr(sp), _ptr(ms), _ptr(ks), T)


def cm_correction_species(species, mass_s, k_s, V, T):
    sp, ms, ks = _species_args(species, mass_s, k_s)
    return lib().ora_cm_correction_species(sp.size, _ptr(sp), _ptr(ms), _ptr(ks), V, T)


def free_energy_species(species, mass_s, k_s, V, T, W_f, W_b):
    sp, ms, ks = _species_args(species, mass_s, k_s)
    W_f, W_b = _f64(W_f).ravel(), _f64(W_b).ravel()
    F, se, ed = C.c_double(), C.c_double(), C.c_double()
    _check(lib().ora_free_energy_species(sp.size, _ptr(sp), ms.size, _ptr(ms), _ptr(ks), V, T,
                                         _ptr(W_f), _ptr(W_b), W_f.size, C.byref(F),
                                         C.byref(se), C.byref(ed)), "free_energy_species")
    return F.value, se.value, ed.value


def einstein_F(n, T, mass, k):
    return lib().ora_einstein_F(n, T, mass, k)


def cm_correction(n, V, T, mass, k):
    return lib().ora_cm_correction(n, V, T, mass, k)


def jarzynski(T, W):
    """-kT ln mean exp(-W/kT) (eq. jarz)."""
    W = _f64(W).ravel()
    f = lib().ora_jarzynski
    f.restype = C.c_double
    return f(C.c_double(T), _ptr(W), W.size)


def free_energy(n, V, T, mass, k, W_f, W_b):
    W_f, W_b = _f64(W_f).ravel(), _f64(W_b).ravel()
    F, se, ed = C.c_double(), C.c_double(), C.c_double()
    _check(lib().ora_free_energy(n, V, T, mass, k, _ptr(W_f), _ptr(W_b), W_f.size,
                                 C.byref(F), C.byref(se), C.byref(ed)), "free_energy")
    return F.value, se.value, ed.value


def rs_free_energy(n, T0, F0_T0_total, lambda_f, t_s, Wcum_f, Wcum_b, T_grid):
    Wcum_f = _f64(np.atleast_2d(Wcum_f))
    Wcum_b = _f64(np.atleast_2d(Wcum_b))
    T_grid = _f64(T_grid)
    out = np.zeros(T_grid.size)
    _check(lib().ora_rs_free_energy(n, T0, F0_T0_total, lambda_f, t_s, _ptr(Wcum_f),
                                    _ptr(Wcum_b), Wcum_f.shape[0], _ptr(T_grid),
                                    T_grid.size, _ptr(out)), "rs_free_energy")
    return out
