"""Thin Python binding of libne.so (include/ne.h): one function per C entry
point, same names, argument marshalling only.  Device arrays are torch CUDA
tensors (float64, contiguous); every computation runs in the library's
kernels.  There is no CPU fallback: without the built library or a GPU the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

NE_OK, NE_EINVAL, NE_ENOMEM, NE_ECUDA, NE_ERANGE, NE_ENEIGH, NE_ENAN, NE_ETIMEOUT, NE_ENOTIMPL = range(9)
STATUS = ["NE_OK", "NE_EINVAL", "NE_ENOMEM", "NE_ECUDA", "NE_ERANGE", "NE_ENEIGH", "NE_ENAN",
          "NE_ETIMEOUT", "NE_ENOTIMPL"]
NE_FP64, NE_MIXED = 0, 1
NE_MAX_SPECIES = 8
CRYSTAL_RUNNER_MAX_ATOMS = 4096  # atoms per replica ne_crystal_run_segment holds
CRYSTAL_RUNNER_ATOMS_PER_CTA = 384  # atoms one CTA of its clusters owns
NE_BCC, NE_FCC, NE_HCP = 0, 1, 2
NE_PATH_FL, NE_PATH_RS = 0, 1

# every symbol include/ne.h declares
SYMBOLS = ["ne_ctx_create", "ne_ctx_destroy", "ne_ctx_clone", "ne_ctx_set_theta", "ne_ctx_get_theta",
           "ne_ctx_set_tuning", "ne_ctx_set_cluster_size", "ne_ctx_set_runner", "ne_ctx_boxes", "ne_ctx_replica_status", "ne_ctx_counters", "ne_ctx_last_run_ms", "ne_ctx_crystal_plan",
           "ne_last_error",
           "ne_create_crystal", "ne_create_crystal_ca", "ne_eam_energy_forces", "ne_eam_virial", "ne_eam_energy_forces_noalloc",
           "ne_spring_forces",
           "ne_eam_backward", "ne_eam_backward_acc", "ne_noise", "ne_init_velocities", "ne_langevin_step",
           "ne_switch_run", "ne_rs_run", "ne_switch_run_batched", "ne_switch_run_segment", "ne_switch_run_segment_cum", "ne_switch_run_segment_grad",
           "ne_profile_segment", "ne_crystal_run_segment", "ne_crystal_run_segment_cum",
           "ne_msd_fit", "ne_msd_fit_batched", "ne_msd_fit_species", "ne_free_energy", "ne_free_energy_species", "ne_jarzynski", "ne_lambda", "ne_pressure",
           "ne_rs_free_energy"]


class NeError(RuntimeError):
    def __init__(self, code, what, msg=""):
        super().__init__("%s: %s%s" % (what, STATUS[code] if 0 <= code < len(STATUS) else code,
                                        (" (" + msg + ")") if msg else ""))
        self.code = code


class EamParams(C.Structure):
    _fields_ = [("A", C.c_double), ("alpha", C.c_double), ("beta", C.c_double),
                ("B", C.c_double), ("r_e", C.c_double), ("r_s", C.c_double),
                ("r_c", C.c_double), ("rho_max", C.c_double), ("n_knots", C.c_int)]


class Crystal(C.Structure):
    _fields_ = [("lattice", C.c_int), ("a", C.c_double), ("nx", C.c_int), ("ny", C.c_int),
                ("nz", C.c_int), ("c_over_a", C.c_double)]


class MdParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("T", C.c_double), ("damp", C.c_double),
                ("mass", C.c_double), ("k_spring", C.c_double), ("skin", C.c_double),
                ("lambda_fn", C.c_int), ("path", C.c_int), ("t_eq", C.c_longlong),
                ("t_s", C.c_longlong), ("lambda_f", C.c_double), ("seed", C.c_ulonglong),
                ("replica", C.c_uint), ("fix_cm", C.c_int), ("prec", C.c_int),
                ("npt", C.c_int), ("P0", C.c_double), ("beta_T", C.c_double), ("tau_p", C.c_double),
                ("n_species", C.c_int), ("mass_s", C.c_double * 8), ("k_s", C.c_double * 8),
                ("species_dev", C.c_void_p)]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libne.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(path):
                raise NeError(NE_ECUDA, "load", "libne.so is not built")
            L = C.CDLL(path)
            p, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
            sigs = {
                "ne_ctx_create": [p, i, i, p],
                "ne_ctx_destroy": [p],
                "ne_ctx_clone": [p, i, i, p],
                "ne_ctx_set_theta": [p, p, p],
                "ne_ctx_get_theta": [p, p, p],
                "ne_ctx_set_tuning": [p, i],
                "ne_ctx_set_cluster_size": [p, i],
                "ne_ctx_set_runner": [p, i],
                "ne_ctx_boxes": [p, i, p],
                "ne_ctx_replica_status": [p, i, p],
                "ne_ctx_counters": [p, p, p, p, p],
                "ne_ctx_last_run_ms": [p, p],
                "ne_ctx_crystal_plan": [p, p, p, p, p],
                "ne_last_error": [p, p, p, i],
                "ne_create_crystal": [i, d, i, i, i, p, p, p],
                "ne_create_crystal_ca": [i, d, d, i, i, i, p, p, p],
                "ne_eam_energy_forces": [p, i, p, i, p, p, p, p, p],
                "ne_eam_virial": [p, p, i, p, p, p],
                "ne_eam_energy_forces_noalloc": [p, i, p, i, p, p, p, p],
                "ne_spring_forces": [p, p, i, d, p, p, p],
                "ne_eam_backward": [p, i, p, i, p, d, p, p, p],
                "ne_eam_backward_acc": [p, i, p, i, p, d, p, p],
                "ne_noise": [C.c_ulonglong, C.c_uint, i, ll, i, i, p, p],
                "ne_init_velocities": [p, p, i, p, p],
                "ne_langevin_step": [p, p, p, p, p, i, p, ll, d, d, p, p],
                "ne_switch_run": [p, p, p, p, p, i, p, p, p, p, p, p, i, p],
                "ne_rs_run": [p, p, d, p, p, p, i, p, p, p, p],
                "ne_switch_run_batched": [p, p, i, p, p, p, p, p, p, p, p],
                "ne_switch_run_segment": [p, p, i, p, p, p, p, p, p, ll, ll, p],
                "ne_switch_run_segment_cum": [p, p, i, p, p, p, p, p, p, p, ll, ll, p],
                "ne_switch_run_segment_grad": [p, p, i, p, p, p, p, p, p, ll, ll, p, p, p],
                "ne_profile_segment": [p, p, i, p, p, p, p, p, p, ll, ll, p, p, p],
                "ne_crystal_run_segment": [p, p, p, i, p, p, p, ll, ll, p],
                "ne_crystal_run_segment_cum": [p, p, p, i, p, p, p, p, ll, ll, p],
                "ne_msd_fit": [p, p, p, p, p, i, p, ll, ll, i, p, p, p],
                "ne_msd_fit_batched": [p, p, i, p, p, p, p, p, ll, ll, i, p, p, p],
                "ne_msd_fit_species": [p, p, p, p, p, i, p, ll, ll, i, p, p, p],
                "ne_free_energy": [i, d, d, d, d, p, p, i, p, p, p],
                "ne_free_energy_species": [i, p, i, p, p, d, d, p, p, i, p, p, p],
                "ne_jarzynski": [d, p, i, p],
                "ne_lambda": [p, ll, p],
                "ne_pressure": [i, d, d, p, i, p, p],
                "ne_rs_free_energy": [i, d, d, d, ll, p, p, i, p, i, p],
            }
            for name, args in sigs.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int
            _lib = L
    return _lib


# ------------------------------------------------------------------ helpers
def _torch():
    import torch
    return torch


def _dev(t, n=None):
    """Pointer of a contiguous float64 CUDA tensor (or None) holding at least
    n elements; the size is checked first, so a host tensor of the right size
    fails only on its device."""
    if t is None:
        return None
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise NeError(NE_EINVAL, "argument", "expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() < n:
        raise NeError(NE_EINVAL, "argument", "tensor too small: %d < %d elements" % (t.numel(), n))
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise NeError(NE_EINVAL, "argument", "expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


_BASIS = {NE_BCC: 2, NE_FCC: 4, NE_HCP: 4}
_CTX_EAM = {}  # context handle -> (n_knots, r_c) of its potential


def _knots6(ctx):
    """Elements of a theta buffer [3][n_knots][2] of ctx (None when unknown)."""
    e = _CTX_EAM.get(getattr(ctx, "value", None))
    return None if e is None else 6 * e[0]


def ctx_cutoff(ctx):
    """Cutoff r_c (A) of the potential of a context this binding created, else None."""
    e = _CTX_EAM.get(getattr(ctx, "value", None))
    return None if e is None else e[1]


def _batch_atoms(offsets, n_rep):
    """Atoms of a batch from its offsets (n_rep + 1 entries, ascending from 0)."""
    off = [int(o) for o in offsets]
    if len(off) != n_rep + 1 or off[0] != 0 or any(b <= a for a, b in zip(off[:-1], off[1:])):
        raise NeError(NE_EINVAL, "argument", "offsets must be n_rep + 1 ascending entries from 0")
    return off[-1]


def _crystal_atoms(crystals):
    """Atoms of the crystal-runner replicas (lattice, a, nx, ny, nz[, c_over_a])."""
    tot = 0
    for c in crystals:
        if int(c[0]) not in _BASIS:
            raise NeError(NE_EINVAL, "argument", "unknown lattice")
        tot += _BASIS[int(c[0])] * int(c[2]) * int(c[3]) * int(c[4])
    return tot


def _trace_rows(md, trace_stride):
    """Rows ne_switch_run writes to its trace: every trace_stride steps of the
    2 t_eq + 2 t_s steps of the run."""
    stride = int(trace_stride) if int(trace_stride) > 0 else 1
    return (2 * int(md.t_eq) + 2 * int(md.t_s) - 1) // stride + 1


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream)
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _box(box):
    return (C.c_double * 3)(*[float(b) for b in box])


def _err(ctx, code, what):
    if code != NE_OK:
        msg = ""
        if ctx is not None:
            buf = C.create_string_buffer(256)
            st = C.c_int()
            load().ne_last_error(ctx, C.byref(st), buf, 256)
            msg = buf.value.decode()
        raise NeError(code, what, msg)


def eam_params(A, alpha, beta, B, r_e, r_s, r_c, rho_max, n_knots) -> EamParams:
    return EamParams(A, alpha, beta, B, r_e, r_s, r_c, rho_max, int(n_knots))


def md_params(dt=1e-3, T=100.0, damp=0.1, mass=None, k_spring=5.0, skin=0.5, lambda_fn=2,
              path=NE_PATH_FL, t_eq=0, t_s=1, lambda_f=0.5, seed=1, replica=0, fix_cm=1,
              prec=NE_FP64, npt=0, P0=0.0, beta_T=0.0, tau_p=0.0, species=None, mass_s=None,
              k_s=None) -> MdParams:
    """npt = 1: isotropic barostat at P0 (eV/A^3), coupling compressibility
    beta_T (A^3/eV) and time tau_p (ps); npt = 2: one such equation per box
    edge (non-cubic cells); reversible-scaling path only.

    species (a uint8 CUDA tensor, one entry per atom of the replica), mass_s
    and k_s (one value per species, 2 .. NE_MAX_SPECIES): one mass and one
    Einstein spring per species (Sec. V); the returned block keeps a
    reference to the tensor."""
    if mass is None:
        mass = 55.845 * 1.0364269656262175e-4
    m = MdParams(dt, T, damp, mass, k_spring, skin, lambda_fn, path, t_eq, t_s, lambda_f,
                 seed, replica, fix_cm, prec, npt, P0, beta_T, tau_p)
    if species is not None:
        torch = _torch()
        ms, ks = list(mass_s), list(k_s)
        if not (2 <= len(ms) <= NE_MAX_SPECIES and len(ks) == len(ms)):
            raise NeError(NE_EINVAL, "md_params", "2..%d species, one mass and one spring each" % NE_MAX_SPECIES)
        if not (isinstance(species, torch.Tensor) and species.is_cuda and species.dtype == torch.uint8
                and species.is_contiguous()):
            raise NeError(NE_EINVAL, "md_params", "species must be a contiguous uint8 CUDA tensor")
        m.n_species = len(ms)
        for q in range(len(ms)):
            m.mass_s[q] = float(ms[q])
            m.k_s[q] = float(ks[q])
        m.species_dev = species.data_ptr()
        m._species_ref = species
    return m


# ------------------------------------------------------------------ entry points
def ne_ctx_create(eam: EamParams, max_atoms: int, max_replicas: int = 1):
    h = C.c_void_p()
    _err(None, load().ne_ctx_create(C.byref(eam), int(max_atoms), int(max_replicas), C.byref(h)),
         "ne_ctx_create")
    _CTX_EAM[h.value] = (int(eam.n_knots), float(eam.r_c))
    return h


def ne_ctx_destroy(ctx):
    _err(None, load().ne_ctx_destroy(ctx), "ne_ctx_destroy")
    _CTX_EAM.pop(getattr(ctx, "value", None), None)


def ne_ctx_clone(src, max_atoms: int, max_replicas: int = 1):
    """A second context with src's potential, theta and tuning."""
    h = C.c_void_p()
    _err(src, load().ne_ctx_clone(src, int(max_atoms), int(max_replicas), C.byref(h)), "ne_ctx_clone")
    if getattr(src, "value", None) in _CTX_EAM:
        _CTX_EAM[h.value] = _CTX_EAM[src.value]
    return h


def ne_ctx_set_theta(ctx, theta, stream=None):
    _err(ctx, load().ne_ctx_set_theta(ctx, _dev(theta, _knots6(ctx)), _stream(stream)), "ne_ctx_set_theta")


def ne_ctx_get_theta(ctx, theta, stream=None):
    _err(ctx, load().ne_ctx_get_theta(ctx, _dev(theta, _knots6(ctx)), _stream(stream)), "ne_ctx_get_theta")


def ne_ctx_set_tuning(ctx, threads_per_atom):
    _err(ctx, load().ne_ctx_set_tuning(ctx, int(threads_per_atom)), "ne_ctx_set_tuning")


def ne_ctx_boxes(ctx, n_rep):
    """Boxes [n_rep][3] at the end of the last multi-kernel run (the barostat's)."""
    import numpy as np
    out = np.zeros((n_rep, 3))
    _err(ctx, load().ne_ctx_boxes(ctx, int(n_rep), out.ctypes.data_as(C.c_void_p)), "ne_ctx_boxes")
    return out


def ne_ctx_replica_status(ctx, n_rep):
    """Per-replica status codes (NE_OK, NE_ERANGE, ...) of the last crystal-runner call."""
    import numpy as np
    out = np.zeros(int(n_rep), dtype=np.int32)
    _err(ctx, load().ne_ctx_replica_status(ctx, int(n_rep), out.ctypes.data_as(C.c_void_p)), "ne_ctx_replica_status")
    return out


def ne_ctx_set_cluster_size(ctx, ctas):
    """CTAs per cluster of the crystal runner (0: chosen per batch)."""
    _err(ctx, load().ne_ctx_set_cluster_size(ctx, int(ctas)), "ne_ctx_set_cluster_size")


def ne_ctx_set_runner(ctx, runner):
    """0 automatic, 1 cluster runner only, 2 brick runner for every batch."""
    _err(ctx, load().ne_ctx_set_runner(ctx, int(runner)), "ne_ctx_set_runner")


def ne_ctx_counters(ctx):
    """(list builds, stencil entries visited, pairs inside r_c, crystal-runner
    kernel launches) so far."""
    a, b, c, d = C.c_longlong(), C.c_longlong(), C.c_longlong(), C.c_longlong()
    _err(ctx, load().ne_ctx_counters(ctx, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), "ne_ctx_counters")
    return a.value, b.value, c.value, d.value


def ne_ctx_last_run_ms(ctx):
    """Device time (ms) of the cluster launches of the last crystal-runner call."""
    ms = C.c_double()
    _err(ctx, load().ne_ctx_last_run_ms(ctx, C.byref(ms)), "ne_ctx_last_run_ms")
    return ms.value


def ne_ctx_crystal_plan(ctx):
    """Launch plan of the last crystal-runner call: dict with runner
    ("cluster" or "brick"), threads_per_atom, ctas and cluster_ctas."""
    r, t, n, c = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _err(ctx, load().ne_ctx_crystal_plan(ctx, C.byref(r), C.byref(t), C.byref(n), C.byref(c)), "ne_ctx_crystal_plan")
    return {"runner": "cluster" if r.value == 1 else "brick", "threads_per_atom": t.value, "ctas": n.value,
            "cluster_ctas": c.value}


def ne_last_error(ctx):
    buf = C.create_string_buffer(256)
    st = C.c_int()
    load().ne_last_error(ctx, C.byref(st), buf, 256)
    return st.value, buf.value.decode()


def ne_create_crystal(lattice, a, nx, ny, nz, c_over_a=None):
    """Host: returns (x0 numpy [n][3], box numpy [3]); hcp with c = c_over_a * a
    (ne_create_crystal_ca) or the ideal axial ratio."""
    import numpy as np
    n = C.c_int()
    box = (C.c_double * 3)()
    L = load()
    if c_over_a is None:
        def call(ptr):
            return L.ne_create_crystal(int(lattice), float(a), nx, ny, nz, ptr, box, C.byref(n))
    else:
        def call(ptr):
            return L.ne_create_crystal_ca(int(lattice), float(a), float(c_over_a), nx, ny, nz, ptr, box, C.byref(n))
    _err(None, call(None), "ne_create_crystal")
    x0 = np.zeros((n.value, 3))
    _err(None, call(x0.ctypes.data_as(C.c_void_p)), "ne_create_crystal")
    return x0, np.array(list(box))


def ne_eam_energy_forces(ctx, prec, x, box, f=None, e=None, rho=None, stream=None):
    n = x.shape[0]
    _err(ctx, load().ne_eam_energy_forces(ctx, int(prec), _dev(x, 3 * n), n, _box(box),
                                          _dev(f, 3 * n), _dev(e, 1), _dev(rho, n),
                                          _stream(stream)), "ne_eam_energy_forces")


def ne_eam_virial(ctx, x, box, w, stream=None):
    """Configurational virial W = -dU/d(eps) (FP64) into the 1-element device tensor w."""
    n = x.shape[0]
    _err(ctx, load().ne_eam_virial(ctx, _dev(x, 3 * n), n, _box(box), _dev(w, 1), _stream(stream)),
         "ne_eam_virial")


NE_NOALLOC_MAX_ATOMS = 2048


def ne_eam_energy_forces_noalloc(eam: EamParams, prec, x, box, f=None, e=None, stream=None):
    """EAM energy/forces with no device allocation (scratch in a static
    device array of the library; n <= NE_NOALLOC_MAX_ATOMS)."""
    n = x.shape[0]
    _err(None, load().ne_eam_energy_forces_noalloc(C.byref(eam), int(prec), _dev(x, 3 * n), n,
                                                   _box(box), _dev(f, 3 * n), _dev(e, 1),
                                                   _stream(stream)),
         "ne_eam_energy_forces_noalloc")


def ne_spring_forces(x, x0, k, f=None, e=None, stream=None):
    n = x.shape[0]
    _err(None, load().ne_spring_forces(_dev(x, 3 * n), _dev(x0, 3 * n), n, float(k),
                                       _dev(f, 3 * n), _dev(e, 1), _stream(stream)),
         "ne_spring_forces")


def ne_eam_backward(ctx, prec, x, box, gE, gx, gtheta, stream=None):
    n = x.shape[0]
    _err(ctx, load().ne_eam_backward(ctx, int(prec), _dev(x, 3 * n), n, _box(box), float(gE),
                                     _dev(gx, 3 * n), _dev(gtheta, _knots6(ctx)), _stream(stream)),
         "ne_eam_backward")


def ne_eam_backward_acc(ctx, prec, x, box, gE, gtheta_acc, stream=None):
    """gtheta_acc += gE dU/dtheta at configuration x (device tensors)."""
    n = x.shape[0]
    _err(ctx, load().ne_eam_backward_acc(ctx, int(prec), _dev(x, 3 * n), n, _box(box), float(gE),
                                         _dev(gtheta_acc, _knots6(ctx)), _stream(stream)), "ne_eam_backward_acc")


def ne_noise(seed, replica, noise_stream, step, z, prec=NE_FP64, stream=None):
    n = z.shape[0]
    _err(None, load().ne_noise(int(seed), int(replica), int(noise_stream), int(step), n, int(prec),
                               _dev(z, 3 * n), _stream(stream)), "ne_noise")


def ne_init_velocities(ctx, md: MdParams, v, stream=None):
    n = v.shape[0]
    _err(ctx, load().ne_init_velocities(ctx, C.byref(md), n, _dev(v, 3 * n), _stream(stream)),
         "ne_init_velocities")


def ne_langevin_step(ctx, md: MdParams, x, v, x0, box, step, lambda_k, lambda_k1, W=None,
                     stream=None):
    n = x.shape[0]
    _err(ctx, load().ne_langevin_step(ctx, C.byref(md), _dev(x, 3 * n), _dev(v, 3 * n),
                                      _dev(x0, 3 * n), n, _box(box), int(step), float(lambda_k),
                                      float(lambda_k1), _dev(W, 1), _stream(stream)),
         "ne_langevin_step")


def ne_switch_run(ctx, md: MdParams, x, v, x0, box, W_fwd, W_bwd, Wcum_fwd=None, Wcum_bwd=None,
                  trace=None, trace_stride=0, stream=None):
    n = x.shape[0]
    ncum = int(md.t_s) + 1
    _err(ctx, load().ne_switch_run(ctx, C.byref(md), _dev(x, 3 * n), _dev(v, 3 * n),
                                   _dev(x0, 3 * n), n, _box(box), _dev(W_fwd, 1), _dev(W_bwd, 1),
                                   _dev(Wcum_fwd, ncum), _dev(Wcum_bwd, ncum),
                                   _dev(trace, 8 * _trace_rows(md, trace_stride)), int(trace_stride),
                                   _stream(stream)), "ne_switch_run")


def ne_rs_run(ctx, md: MdParams, lambda_f, x, v, x0, box, Wcum_fwd, Wcum_bwd, stream=None):
    n = x.shape[0]
    _err(ctx, load().ne_rs_run(ctx, C.byref(md), float(lambda_f), _dev(x, 3 * n), _dev(v, 3 * n),
                               _dev(x0, 3 * n), n, _box(box), _dev(Wcum_fwd, int(md.t_s) + 1),
                               _dev(Wcum_bwd, int(md.t_s) + 1), _stream(stream)), "ne_rs_run")


def _batch_args(mds, offsets, boxes):
    """(n_rep, md array, offsets array, boxes array, 3 * atoms) of a batch."""
    n_rep = len(mds)
    n_atoms = _batch_atoms(offsets, n_rep)
    if len(boxes) != n_rep or any(len(b) != 3 for b in boxes):
        raise NeError(NE_EINVAL, "argument", "one box of 3 edges per replica")
    arr = (MdParams * n_rep)(*mds)
    off = (C.c_int * (n_rep + 1))(*[int(o) for o in offsets])
    flat = [float(b) for bx in boxes for b in bx]
    return n_rep, arr, off, (C.c_double * len(flat))(*flat), 3 * n_atoms


def ne_switch_run_batched(ctx, mds, offsets, x, v, x0, boxes, W_fwd, W_bwd, stream=None):
    n_rep, arr, off, bx, n3 = _batch_args(mds, offsets, boxes)
    _err(ctx, load().ne_switch_run_batched(ctx, arr, n_rep, off, _dev(x, n3), _dev(v, n3), _dev(x0, n3), bx,
                                           _dev(W_fwd, n_rep), _dev(W_bwd, n_rep),
                                           _stream(stream)), "ne_switch_run_batched")


def ne_switch_run_segment(ctx, mds, offsets, x, v, x0, boxes, W, step_begin, n_steps, stream=None):
    n_rep, arr, off, bx, n3 = _batch_args(mds, offsets, boxes)
    _err(ctx, load().ne_switch_run_segment(ctx, arr, n_rep, off, _dev(x, n3), _dev(v, n3), _dev(x0, n3), bx,
                                           _dev(W, 2 * n_rep), int(step_begin), int(n_steps),
                                           _stream(stream)), "ne_switch_run_segment")


def ne_switch_run_segment_cum(ctx, mds, offsets, x, v, x0, boxes, W, Wcum, step_begin, n_steps, stream=None):
    """ne_switch_run_segment plus the cumulative works Wcum [n_rep][2][t_s + 1]."""
    n_rep, md_arr, off, bx, n3 = _batch_args(mds, offsets, boxes)
    _err(ctx, load().ne_switch_run_segment_cum(ctx, md_arr, n_rep, off, _dev(x, n3), _dev(v, n3), _dev(x0, n3), bx,
                                               _dev(W, 2 * n_rep), _dev(Wcum, n_rep * 2 * (int(mds[0].t_s) + 1)),
                                               int(step_begin), int(n_steps), _stream(stream)),
         "ne_switch_run_segment_cum")


def ne_switch_run_segment_grad(ctx, mds, offsets, x, v, x0, boxes, W, step_begin, n_steps, w, gtheta, stream=None):
    """ne_switch_run_segment plus gtheta += sum_k w[k - step_begin] dU/dtheta(x_k)
    (w: device float64 [n_steps + 1]; gtheta: device float64 [3 * n_knots * 2])."""
    n_rep, arr, off, bx, n3 = _batch_args(mds, offsets, boxes)
    _err(ctx, load().ne_switch_run_segment_grad(ctx, arr, n_rep, off, _dev(x, n3), _dev(v, n3), _dev(x0, n3), bx,
                                                _dev(W, 2 * n_rep), int(step_begin), int(n_steps),
                                                _dev(w, int(n_steps) + 1), _dev(gtheta, _knots6(ctx)),
                                                _stream(stream)),
         "ne_switch_run_segment_grad")


def ne_profile_segment(ctx, mds, offsets, x, v, x0, boxes, W, step_begin, n_steps, stream=None):
    """Returns (mean ms per launch [4], launches [4]) for list build, pass 1,
    pass 2 and the fused step."""
    n_rep, arr, off, bx, n3 = _batch_args(mds, offsets, boxes)
    ms = (C.c_double * 4)()
    cnt = (C.c_longlong * 4)()
    _err(ctx, load().ne_profile_segment(ctx, arr, n_rep, off, _dev(x, n3), _dev(v, n3), _dev(x0, n3), bx,
                                        _dev(W, 2 * n_rep), int(step_begin), int(n_steps), ms, cnt,
                                        _stream(stream)), "ne_profile_segment")
    return list(ms), list(cnt)


class CrystalBatch:
    """The md and crystal arrays of a crystal-runner batch, packed once for
    repeated ne_crystal_run_segment calls (pass it as `mds`, crystals=None)."""

    def __init__(self, mds, crystals):
        self.n_rep = len(mds)
        self.md = (MdParams * self.n_rep)(*mds)
        self.cr = (Crystal * self.n_rep)(*[Crystal(int(c[0]), float(c[1]), int(c[2]), int(c[3]), int(c[4]),
                                                   float(c[5]) if len(c) > 5 else 0.0) for c in crystals])
        self.n3 = 3 * _crystal_atoms(crystals)


def ne_crystal_run_segment(ctx, mds, crystals, x, v, W, step_begin, n_steps, stream=None):
    """crystals: list of (lattice, a, nx, ny, nz[, c_over_a]); or mds a
    CrystalBatch and crystals None."""
    b = mds if isinstance(mds, CrystalBatch) else CrystalBatch(mds, crystals)
    _err(ctx, load().ne_crystal_run_segment(ctx, b.md, b.cr, b.n_rep, _dev(x, b.n3), _dev(v, b.n3),
                                            _dev(W, 2 * b.n_rep), int(step_begin), int(n_steps),
                                            _stream(stream)),
         "ne_crystal_run_segment")


def ne_crystal_run_segment_cum(ctx, mds, crystals, x, v, W, Wcum, step_begin, n_steps, stream=None):
    """ne_crystal_run_segment plus the cumulative works Wcum [n_rep][2][t_s + 1]."""
    n_rep = len(mds)
    arr = (MdParams * n_rep)(*mds)
    cr = (Crystal * n_rep)(*[Crystal(int(c[0]), float(c[1]), int(c[2]), int(c[3]), int(c[4]),
                                     float(c[5]) if len(c) > 5 else 0.0) for c in crystals])
    n3 = 3 * _crystal_atoms(crystals)
    _err(ctx, load().ne_crystal_run_segment_cum(ctx, arr, cr, n_rep, _dev(x, n3), _dev(v, n3), _dev(W, 2 * n_rep),
                                                _dev(Wcum, n_rep * 2 * (int(mds[0].t_s) + 1)),
                                                int(step_begin), int(n_steps), _stream(stream)),
         "ne_crystal_run_segment_cum")


def ne_msd_fit(ctx, md: MdParams, x, v, x0, box, n_eq, n_samples, stride, stream=None):
    n = x.shape[0]
    msd, k = C.c_double(), C.c_double()
    _err(ctx, load().ne_msd_fit(ctx, C.byref(md), _dev(x, 3 * n), _dev(v, 3 * n),
                                _dev(x0, 3 * n), n, _box(box), int(n_eq), int(n_samples),
                                int(stride), C.byref(msd), C.byref(k), _stream(stream)),
         "ne_msd_fit")
    return msd.value, k.value


def ne_msd_fit_species(ctx, md: MdParams, x, v, x0, box, n_eq, n_samples, stride, stream=None):
    """Per-species (msd_s, k_s) numpy arrays of a replica with species tables."""
    import numpy as np
    n = x.shape[0]
    msd = np.zeros(md.n_species)
    k = np.zeros(md.n_species)
    _err(ctx, load().ne_msd_fit_species(ctx, C.byref(md), _dev(x, 3 * n), _dev(v, 3 * n), _dev(x0, 3 * n), n,
                                        _box(box), int(n_eq), int(n_samples), int(stride),
                                        msd.ctypes.data_as(C.c_void_p), k.ctypes.data_as(C.c_void_p),
                                        _stream(stream)),
         "ne_msd_fit_species")
    return msd, k


def ne_msd_fit_batched(ctx, mds, offsets, x, v, x0, boxes, n_eq, n_samples, stride, stream=None):
    """Per-replica (msd, k) of a batch (numpy arrays of n_rep)."""
    import numpy as np
    n_rep = len(mds)
    arr = (MdParams * n_rep)(*mds)
    off = (C.c_int * (n_rep + 1))(*[int(o) for o in offsets])
    n3 = 3 * _batch_atoms(offsets, n_rep)
    bx = (C.c_double * (3 * n_rep))(*[float(b) for box in boxes for b in box])
    msd = np.zeros(n_rep)
    k = np.zeros(n_rep)
    _err(ctx, load().ne_msd_fit_batched(ctx, arr, n_rep, off, _dev(x, n3), _dev(v, n3), _dev(x0, n3), bx,
                                        int(n_eq), int(n_samples), int(stride), msd.ctypes.data_as(C.c_void_p),
                                        k.ctypes.data_as(C.c_void_p), _stream(stream)),
         "ne_msd_fit_batched")
    return msd, k


def ne_free_energy(n, V, T, mass, k, W_fwd, W_bwd):
    import numpy as np
    wf = np.ascontiguousarray(W_fwd, np.float64).ravel()
    wb = np.ascontiguousarray(W_bwd, np.float64).ravel()
    F, se, ed = C.c_double(), C.c_double(), C.c_double()
    _err(None, load().ne_free_energy(int(n), float(V), float(T), float(mass), float(k),
                                     wf.ctypes.data_as(C.c_void_p), wb.ctypes.data_as(C.c_void_p),
                                     wf.size, C.byref(F), C.byref(se), C.byref(ed)),
         "ne_free_energy")
    return F.value, se.value, ed.value


def ne_free_energy_species(species, mass_s, k_s, V, T, W_fwd, W_bwd):
    """Eq. fl + eq. cm with one mass and one spring per species (Sec. V);
    species [n] ints, mass_s and k_s [n_species]."""
    import numpy as np
    sp = np.ascontiguousarray(species, np.int32).ravel()
    ms = np.ascontiguousarray(mass_s, np.float64).ravel()
    ks = np.ascontiguousarray(k_s, np.float64).ravel()
    if ms.size != ks.size:
        raise ValueError("mass_s and k_s need one entry per species")
    wf = np.ascontiguousarray(W_fwd, np.float64).ravel()
    wb = np.ascontiguousarray(W_bwd, np.float64).ravel()
    if wf.size != wb.size:
        raise ValueError("W_fwd and W_bwd need one entry per seed")
    F, se, ed = C.c_double(), C.c_double(), C.c_double()
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)
    _err(None, load().ne_free_energy_species(sp.size, ptr(sp), ms.size, ptr(ms), ptr(ks), float(V), float(T),
                                             ptr(wf), ptr(wb), wf.size, C.byref(F), C.byref(se),
                                             C.byref(ed)), "ne_free_energy_species")
    return F.value, se.value, ed.value


def ne_lambda(md: MdParams, step):
    """Lambda in force at the start of `step` of md's four-phase schedule."""
    lam = C.c_double()
    _err(None, load().ne_lambda(C.byref(md), int(step), C.byref(lam)), "ne_lambda")
    return lam.value


def ne_pressure(n_dof, T, V, W):
    """(P, standard error) in eV/A^3 from virial samples W (eV)."""
    import numpy as np
    w = np.ascontiguousarray(np.atleast_1d(W), np.float64).ravel()
    P, se = C.c_double(), C.c_double()
    _err(None, load().ne_pressure(int(n_dof), float(T), float(V), w.ctypes.data_as(C.c_void_p), w.size,
                                  C.byref(P), C.byref(se)), "ne_pressure")
    return P.value, se.value


def ne_jarzynski(T, W):
    """-k_B T ln mean exp(-W / k_B T) (eq. jarz); W: works done on the system (eV)."""
    import numpy as np
    w = np.ascontiguousarray(W, np.float64).ravel()
    out = C.c_double()
    _err(None, load().ne_jarzynski(float(T), w.ctypes.data_as(C.c_void_p), w.size, C.byref(out)), "ne_jarzynski")
    return out.value


def ne_rs_free_energy(n, T0, F0_T0, lambda_f, t_s, Wcum_fwd, Wcum_bwd, T_grid):
    import numpy as np
    cf = np.ascontiguousarray(np.atleast_2d(Wcum_fwd), np.float64)
    cb = np.ascontiguousarray(np.atleast_2d(Wcum_bwd), np.float64)
    tg = np.ascontiguousarray(T_grid, np.float64)
    out = np.zeros(tg.size)
    _err(None, load().ne_rs_free_energy(int(n), float(T0), float(F0_T0), float(lambda_f),
                                        int(t_s), cf.ctypes.data_as(C.c_void_p),
                                        cb.ctypes.data_as(C.c_void_p), cf.shape[0],
                                        tg.ctypes.data_as(C.c_void_p), tg.size,
                                        out.ctypes.data_as(C.c_void_p)), "ne_rs_free_energy")
    return out


# ------------------------------------------------------------------ autograd
def eam_energy_function():
    """torch.autograd.Function whose forward is ne_eam_energy_forces and whose
    backward is ne_eam_backward: EAMEnergy.apply(x, theta, ctx, box, prec) -> U."""
    torch = _torch()

    class EAMEnergy(torch.autograd.Function):
        @staticmethod
        def forward(fctx, x, theta, ctx, box, prec):
            ne_ctx_set_theta(ctx, theta.detach().contiguous())
            e = torch.zeros(1, dtype=torch.float64, device=x.device)
            ne_eam_energy_forces(ctx, prec, x.detach().contiguous(), box, e=e)
            fctx.save_for_backward(x, theta)
            fctx.ne = (ctx, tuple(box), prec)
            return e[0]

        @staticmethod
        def backward(fctx, gE):
            x, theta = fctx.saved_tensors
            ctx, box, prec = fctx.ne
            ne_ctx_set_theta(ctx, theta.detach().contiguous())
            gx = torch.empty_like(x, memory_format=torch.contiguous_format)
            gth = torch.empty_like(theta, memory_format=torch.contiguous_format)
            ne_eam_backward(ctx, prec, x.detach().contiguous(), box, float(gE), gx, gth)
            return gx, gth, None, None, None

    return EAMEnergy
