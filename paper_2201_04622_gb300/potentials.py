"""EAM potentials from tabulated files, for a user-supplied potential in place
of the analytic Fe-like one (the paper's runs use a published EAM for Fe,
Sec. III.A, read by LAMMPS from such a file).

Two plain-text formats are read, both single-element:

- funcfl: comment line; atomic number, mass, lattice constant, lattice type;
  Nrho, drho, Nr, dr, cutoff; then F(rho) at rho = k drho (Nrho values),
  Z(r) at r = k dr (Nr values) and the density f(r) at the same r (Nr
  values).  The pair term is phi(r) = 27.2 * 0.529 * Z(r)^2 / r (Hartree and
  Bohr in eV and A, the values that format assumes).
- setfl with one element: three comment lines; "1 <element>"; Nrho, drho,
  Nr, dr, cutoff; atomic number, mass, lattice constant, lattice type;
  F(rho) (Nrho values), f(r) (Nr values), then r * phi(r) (Nr values).
  A single-element Finnis-Sinclair file (one density function per element
  pair, so one in all) has the same layout and is read the same way.

Numbers may be spread over lines in any way.  The tables are interpolated
with not-a-knot cubic splines (scipy) and resampled onto the library's
knots: value and slope of phi and f at n_knots uniform points of [0, r_c]
and of F on [0, rho_max], rho_max the last tabulated density.  phi is
singular at r = 0; below the first positive grid point its knots repeat the
value there with zero slope (the library rejects pairs closer than 0.2 A).

load_eam(path) returns the parameter block for ne_ctx_create (r_c, rho_max
and n_knots set; the analytic fields are placeholders, replaced as soon as
the knots are loaded) and theta [3][n_knots][2] for ne_ctx_set_theta and the
oracle.  ne_eam_energy_forces_noalloc builds its tables from the analytic
parameters on every call and cannot take loaded knots.
"""
from __future__ import annotations

import numpy as np

HARTREE_BOHR = 27.2 * 0.529  # eV A: phi = HARTREE_BOHR * Z^2 / r in funcfl files


def _numbers(lines):
    out = []
    for ln in lines:
        out.extend(ln.replace("D", "E").replace("d", "e").split())
    return out


def read_eam(path):
    """Parse a funcfl or single-element setfl file into tabulated functions:
    dict(r, rho, F, f, rphi, cutoff, mass_amu, element)."""
    with open(path) as fh:
        lines = fh.read().splitlines()
    if len(lines) < 4:
        raise ValueError("%s: too short for an EAM file" % path)
    # setfl: line 4 holds the element count followed by that many names
    head4 = lines[3].split() if len(lines) > 3 else []
    if head4 and head4[0].isdigit() and len(head4) == int(head4[0]) + 1:
        n_el = int(head4[0])
        if n_el != 1:
            raise ValueError("%s: %d elements; only single-element files are read" % (path, n_el))
        grid = lines[4].split()
        nrho, drho, nr, dr, cutoff = int(grid[0]), float(grid[1]), int(grid[2]), float(grid[3]), float(grid[4])
        el = lines[5].split()
        mass = float(el[1])
        vals = np.array([float(t) for t in _numbers(lines[6:])])
        need = nrho + 2 * nr
        if vals.size < need:
            raise ValueError("%s: %d table values, %d expected" % (path, vals.size, need))
        F = vals[:nrho]
        f = vals[nrho:nrho + nr]
        rphi = vals[nrho + nr:nrho + 2 * nr]
        element = head4[1]
    else:
        el = lines[1].split()
        mass = float(el[1])
        grid = lines[2].split()
        nrho, drho, nr, dr, cutoff = int(grid[0]), float(grid[1]), int(grid[2]), float(grid[3]), float(grid[4])
        vals = np.array([float(t) for t in _numbers(lines[3:])])
        need = nrho + 2 * nr
        if vals.size < need:
            raise ValueError("%s: %d table values, %d expected" % (path, vals.size, need))
        F = vals[:nrho]
        Z = vals[nrho:nrho + nr]
        f = vals[nrho + nr:nrho + 2 * nr]
        rphi = HARTREE_BOHR * Z * Z
        element = el[0]
    if nrho < 4 or nr < 4 or not (drho > 0 and dr > 0 and cutoff > 0):
        raise ValueError("%s: bad grid (Nrho %d, drho %g, Nr %d, dr %g, cutoff %g)" % (path, nrho, drho, nr, dr, cutoff))
    return dict(r=dr * np.arange(nr), rho=drho * np.arange(nrho), F=F, f=f, rphi=rphi, cutoff=cutoff,
                mass_amu=mass, element=element)


def theta_from_tables(tab, n_knots=5000):
    """Resample tabulated functions onto the library's knots; returns
    (r_c, rho_max, theta [3][n_knots][2])."""
    from scipy.interpolate import CubicSpline
    r, rho = tab["r"], tab["rho"]
    r_c = min(tab["cutoff"], r[-1])
    rho_max = rho[-1]
    rk = np.linspace(0.0, r_c, n_knots)
    pk = np.linspace(0.0, rho_max, n_knots)
    theta = np.zeros((3, n_knots, 2))
    # phi from r * phi: spline r phi, then phi = (r phi)/r, phi' = ((r phi)' - phi)/r
    pos = r > 0
    s_rphi = CubicSpline(r[pos], tab["rphi"][pos])
    r0 = r[pos][0]
    inside = rk >= r0
    rphi, drphi = s_rphi(rk[inside]), s_rphi(rk[inside], 1)
    phi = rphi / rk[inside]
    theta[0, inside, 0] = phi
    theta[0, inside, 1] = (drphi - phi) / rk[inside]
    theta[0, ~inside, 0] = phi[0]
    theta[0, ~inside, 1] = 0.0
    s_f = CubicSpline(r, tab["f"])
    theta[1, :, 0], theta[1, :, 1] = s_f(rk), s_f(rk, 1)
    s_F = CubicSpline(rho, tab["F"])
    theta[2, :, 0], theta[2, :, 1] = s_F(pk), s_F(pk, 1)
    return r_c, rho_max, theta


def load_eam(path, n_knots=5000):
    """(eam parameter dict for ne.eam_params / oracle.eam, theta, mass in u)
    of a funcfl or single-element setfl file.

    The potential is theta; the dict carries the knot grid (r_c, rho_max,
    n_knots) and NaN in place of the analytic parameters A, alpha, beta, B,
    so a context made from it gives non-finite energies (NE_ENAN) until
    ne_ctx_set_theta installs theta, and the allocation-free entry point,
    which tabulates the analytic form only, refuses it (NE_EINVAL).
    context_from_file does both steps at once."""
    tab = read_eam(path)
    r_c, rho_max, theta = theta_from_tables(tab, n_knots)
    nan = float("nan")
    params = dict(A=nan, alpha=nan, beta=nan, B=nan, r_e=1.0, r_s=0.5 * r_c, r_c=r_c, rho_max=rho_max,
                  n_knots=n_knots)
    return params, theta, tab["mass_amu"]


def context_from_file(path, max_atoms, max_replicas=1, n_knots=5000, device="cuda"):
    """A library context holding the potential of a funcfl or single-element
    setfl file: ne_ctx_create on the file's knot grid, then ne_ctx_set_theta
    with its knots.  Returns (ctx, mass in u)."""
    import torch
    from . import ne
    params, theta, mass = load_eam(path, n_knots)
    ctx = ne.ne_ctx_create(ne.eam_params(**params), max_atoms, max_replicas)
    try:
        ne.ne_ctx_set_theta(ctx, torch.tensor(theta.reshape(-1), dtype=torch.float64, device=device))
        torch.cuda.synchronize()
    except Exception:
        ne.ne_ctx_destroy(ctx)
        raise
    return ctx, mass
