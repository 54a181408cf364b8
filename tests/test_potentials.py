"""Tabulated EAM files (funcfl, single-element setfl) read into the library's
knot tables, on the CPU.  Files written here from the analytic Fe-like
potential must give, through the oracle, the energies and forces of the
analytic knots to interpolation accuracy."""
import numpy as np
import pytest

import oracle as O
from paper_2201_04622_gb300 import potentials as P
from paper_2201_04622_gb300 import workloads as W


def _analytic(p, which, x):
    return np.array([O.eam_analytic(p, which, float(t))[0] for t in x])


def _write(path, lines, values, per_line=5):
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
        for i in range(0, len(values), per_line):
            fh.write(" ".join("%.16e" % v for v in values[i:i + per_line]) + "\n")


def _tables(nr=20000, nrho=20000):
    p = O.eam(**W.EAM_FE_LIKE)
    r_c, rho_max = W.EAM_FE_LIKE["r_c"], W.EAM_FE_LIKE["rho_max"]
    dr, drho = r_c / (nr - 1), rho_max / (nrho - 1)
    r, rho = dr * np.arange(nr), drho * np.arange(nrho)
    return p, r, rho, dr, drho, _analytic(p, 2, rho), _analytic(p, 1, r), r * _analytic(p, 0, r)


def write_setfl(path, nr=20000, nrho=20000):
    p, r, rho, dr, drho, F, f, rphi = _tables(nr, nrho)
    head = ["analytic Fe-like EAM", "written by the test-suite", "single element",
            "1 Fe", "%d %.16e %d %.16e %.16e" % (nrho, drho, nr, dr, W.EAM_FE_LIKE["r_c"]),
            "26 55.845 2.87 bcc"]
    _write(path, head, np.concatenate([F, f, rphi]))


def write_funcfl(path, nr=20000, nrho=20000):
    p, r, rho, dr, drho, F, f, rphi = _tables(nr, nrho)
    Z = np.sqrt(np.maximum(rphi, 0.0) / P.HARTREE_BOHR)
    head = ["analytic Fe-like EAM (funcfl)", "26 55.845 2.87 bcc",
            "%d %.16e %d %.16e %.16e" % (nrho, drho, nr, dr, W.EAM_FE_LIKE["r_c"])]
    _write(path, head, np.concatenate([F, Z, f]))


@pytest.mark.parametrize("fmt", ["setfl", "funcfl"])
def test_file_potential_reproduces_the_analytic_one(tmp_path, fmt):
    path = str(tmp_path / ("fe." + fmt))
    (write_setfl if fmt == "setfl" else write_funcfl)(path)
    params, theta, mass = P.load_eam(path)
    assert mass == 55.845 and params["r_c"] == W.EAM_FE_LIKE["r_c"]
    assert params["rho_max"] == pytest.approx(W.EAM_FE_LIKE["rho_max"], rel=1e-14)
    p = O.eam(**W.EAM_FE_LIKE)
    th = O.eam_theta(p)
    # knots where the library evaluates: pairs beyond 0.2 A, densities away from the sqrt at 0
    rk = np.linspace(0.0, params["r_c"], params["n_knots"])
    use = rk >= 0.2
    for which in (0, 1):
        assert np.allclose(theta[which, use, 0], th[which, use, 0], rtol=1e-9, atol=1e-11)
        assert np.allclose(theta[which, use, 1], th[which, use, 1], rtol=1e-6, atol=1e-8)
    pk = np.linspace(0.0, params["rho_max"], params["n_knots"])
    dense = pk >= 1.0
    assert np.allclose(theta[2, dense, 0], th[2, dense, 0], rtol=1e-10)
    assert np.allclose(theta[2, dense, 1], th[2, dense, 1], rtol=1e-7)
    # energies and forces of a hot, displaced crystal through the oracle
    pf = O.eam(**params)
    x0, box = O.create_crystal(O.BCC, W.A_BCC, 5, 5, 5)
    x = W.displaced(x0, 0.25, 31)
    E0, f0, rho0 = O.eam_energy_forces(p, th, x, box)
    E1, f1, rho1 = O.eam_energy_forces(pf, theta.reshape(-1), x, box)
    assert rho1.min() > 1.0
    assert E1 == pytest.approx(E0, rel=1e-10)
    assert np.abs(f1 - f0).max() < 1e-7 * np.abs(f0).max()


def test_malformed_and_multi_element_files_are_rejected(tmp_path):
    short = tmp_path / "short.eam"
    short.write_text("comment\n26 55.845 2.87 bcc\n100 0.01 100 0.05 5.0\n1 2 3\n")
    with pytest.raises(ValueError, match="table values"):
        P.read_eam(str(short))
    two = tmp_path / "alloy.setfl"
    two.write_text("c1\nc2\nc3\n2 Fe Ni\n10 0.1 10 0.5 5.0\n" + "0 " * 100 + "\n")
    with pytest.raises(ValueError, match="single-element"):
        P.read_eam(str(two))


def test_file_potential_placeholders_are_refused_by_the_analytic_entry_point(tmp_path):
    """A potential loaded from a file carries NaN analytic parameters, so the
    allocation-free entry point (it tabulates the analytic form only) refuses
    it before touching the device (the pointers are never dereferenced)."""
    import ctypes as C
    from paper_2201_04622_gb300 import ne
    path = tmp_path / "fe.eam"
    write_funcfl(str(path), nr=2000, nrho=2000)
    params, _, _ = P.load_eam(str(path))
    assert all(np.isnan(params[k]) for k in ("A", "alpha", "beta", "B"))
    L = ne.load()
    box = (C.c_double * 3)(30.0, 30.0, 30.0)
    e_ = ne.eam_params(**params)
    assert L.ne_eam_energy_forces_noalloc(C.byref(e_), ne.NE_FP64, C.c_void_p(256), 128, box,
                                          C.c_void_p(256), C.c_void_p(256), None) == ne.NE_EINVAL
