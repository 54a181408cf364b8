/*
 * ne_oracle.c -- plain FP64 CPU oracle of nonequilibrium free-energy switching
 * MD (Freitas, Asta & de Koning, "Nonequilibrium free-energy calculation of
 * solids using LAMMPS").
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test-suite, the package smoke check
 * and the CPU-baseline leg of the benchmark, never by the product path.  It
 * shares no code with the CUDA library.  Every routine follows the paper's
 * definitions in its order and notation, one plain loop at a time; nothing is
 * blocked, fused or reordered for speed.
 *
 * Where the paper is silent (the interatomic potential, the spline form, the
 * random-number layout, the exact step order) the readings are written next
 * to the code that adopts them.
 */
#include "ne_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- constants */
/* Metal units.  k_B and hbar are the CODATA-2018 values; the mass unit is
 * derived from the SI values of the atomic mass unit and the electronvolt. */
static const double KB_EV_PER_K = 8.617333262e-5;
static const double HBAR_EV_PS = 6.582119569e-4;
static const double AMU_KG = 1.66053906660e-27;
static const double EV_J = 1.602176634e-19;
/* 1 eV ps^2 / A^2 expressed in kg: 1 eV * (1e-12 s)^2 / (1e-10 m)^2. */
static const double EV_PS2_PER_A2_KG = 1.602176634e-19 * 1.0e-4;
/* A: shorter pair distances are an error.  Near lambda = 1 of the
 * Frenkel-Ladd path the crystal is a set of independent Einstein oscillators
 * (Sec. II.B, eq. einstein) whose atoms may overlap, and the tables cover
 * [0, r_c]; only near-coincident atoms are rejected. */
static const double R_MIN = 0.2;

double ora_kB(void) { return KB_EV_PER_K; }
double ora_hbar(void) { return HBAR_EV_PS; }
double ora_amu(void) { (void)EV_J; return AMU_KG / EV_PS2_PER_A2_KG; }

/* ------------------------------------------------------------------ crystal */
/* Lattice sites r0 of a bcc or fcc supercell (the Einstein-crystal anchor
 * points of Sec. II.B, eq. einstein).  Atom order: ((ix*ny+iy)*nz+iz)*nb+b. */
/* Orthorhombic supercells of cubic bcc and fcc cells (edge a) and of the
 * orthohexagonal hcp cell (edges a, sqrt(3) a, c) with its four atoms:
 * A layer at (0,0,0), (1/2,1/2,0); B layer above the triangle centres at
 * (0,1/3,1/2), (1/2,5/6,1/2) (fractions of the cell edges). */
int ora_create_crystal_ca(int lattice, double a, double c_over_a, int nx, int ny, int nz,
                          double* x0, double box[3], int* n_out)
{
    static const double bcc[2][3] = {{0, 0, 0}, {0.5, 0.5, 0.5}};
    static const double fcc[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
    static const double hcp[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0, 1.0 / 3.0, 0.5}, {0.5, 5.0 / 6.0, 0.5}};
    const double(*basis)[3];
    int nb;
    double cell[3] = {a, a, a};
    if (lattice == ORA_BCC) { basis = bcc; nb = 2; }
    else if (lattice == ORA_FCC) { basis = fcc; nb = 4; }
    else if (lattice == ORA_HCP) {
        if (!(c_over_a > 0)) return ORA_EINVAL;
        basis = hcp;
        nb = 4;
        cell[1] = sqrt(3.0) * a;
        cell[2] = c_over_a * a;
    } else return ORA_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || !(a > 0)) return ORA_EINVAL;
    int i = 0;
    for (int ix = 0; ix < nx; ix++)
        for (int iy = 0; iy < ny; iy++)
            for (int iz = 0; iz < nz; iz++)
                for (int b = 0; b < nb; b++) {
                    if (x0) {
                        x0[3 * i + 0] = cell[0] * (ix + basis[b][0]);
                        x0[3 * i + 1] = cell[1] * (iy + basis[b][1]);
                        x0[3 * i + 2] = cell[2] * (iz + basis[b][2]);
                    }
                    i++;
                }
    if (box) { box[0] = cell[0] * nx; box[1] = cell[1] * ny; box[2] = cell[2] * nz; }
    if (n_out) *n_out = i;
    return ORA_OK;
}

int ora_create_crystal(int lattice, double a, int nx, int ny, int nz,
                       double* x0, double box[3], int* n_out)
{
    return ora_create_crystal_ca(lattice, a, sqrt(8.0 / 3.0), nx, ny, nz, x0, box, n_out);
}

/* ------------------------------------------------------------ analytic EAM */
/* Quintic taper, 1 below r_s and 0 above r_c, continuous to 2nd derivative. */
static void taper(const ora_eam* p, double r, double* s, double* ds)
{
    if (r <= p->r_s) { *s = 1.0; *ds = 0.0; return; }
    if (r >= p->r_c) { *s = 0.0; *ds = 0.0; return; }
    double w = p->r_c - p->r_s;
    double x = (r - p->r_s) / w;
    double om = 1.0 - x;
    *s = om * om * om * (1.0 + 3.0 * x + 6.0 * x * x);
    *ds = -30.0 * x * x * om * om / w;
}

/* phi(r) = A exp(-alpha (r/r_e - 1)) s(r);  f(r) = exp(-beta (r/r_e - 1)) s(r);
 * F(rho) = -B sqrt(rho).  The EAM energy U of eq. H (Sec. II.B). */
void ora_eam_analytic(const ora_eam* p, int which, double x, double* y, double* dy)
{
    if (which == 2) {
        *y = -p->B * sqrt(x);
        *dy = x > 0 ? -0.5 * p->B / sqrt(x) : -INFINITY;
        return;
    }
    double s, ds;
    taper(p, x, &s, &ds);
    double c = which == 0 ? p->alpha : p->beta;
    double amp = which == 0 ? p->A : 1.0;
    double e = amp * exp(-c * (x / p->r_e - 1.0));
    *y = e * s;
    *dy = e * (-c / p->r_e) * s + e * ds;
}

/* Knot parameters theta = (value, slope) at n_knots uniform knots: phi and f
 * on [0, r_c], F on [0, rho_max].  The embedding slope is infinite at rho = 0;
 * that one knot takes the secant slope to the next knot. */
void ora_eam_theta(const ora_eam* p, double* theta)
{
    int n = p->n_knots;
    for (int which = 0; which < 3; which++) {
        double xmax = which == 2 ? p->rho_max : p->r_c;
        double h = xmax / (n - 1);
        for (int k = 0; k < n; k++) {
            double y, dy;
            ora_eam_analytic(p, which, k * h, &y, &dy);
            theta[(which * n + k) * 2 + 0] = y;
            theta[(which * n + k) * 2 + 1] = dy;
        }
        if (which == 2) {
            double y1, dy1;
            ora_eam_analytic(p, 2, h, &y1, &dy1);
            theta[(2 * n + 0) * 2 + 1] = (y1 - theta[(2 * n + 0) * 2 + 0]) / h;
        }
    }
}

/* Cubic Hermite basis on interval k of a uniform grid over [0, xmax]:
 * y(x) = w0 y_k + w1 m_k + w2 y_{k+1} + w3 m_{k+1}, with the slope weights
 * carrying the knot spacing; dw = d/dx of the weights. */
static int hermite_basis(int n, double xmax, double x, int* k_out, double w[4],
                         double dw[4])
{
    double h = xmax / (n - 1);
    if (!(x >= 0.0) || x > xmax) return ORA_ERANGE;
    double t = x / h;
    int k = (int)floor(t);
    if (k > n - 2) k = n - 2;
    double u = t - k;
    double u2 = u * u, u3 = u2 * u;
    w[0] = 2 * u3 - 3 * u2 + 1;
    w[1] = (u3 - 2 * u2 + u) * h;
    w[2] = -2 * u3 + 3 * u2;
    w[3] = (u3 - u2) * h;
    dw[0] = (6 * u2 - 6 * u) / h;
    dw[1] = 3 * u2 - 4 * u + 1;
    dw[2] = (-6 * u2 + 6 * u) / h;
    dw[3] = 3 * u2 - 2 * u;
    *k_out = k;
    return ORA_OK;
}

int ora_hermite(const double* th, int n, double xmax, double x, double* y, double* dy)
{
    int k;
    double w[4], dw[4];
    int st = hermite_basis(n, xmax, x, &k, w, dw);
    if (st) return st;
    double yk = th[2 * k], mk = th[2 * k + 1], yk1 = th[2 * k + 2], mk1 = th[2 * k + 3];
    *y = w[0] * yk + w[1] * mk + w[2] * yk1 + w[3] * mk1;
    *dy = dw[0] * yk + dw[1] * mk + dw[2] * yk1 + dw[3] * mk1;
    return ORA_OK;
}

/* ------------------------------------------------------------- neighbours */
static void min_image(const double box[3], double d[3])
{
    for (int c = 0; c < 3; c++) d[c] -= box[c] * nearbyint(d[c] / box[c]);
}

int ora_pairs_brute(const double* x, int n, const double box[3], double rcut,
                    int* pi, int* pj, int max_pairs, int* n_pairs)
{
    int m = 0;
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) {
            double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1],
                           x[3 * j + 2] - x[3 * i + 2]};
            min_image(box, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < rcut * rcut) {
                if (m < max_pairs) { pi[m] = i; pj[m] = j; }
                m++;
            }
        }
    *n_pairs = m;
    return ORA_OK;
}

/* Cell binning over wrapped positions; falls back to all pairs when a box
 * holds fewer than three cells along any axis. */
int ora_pairs_cells(const double* x, int n, const double box[3], double rcut,
                    int* pi, int* pj, int max_pairs, int* n_pairs)
{
    int nc[3];
    for (int c = 0; c < 3; c++) nc[c] = (int)floor(box[c] / rcut);
    if (nc[0] < 3 || nc[1] < 3 || nc[2] < 3)
        return ora_pairs_brute(x, n, box, rcut, pi, pj, max_pairs, n_pairs);
    int ncell = nc[0] * nc[1] * nc[2];
    int* head = malloc(sizeof(int) * ncell);
    int* next = malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int c = 0; c < ncell; c++) head[c] = -1;
    for (int i = n - 1; i >= 0; i--) {
        int ci[3];
        for (int c = 0; c < 3; c++) {
            double s = x[3 * i + c] - box[c] * floor(x[3 * i + c] / box[c]);
            int q = (int)(s / (box[c] / nc[c]));
            if (q >= nc[c]) q = nc[c] - 1;
            if (q < 0) q = 0;
            ci[c] = q;
        }
        int cell = (ci[0] * nc[1] + ci[1]) * nc[2] + ci[2];
        next[i] = head[cell];
        head[cell] = i;
    }
    int m = 0;
    for (int cx = 0; cx < nc[0]; cx++)
        for (int cy = 0; cy < nc[1]; cy++)
            for (int cz = 0; cz < nc[2]; cz++) {
                int cell = (cx * nc[1] + cy) * nc[2] + cz;
                for (int dx = -1; dx <= 1; dx++)
                    for (int dy = -1; dy <= 1; dy++)
                        for (int dz = -1; dz <= 1; dz++) {
                            int ox = (cx + dx + nc[0]) % nc[0];
                            int oy = (cy + dy + nc[1]) % nc[1];
                            int oz = (cz + dz + nc[2]) % nc[2];
                            int other = (ox * nc[1] + oy) * nc[2] + oz;
                            for (int i = head[cell]; i >= 0; i = next[i])
                                for (int j = head[other]; j >= 0; j = next[j]) {
                                    if (j <= i) continue;
                                    double d[3] = {x[3 * j] - x[3 * i],
                                                   x[3 * j + 1] - x[3 * i + 1],
                                                   x[3 * j + 2] - x[3 * i + 2]};
                                    min_image(box, d);
                                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                                    if (r2 < rcut * rcut) {
                                        if (m < max_pairs) { pi[m] = i; pj[m] = j; }
                                        m++;
                                    }
                                }
                        }
            }
    free(head);
    free(next);
    *n_pairs = m;
    return ORA_OK;
}

/* All pairs within rcut, in freshly allocated arrays. */
static int pair_list(const double* x, int n, const double box[3], double rcut,
                     int** pi, int** pj, int* np)
{
    for (int c = 0; c < 3; c++)
        if (!(rcut < 0.5 * box[c])) return ORA_EINVAL;
    int cap = 64 * n + 16;
    for (;;) {
        *pi = malloc(sizeof(int) * cap);
        *pj = malloc(sizeof(int) * cap);
        ora_pairs_cells(x, n, box, rcut, *pi, *pj, cap, np);
        if (*np <= cap) return ORA_OK;
        free(*pi);
        free(*pj);
        cap = *np + 16;
    }
}

/* ------------------------------------------------------------------- EAM */
/* U = sum_{i<j} phi(r_ij) + sum_i F(rho_i),  rho_i = sum_{j!=i} f(r_ij);
 * F_i = sum_j [phi'(r_ij) + (F'(rho_i) + F'(rho_j)) f'(r_ij)] (r_j - r_i)/r_ij. */
int ora_eam_energy_forces(const ora_eam* p, const double* theta, const double* x,
                          int n, const double box[3], double* f, double* E,
                          double* rho)
{
    int nk = p->n_knots;
    const double* th_phi = theta;
    const double* th_f = theta + 2 * nk;
    const double* th_F = theta + 4 * nk;
    int *pi, *pj, np;
    int st = pair_list(x, n, box, p->r_c, &pi, &pj, &np);
    if (st) return st;
    double* rh = calloc(n > 0 ? n : 1, sizeof(double));
    double* dF = calloc(n > 0 ? n : 1, sizeof(double));
    double e_pair = 0.0, e_emb = 0.0;
    st = ORA_OK;
    for (int q = 0; q < np && !st; q++) {
        int i = pi[q], j = pj[q];
        double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1],
                       x[3 * j + 2] - x[3 * i + 2]};
        min_image(box, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (r < R_MIN) { st = ORA_ERANGE; break; }
        double fr, dfr, ph, dph;
        ora_hermite(th_f, nk, p->r_c, r, &fr, &dfr);
        ora_hermite(th_phi, nk, p->r_c, r, &ph, &dph);
        rh[i] += fr;
        rh[j] += fr;
        e_pair += ph;
    }
    for (int i = 0; i < n && !st; i++) {
        if (!(rh[i] < p->rho_max)) { st = ORA_ERANGE; break; }
        double Fi, dFi;
        ora_hermite(th_F, nk, p->rho_max, rh[i], &Fi, &dFi);
        e_emb += Fi;
        dF[i] = dFi;
    }
    if (!st && f) {
        for (int i = 0; i < 3 * n; i++) f[i] = 0.0;
        for (int q = 0; q < np; q++) {
            int i = pi[q], j = pj[q];
            double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1],
                           x[3 * j + 2] - x[3 * i + 2]};
            min_image(box, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double fr, dfr, ph, dph;
            ora_hermite(th_f, nk, p->r_c, r, &fr, &dfr);
            ora_hermite(th_phi, nk, p->r_c, r, &ph, &dph);
            double s = (dph + (dF[i] + dF[j]) * dfr) / r;
            for (int c = 0; c < 3; c++) {
                f[3 * i + c] += s * d[c];
                f[3 * j + c] -= s * d[c];
            }
        }
    }
    if (!st) {
        if (E) *E = e_pair + e_emb;
        if (rho)
            for (int i = 0; i < n; i++) rho[i] = rh[i];
        for (int i = 0; i < n; i++)
            if (!isfinite(rh[i])) st = ORA_ENAN;
    }
    free(pi);
    free(pj);
    free(rh);
    free(dF);
    return st;
}

/* dU/dtheta for every knot value and slope of phi, f and F.  U is linear in
 * the phi and F knots; the f knots enter through rho, weighted by
 * F'(rho_i) + F'(rho_j) for each pair. */
/* Virial: the r dU/dr of every pair inside r_c, with dU/dr = phi'(r) +
 * (F'(rho_i) + F'(rho_j)) f'(r); W = -sum over pairs. */
int ora_eam_virial(const ora_eam* p, const double* theta, const double* x, int n,
                   const double box[3], double* W)
{
    int nk = p->n_knots;
    const double* th_phi = theta;
    const double* th_f = theta + 2 * nk;
    const double* th_F = theta + 4 * nk;
    double* rho = calloc(n > 0 ? n : 1, sizeof(double));
    double E;
    int st = ora_eam_energy_forces(p, theta, x, n, box, NULL, &E, rho);
    if (st) { free(rho); return st; }
    int *pi, *pj, np;
    st = pair_list(x, n, box, p->r_c, &pi, &pj, &np);
    if (st) { free(rho); return st; }
    double w = 0.0;
    for (int q = 0; q < np; q++) {
        int i = pi[q], j = pj[q];
        double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
        min_image(box, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double fr, dfr, ph, dph, Fi, dFi, Fj, dFj;
        ora_hermite(th_f, nk, p->r_c, r, &fr, &dfr);
        ora_hermite(th_phi, nk, p->r_c, r, &ph, &dph);
        ora_hermite(th_F, nk, p->rho_max, rho[i], &Fi, &dFi);
        ora_hermite(th_F, nk, p->rho_max, rho[j], &Fj, &dFj);
        w -= r * (dph + (dFi + dFj) * dfr);
    }
    free(pi);
    free(pj);
    free(rho);
    *W = w;
    return ORA_OK;
}

/* Diagonal of the configurational virial tensor, W_a = sum_{i<j} r_ij,a F_ij,a
 * = -sum_{i<j} (r_ij,a^2 / r) dU/dr, the axis-by-axis form of the zero-stress
 * condition of the anisotropic barostat (Sec. III.A, fix nph aniso):
 * W_a = -dU/d eps_a when axis a and its coordinates scale by e^eps_a.  The
 * three sum to the virial above. */
int ora_eam_virial_axes(const ora_eam* p, const double* theta, const double* x, int n,
                        const double box[3], double W[3])
{
    int nk = p->n_knots;
    const double* th_phi = theta;
    const double* th_f = theta + 2 * nk;
    const double* th_F = theta + 4 * nk;
    double* rho = calloc(n > 0 ? n : 1, sizeof(double));
    double E;
    int st = ora_eam_energy_forces(p, theta, x, n, box, NULL, &E, rho);
    if (st) { free(rho); return st; }
    int *pi, *pj, np;
    st = pair_list(x, n, box, p->r_c, &pi, &pj, &np);
    if (st) { free(rho); return st; }
    double w[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < np; q++) {
        int i = pi[q], j = pj[q];
        double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
        min_image(box, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double fr, dfr, ph, dph, Fi, dFi, Fj, dFj;
        ora_hermite(th_f, nk, p->r_c, r, &fr, &dfr);
        ora_hermite(th_phi, nk, p->r_c, r, &ph, &dph);
        ora_hermite(th_F, nk, p->rho_max, rho[i], &Fi, &dFi);
        ora_hermite(th_F, nk, p->rho_max, rho[j], &Fj, &dFj);
        double dU_dr = dph + (dFi + dFj) * dfr;
        for (int a = 0; a < 3; a++) w[a] -= d[a] * d[a] / r * dU_dr;
    }
    free(pi);
    free(pj);
    free(rho);
    for (int a = 0; a < 3; a++) W[a] = w[a];
    return ORA_OK;
}

int ora_eam_grad_theta(const ora_eam* p, const double* theta, const double* x,
                       int n, const double box[3], double* grad)
{
    int nk = p->n_knots;
    const double* th_F = theta + 4 * nk;
    double* g_phi = grad;
    double* g_f = grad + 2 * nk;
    double* g_F = grad + 4 * nk;
    for (int q = 0; q < 6 * nk; q++) grad[q] = 0.0;
    double* rho = malloc(sizeof(double) * (n > 0 ? n : 1));
    int st = ora_eam_energy_forces(p, theta, x, n, box, NULL, NULL, rho);
    if (st) { free(rho); return st; }
    double* dF = malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int i = 0; i < n; i++) {
        double Fi;
        ora_hermite(th_F, nk, p->rho_max, rho[i], &Fi, &dF[i]);
        int k;
        double w[4], dw[4];
        hermite_basis(nk, p->rho_max, rho[i], &k, w, dw);
        g_F[2 * k] += w[0];
        g_F[2 * k + 1] += w[1];
        g_F[2 * k + 2] += w[2];
        g_F[2 * k + 3] += w[3];
    }
    int *pi, *pj, np;
    st = pair_list(x, n, box, p->r_c, &pi, &pj, &np);
    if (st) { free(rho); free(dF); return st; }
    for (int q = 0; q < np; q++) {
        int i = pi[q], j = pj[q];
        double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1],
                       x[3 * j + 2] - x[3 * i + 2]};
        min_image(box, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        int k;
        double w[4], dw[4];
        hermite_basis(nk, p->r_c, r, &k, w, dw);
        double wf = dF[i] + dF[j];
        for (int b = 0; b < 2; b++) {
            g_phi[2 * (k + b)] += w[2 * b];
            g_phi[2 * (k + b) + 1] += w[2 * b + 1];
            g_f[2 * (k + b)] += wf * w[2 * b];
            g_f[2 * (k + b) + 1] += wf * w[2 * b + 1];
        }
    }
    free(pi);
    free(pj);
    free(rho);
    free(dF);
    return ORA_OK;
}

/* ------------------------------------------------------- Einstein crystal */
/* U_E = sum_i (1/2) k |r_i - r_i^0|^2 with k = m omega^2 (eq. einstein). */
void ora_spring(const double* x, const double* x0, int n, double k, double* f, double* E)
{
    double e = 0.0;
    for (int i = 0; i < 3 * n; i++) {
        double u = x[i] - x0[i];
        e += 0.5 * k * u * u;
        if (f) f[i] = -k * u;
    }
    if (E) *E = e;
}

/* ------------------------------------------------------------- schedules */
/* Sec. III.B: function 1 is lambda = tau; function 2 is the ninth-order
 * polynomial tau^5 (70 tau^4 - 315 tau^3 + 540 tau^2 - 420 tau + 126). */
double ora_lambda_fl(int fn, double tau)
{
    if (fn == 1) return tau;
    return pow(tau, 5) * (70 * pow(tau, 4) - 315 * pow(tau, 3) + 540 * tau * tau -
                          420 * tau + 126);
}

/* Sec. III.C: lambda(tau) = 1 / (1 + tau (1/lambda_f - 1)), linear in T. */
double ora_lambda_rs(double lambda_f, double tau)
{
    return 1.0 / (1.0 + tau * (1.0 / lambda_f - 1.0));
}

/* Global lambda at the start of step s of the four-phase schedule. */
static double sched_lambda(const ora_md* md, long s)
{
    double li = md->path == ORA_PATH_FL ? 0.0 : 1.0;
    double lf = md->path == ORA_PATH_FL ? 1.0 : md->lambda_f;
    if (s <= md->t_eq) return li;
    long s1 = s - md->t_eq;
    if (s1 <= md->t_s) {
        double tau = (double)s1 / (double)md->t_s;
        return md->path == ORA_PATH_FL ? ora_lambda_fl(md->lambda_fn, tau)
                                       : ora_lambda_rs(md->lambda_f, tau);
    }
    long s2 = s1 - md->t_s;
    if (s2 <= md->t_eq) return lf;
    long s3 = s2 - md->t_eq;
    if (s3 <= md->t_s) {
        double tau = (double)s3 / (double)md->t_s;
        return md->path == ORA_PATH_FL ? 1.0 - ora_lambda_fl(md->lambda_fn, tau)
                                       : ora_lambda_rs(md->lambda_f, 1.0 - tau);
    }
    return li;
}

double ora_sched_lambda(const ora_md* md, long s) { return sched_lambda(md, s); }

/* Sec. III.A: the pressure of an NVT state from the thermostat's degrees of
 * freedom and the configurational virial W (ora_eam_virial) sampled along
 * the run, P = (N_dof k_B T + <W>) / (3 V); its standard error from the
 * scatter of the samples, s(W) / sqrt(n) / (3 V) (0 for one sample). */
void ora_pressure(int n_dof, double T, double V, const double* W, int n, double* P, double* err)
{
    double mean = 0.0;
    for (int i = 0; i < n; i++) mean += W[i];
    mean /= n;
    double ss = 0.0;
    for (int i = 0; i < n; i++) ss += (W[i] - mean) * (W[i] - mean);
    *P = (n_dof * ora_kB() * T + mean) / (3.0 * V);
    *err = n > 1 ? sqrt(ss / (n - 1)) / sqrt((double)n) / (3.0 * V) : 0.0;
}

/* ------------------------------------------------------------------ Philox */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11):
 * ten rounds of two 32x32->64 multiplications with the round keys bumped by
 * the Weyl constants between rounds. */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Three standard normals for (atom, step): one Philox block with key = seed
 * and counter = (atom, step_lo, step_hi, replica<<4 | stream); uniforms
 * (w + 1/2) 2^-32; two Box-Muller pairs, the fourth normal discarded. */
void ora_normals(uint64_t seed, uint32_t replica, uint32_t stream, uint32_t atom,
                 uint64_t step, double z[3])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {atom, (uint32_t)step, (uint32_t)(step >> 32),
                       (replica << 4) | (stream & 15u)};
    uint32_t w[4];
    ora_philox4x32_10(ctr, key, w);
    const double two_pi = 6.283185307179586476925286766559;
    double u[4];
    for (int q = 0; q < 4; q++) u[q] = ((double)w[q] + 0.5) * (1.0 / 4294967296.0);
    double r0 = sqrt(-2.0 * log(u[0]));
    double r1 = sqrt(-2.0 * log(u[2]));
    z[0] = r0 * cos(two_pi * u[1]);
    z[1] = r0 * sin(two_pi * u[1]);
    z[2] = r1 * cos(two_pi * u[3]);
}

void ora_philox_many(int n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out)
{
    for (int i = 0; i < n; i++) ora_philox4x32_10(ctr + 4 * (size_t)i, key, out + 4 * (size_t)i);
}

void ora_normals_many(uint64_t seed, uint32_t replica, uint32_t stream, uint64_t step, int n,
                      double* z)
{
    for (int a = 0; a < n; a++) ora_normals(seed, replica, stream, (uint32_t)a, step, z + 3 * (size_t)a);
}

/* ------------------------------------------------------------ dynamics */
static int dof(const ora_md* md, int n) { return md->fix_cm ? 3 * n - 3 : 3 * n; }

/* Mass of atom i: its species' mass with a species table, md->mass without. */
static double mass_of(const ora_md* md, int i)
{
    return md->species ? md->mass_s[md->species[i]] : md->mass;
}

/* A species table is usable when every index is in range, every mass
 * positive and every spring non-negative; no table is always usable. */
static int species_valid(const ora_md* md, int n)
{
    if (!md->species) return 1;
    if (md->n_species < 1 || !md->mass_s || !md->k_s) return 0;
    for (int s = 0; s < md->n_species; s++)
        if (!(md->mass_s[s] > 0) || !(md->k_s[s] >= 0)) return 0;
    for (int i = 0; i < n; i++)
        if (md->species[i] < 0 || md->species[i] >= md->n_species) return 0;
    return 1;
}

static double kinetic(const ora_md* md, const double* v, int n)
{
    double ke = 0.0;
    for (int i = 0; i < 3 * n; i++) ke += 0.5 * mass_of(md, i / 3) * v[i] * v[i];
    return ke;
}

/* Fixed centre of mass (Sec. III.A), imposed as a projection in the mass
 * metric.  A velocity-like array loses its centre-of-mass velocity,
 * u_i -= sum_j m_j u_j / M; for one species that is the plain mean. */
static void remove_cm_velocity(const ora_md* md, int n, double* u)
{
    for (int c = 0; c < 3; c++) {
        if (!md->species) {
            double mean = 0.0;
            for (int i = 0; i < n; i++) mean += u[3 * i + c];
            mean /= n;
            for (int i = 0; i < n; i++) u[3 * i + c] -= mean;
        } else {
            double P = 0.0, M = 0.0;
            for (int i = 0; i < n; i++) {
                P += mass_of(md, i) * u[3 * i + c];
                M += mass_of(md, i);
            }
            for (int i = 0; i < n; i++) u[3 * i + c] -= P / M;
        }
    }
}

/* A force array loses the part that would accelerate the centre of mass:
 * F_i -= m_i sum_j F_j / M, the constraint force that holds sum_j m_j r_j
 * fixed; for one species that is the plain mean. */
static void remove_cm_force(const ora_md* md, int n, double* F)
{
    for (int c = 0; c < 3; c++) {
        if (!md->species) {
            double mean = 0.0;
            for (int i = 0; i < n; i++) mean += F[3 * i + c];
            mean /= n;
            for (int i = 0; i < n; i++) F[3 * i + c] -= mean;
        } else {
            double S = 0.0, M = 0.0;
            for (int i = 0; i < n; i++) {
                S += F[3 * i + c];
                M += mass_of(md, i);
            }
            for (int i = 0; i < n; i++) F[3 * i + c] -= mass_of(md, i) * S / M;
        }
    }
}

/* Einstein springs of eq. einstein; with a species table atom i has the
 * spring k_s of its species (Sec. V). */
static void spring_md(const ora_md* md, const double* x, const double* x0, int n,
                      double* f, double* E)
{
    if (!md->species) {
        ora_spring(x, x0, n, md->k_spring, f, E);
        return;
    }
    double e = 0.0;
    for (int i = 0; i < 3 * n; i++) {
        double k = md->k_s[md->species[i / 3]];
        double u = x[i] - x0[i];
        e += 0.5 * k * u * u;
        f[i] = -k * u;
    }
    *E = e;
}

/* Maxwell-Boltzmann start: normals times sqrt(kT/m_i), zero total momentum
 * when the centre of mass is fixed (Sec. III.A), rescaled to exactly T. */
int ora_init_velocities(const ora_md* md, int n, double* v)
{
    if (n < 2 || !(md->T > 0) || !species_valid(md, n) || (!md->species && !(md->mass > 0)))
        return ORA_EINVAL;
    for (int i = 0; i < n; i++) {
        double sd = sqrt(KB_EV_PER_K * md->T / mass_of(md, i));
        double z[3];
        ora_normals(md->seed, md->replica, ORA_STREAM_INITV, (uint32_t)i, 0, z);
        for (int c = 0; c < 3; c++) v[3 * i + c] = sd * z[c];
    }
    if (md->fix_cm) remove_cm_velocity(md, n, v);
    double t_now = 2.0 * kinetic(md, v, n) / (dof(md, n) * KB_EV_PER_K);
    double s = sqrt(md->T / t_now);
    for (int i = 0; i < 3 * n; i++) v[i] *= s;
    return ORA_OK;
}

/* Potential terms at one configuration (Wv: virial of U0, with the barostat). */
typedef struct {
    double U0, UE, Wv;
    double Wa[3];  /* diagonal of the virial tensor (anisotropic barostat) */
    double* F0;
    double* FE;
} terms;

static int eval_terms(const ora_eam* p, const double* theta, const ora_md* md,
                      const double* x, const double* x0, int n, const double box[3],
                      terms* t)
{
    t->Wv = 0.0;
    t->Wa[0] = t->Wa[1] = t->Wa[2] = 0.0;
    if (md->h0 == ORA_H0_HARMONIC) {
        ora_spring(x, x0, n, md->k_h0, t->F0, &t->U0);  /* with the barostat: k_h0 = 0, an ideal gas */
    } else {
        int st = ora_eam_energy_forces(p, theta, x, n, box, t->F0, &t->U0, NULL);
        if (st) return st;
        if (md->npt == ORA_NPT_ISO) {
            st = ora_eam_virial(p, theta, x, n, box, &t->Wv);
            if (st) return st;
        } else if (md->npt == ORA_NPT_ANISO) {
            st = ora_eam_virial_axes(p, theta, x, n, box, t->Wa);
            if (st) return st;
        }
    }
    spring_md(md, x, x0, n, t->FE, &t->UE);
    return ORA_OK;
}

/* Total force of H(lambda): (1-lambda) F0 + lambda F_E on the Frenkel-Ladd
 * path (eq. interp), lambda F0 on the reversible-scaling path (eq. H_rs).
 * With the centre of mass fixed, its constraint force is added. */
static void blend_force(const ora_md* md, const terms* t, int n, double lam, double* F)
{
    for (int i = 0; i < 3 * n; i++)
        F[i] = md->path == ORA_PATH_FL ? (1.0 - lam) * t->F0[i] + lam * t->FE[i]
                                       : lam * t->F0[i];
    if (md->fix_cm) remove_cm_force(md, n, F);
}

/* dH/dlambda along the path, in the sign convention that makes eq. fl hold as
 * printed: U0 - U_E for Frenkel-Ladd, U0 for reversible scaling (eq. w_irr_rs). */
static double dH_dlambda(const ora_md* md, const terms* t)
{
    return md->path == ORA_PATH_FL ? t->U0 - t->UE : t->U0;
}

/* One step s -> s+1 at lambda_a = Lambda(s), lambda_b = Lambda(s+1):
 *   1. work increment (lambda_b - lambda_a) dH/dlambda at x_s (the discrete
 *      sum of Sec. II.A, left point), i.e. the Hamiltonian jumps at fixed x;
 *   2. half kick with F(x_s; lambda_b);  3. half drift;
 *   4. Ornstein-Uhlenbeck velocity update (Langevin thermostat, damping
 *      1/gamma), the centre-of-mass velocity of the noise removed when the
 *      centre of mass is fixed;
 *   5. half drift;  5b. with the barostat, the volume update below;
 *   6. forces at x_{s+1};  7. half kick with F(x_{s+1}; lambda_b).
 * t holds the terms at x_s on entry and at x_{s+1} on return.
 *
 * Barostat (md->npt, RS path): the positions at fixed velocities are one
 * configuration of a system whose scaled coordinates x/V^(1/3) and volume
 * V = e^eps sample p(eps) ~ V^(N'+1) exp(-(lambda U + P0 V)/kT) (N' = dof/3
 * independent positions).  eps takes one Euler-Maruyama step of the
 * overdamped Langevin equation with that stationary density and mobility
 * D = kT m_p / V, m_p = beta_T / tau_p (isotropic stochastic cell rescaling
 * at fixed momenta).  Its Ito drift D d(ln p)/d eps + dD/d eps is
 *   d eps = m_p [(dof kT + lambda W)/(3V) - P0] dt + sqrt(2 kT m_p dt / V) eta,
 * W the virial of U at x_s (the Jacobian's kT/V cancels against dD/d eps);
 * positions and box are scaled by e^(d eps / 3) about the origin, eta
 * drawn from the barostat stream.  Per axis (ORA_NPT_ANISO), eps_a = ln L_a
 * of each edge has p ~ V^(N'+1) exp(-(lambda U + P0 V)/kT) too (measure
 * dL_x dL_y dL_z), and the same steps give the drive (N' kT + lambda W_a)/V
 * - P0 per axis, W_a = -dU/d eps_a; coordinate a and edge a scale by
 * e^(d eps_a), eta_a the a-th normal of the barostat stream. */
static int md_step(const ora_eam* p, const double* theta, const ora_md* md,
                   uint32_t stream, long s, double lam_a, double lam_b, double* x,
                   double* v, const double* x0, int n, double box[3], terms* t,
                   double* F, double* xi, double* dW)
{
    double dt = md->dt;
    *dW = (lam_b - lam_a) * dH_dlambda(md, t);
    blend_force(md, t, n, lam_b, F);
    for (int i = 0; i < 3 * n; i++) v[i] += 0.5 * dt / mass_of(md, i / 3) * F[i];
    for (int i = 0; i < 3 * n; i++) x[i] += 0.5 * dt * v[i];
    double gamma = md->damp > 0 ? 1.0 / md->damp : 0.0;
    double c1 = exp(-gamma * dt);
    for (int i = 0; i < n; i++) {
        double z[3];
        ora_normals(md->seed, md->replica, stream, (uint32_t)i, (uint64_t)s, z);
        for (int c = 0; c < 3; c++) xi[3 * i + c] = z[c];
    }
    if (!md->species) {
        double c2 = sqrt((1.0 - c1 * c1) * KB_EV_PER_K * md->T / md->mass);
        if (md->fix_cm) remove_cm_velocity(md, n, xi);
        for (int i = 0; i < 3 * n; i++) v[i] = c1 * v[i] + c2 * xi[i];
    } else {
        /* velocity increments sqrt((1 - c1^2) kT / m_i) xi_i, their
         * centre-of-mass velocity removed */
        for (int i = 0; i < 3 * n; i++)
            xi[i] *= sqrt((1.0 - c1 * c1) * KB_EV_PER_K * md->T / mass_of(md, i / 3));
        if (md->fix_cm) remove_cm_velocity(md, n, xi);
        for (int i = 0; i < 3 * n; i++) v[i] = c1 * v[i] + xi[i];
    }
    for (int i = 0; i < 3 * n; i++) x[i] += 0.5 * dt * v[i];
    if (md->npt == ORA_NPT_ISO) {
        double kT = KB_EV_PER_K * md->T, V = box[0] * box[1] * box[2];
        double mp = md->beta_T / md->tau_p, z[3];
        ora_normals(md->seed, md->replica, ORA_STREAM_BARO, 0, (uint64_t)s, z);
        double drive = (dof(md, n) * kT + lam_b * t->Wv) / (3.0 * V) - md->P0;
        double deps = mp * drive * dt + sqrt(2.0 * kT * mp * dt / V) * z[0];
        double mu = exp(deps / 3.0);
        for (int i = 0; i < 3 * n; i++) x[i] *= mu;
        for (int c = 0; c < 3; c++) box[c] *= mu;
    } else if (md->npt == ORA_NPT_ANISO) {
        /* one such equation per axis, eps_a = ln L_a, with the same mobility:
         * d eps_a = m_p [(N' kT + lambda W_a)/V - P0] dt + sqrt(2 kT m_p dt / V) eta_a */
        double kT = KB_EV_PER_K * md->T, V = box[0] * box[1] * box[2];
        double mp = md->beta_T / md->tau_p, z[3], mu[3];
        ora_normals(md->seed, md->replica, ORA_STREAM_BARO, 0, (uint64_t)s, z);
        for (int c = 0; c < 3; c++) {
            double drive = (dof(md, n) / 3.0 * kT + lam_b * t->Wa[c]) / V - md->P0;
            double deps = mp * drive * dt + sqrt(2.0 * kT * mp * dt / V) * z[c];
            mu[c] = exp(deps);
        }
        for (int i = 0; i < n; i++)
            for (int c = 0; c < 3; c++) x[3 * i + c] *= mu[c];
        for (int c = 0; c < 3; c++) box[c] *= mu[c];
    }
    int st = eval_terms(p, theta, md, x, x0, n, box, t);
    if (st) return st;
    blend_force(md, t, n, lam_b, F);
    for (int i = 0; i < 3 * n; i++) v[i] += 0.5 * dt / mass_of(md, i / 3) * F[i];
    for (int i = 0; i < 3 * n; i++)
        if (!isfinite(x[i]) || !isfinite(v[i])) return ORA_ENAN;
    return ORA_OK;
}

typedef struct {
    terms t;
    double *F, *xi;
} workspace;

static void ws_alloc(workspace* w, int n)
{
    w->t.F0 = malloc(sizeof(double) * 3 * n);
    w->t.FE = malloc(sizeof(double) * 3 * n);
    w->F = malloc(sizeof(double) * 3 * n);
    w->xi = malloc(sizeof(double) * 3 * n);
}

static void ws_free(workspace* w)
{
    free(w->t.F0);
    free(w->t.FE);
    free(w->F);
    free(w->xi);
}

/* Schedule of Sec. III.B (fix ti/spring) and Sec. III.C: equilibrate at the
 * initial lambda, switch forward over t_s steps, equilibrate at the final
 * lambda, switch back.  W_f and W_b are the two irreversible works.  The
 * run stops after s_end steps of the schedule (all of it when s_end is
 * 2 t_eq + 2 t_s). */
static int switch_run_steps(const ora_eam* p, const double* theta, const ora_md* md,
                            double* x, double* v, const double* x0, int n,
                            double box[3], double* W_f, double* W_b,
                            double* Wcum_f, double* Wcum_b, double* trace,
                            int trace_stride, int n_trace_max, long s_end)
{
    if (n < 2 || md->t_s < 1 || md->t_eq < 0 || !species_valid(md, n)) return ORA_EINVAL;
    if (md->path == ORA_PATH_RS && !(md->lambda_f > 0 && md->lambda_f < 1)) return ORA_EINVAL;
    if (md->npt < 0 || md->npt > ORA_NPT_ANISO) return ORA_EINVAL;
    if (md->npt && (md->path != ORA_PATH_RS || !(md->beta_T > 0) || !(md->tau_p > 0) || md->P0 < 0 ||
                    (md->h0 == ORA_H0_HARMONIC && md->k_h0 != 0.0)))
        return ORA_EINVAL;  /* the Einstein crystal has no pressure (Sec. III.A) */
    workspace w;
    ws_alloc(&w, n);
    uint32_t stream = md->path == ORA_PATH_FL ? ORA_STREAM_FL : ORA_STREAM_RS;
    int st = eval_terms(p, theta, md, x, x0, n, box, &w.t);
    long S = 2 * md->t_eq + 2 * md->t_s;
    long fwd0 = md->t_eq, bwd0 = 2 * md->t_eq + md->t_s;
    double wf = 0.0, wb = 0.0;
    int nt = 0;
    if (Wcum_f) Wcum_f[0] = 0.0;
    if (Wcum_b) Wcum_b[0] = 0.0;
    if (s_end < S) S = s_end;
    for (long s = 0; s < S && !st; s++) {
        if (trace && trace_stride > 0 && s % trace_stride == 0 && nt < n_trace_max) {
            double* r = trace + 8 * nt++;
            r[0] = (double)s;
            r[1] = sched_lambda(md, s);
            r[2] = dH_dlambda(md, &w.t);
            r[3] = w.t.U0;
            r[4] = w.t.UE;
            r[5] = 2.0 * kinetic(md, v, n) / (dof(md, n) * KB_EV_PER_K);
            r[6] = wf;
            r[7] = wb;
        }
        double la = sched_lambda(md, s), lb = sched_lambda(md, s + 1), dW;
        st = md_step(p, theta, md, stream, s, la, lb, x, v, x0, n, box, &w.t, w.F, w.xi, &dW);
        if (s >= fwd0 && s < fwd0 + md->t_s) {
            wf += dW;
            if (Wcum_f) Wcum_f[s - fwd0 + 1] = wf;
        } else if (s >= bwd0 && s < bwd0 + md->t_s) {
            wb += dW;
            if (Wcum_b) Wcum_b[s - bwd0 + 1] = wb;
        }
    }
    ws_free(&w);
    if (W_f) *W_f = wf;
    if (W_b) *W_b = wb;
    return st;
}

int ora_switch_run(const ora_eam* p, const double* theta, const ora_md* md,
                   double* x, double* v, const double* x0, int n,
                   double box[3], double* W_f, double* W_b,
                   double* Wcum_f, double* Wcum_b, double* trace,
                   int trace_stride, int n_trace_max)
{
    return switch_run_steps(p, theta, md, x, v, x0, n, box, W_f, W_b, Wcum_f, Wcum_b, trace,
                            trace_stride, n_trace_max, 2 * md->t_eq + 2 * md->t_s);
}

int ora_switch_run_prefix(const ora_eam* p, const double* theta, const ora_md* md,
                          double* x, double* v, const double* x0, int n, double box[3],
                          long n_steps, double* W_f, double* W_b, double* Wcum_f,
                          double* Wcum_b)
{
    if (n_steps < 0) return ORA_EINVAL;
    return switch_run_steps(p, theta, md, x, v, x0, n, box, W_f, W_b, Wcum_f, Wcum_b, NULL, 0, 0,
                            n_steps);
}

int ora_langevin_steps(const ora_eam* p, const double* theta, const ora_md* md,
                       double lambda, double* x, double* v, const double* x0,
                       int n, const double box[3], long step0, long n_steps)
{
    if (n < 2 || md->npt || !species_valid(md, n)) return ORA_EINVAL;  /* fixed box */
    double bx[3] = {box[0], box[1], box[2]};
    workspace w;
    ws_alloc(&w, n);
    int st = eval_terms(p, theta, md, x, x0, n, bx, &w.t);
    for (long s = 0; s < n_steps && !st; s++) {
        double dW;
        st = md_step(p, theta, md, ORA_STREAM_STEP, step0 + s, lambda, lambda, x, v, x0,
                     n, bx, &w.t, w.F, w.xi, &dW);
    }
    ws_free(&w);
    return st;
}

/* Eq. msd (Sec. III.A): k = 3 k_B T / <|dr|^2>, with dr the displacement from
 * the initial site corrected for the centre-of-mass motion (compute msd com).
 * The average runs per class of atoms: the species with a species table (the
 * centre of mass then mass-weighted, the one the dynamics holds fixed), one
 * class of all atoms without.  acc[c] sums, over the samples, the class mean
 * of |dr|^2. */
static int msd_run(const ora_eam* p, const double* theta, const ora_md* md, double* x,
                   double* v, const double* x0, int n, const double box[3], long n_eq,
                   long n_samples, int stride, int n_class, double* acc)
{
    ora_md m0 = *md;
    m0.path = ORA_PATH_FL;
    m0.npt = 0;
    double bx[3] = {box[0], box[1], box[2]};
    int* count = calloc(n_class, sizeof(int));
    double* msd = calloc(n_class, sizeof(double));
    for (int i = 0; i < n; i++) count[md->species ? md->species[i] : 0]++;
    for (int c = 0; c < n_class; c++) acc[c] = 0.0;
    int st = ORA_OK;
    for (int c = 0; c < n_class; c++)
        if (count[c] == 0) st = ORA_EINVAL;
    workspace w;
    ws_alloc(&w, n);
    if (!st) st = eval_terms(p, theta, &m0, x, x0, n, box, &w.t);
    long s = 0;
    for (; s < n_eq && !st; s++) {
        double dW;
        st = md_step(p, theta, &m0, ORA_STREAM_MSD, s, 0.0, 0.0, x, v, x0, n, bx, &w.t,
                     w.F, w.xi, &dW);
    }
    for (long q = 0; q < n_samples && !st; q++) {
        for (int r = 0; r < stride && !st; r++, s++) {
            double dW;
            st = md_step(p, theta, &m0, ORA_STREAM_MSD, s, 0.0, 0.0, x, v, x0, n, bx,
                         &w.t, w.F, w.xi, &dW);
        }
        double R[3] = {0, 0, 0}, R0[3] = {0, 0, 0};
        if (!md->species) {
            for (int i = 0; i < n; i++)
                for (int c = 0; c < 3; c++) {
                    R[c] += x[3 * i + c] / n;
                    R0[c] += x0[3 * i + c] / n;
                }
        } else {
            double M = 0.0;
            for (int i = 0; i < n; i++) M += mass_of(md, i);
            for (int i = 0; i < n; i++)
                for (int c = 0; c < 3; c++) {
                    R[c] += mass_of(md, i) * x[3 * i + c] / M;
                    R0[c] += mass_of(md, i) * x0[3 * i + c] / M;
                }
        }
        for (int c = 0; c < n_class; c++) msd[c] = 0.0;
        for (int i = 0; i < n; i++)
            for (int c = 0; c < 3; c++) {
                double d = (x[3 * i + c] - x0[3 * i + c]) - (R[c] - R0[c]);
                msd[md->species ? md->species[i] : 0] += d * d;
            }
        for (int c = 0; c < n_class; c++) acc[c] += msd[c] / count[c];
    }
    ws_free(&w);
    free(count);
    free(msd);
    return st;
}

int ora_msd_fit(const ora_eam* p, const double* theta, const ora_md* md, double* x,
                double* v, const double* x0, int n, const double box[3],
                long n_eq, long n_samples, int stride, double* msd_out, double* k_out)
{
    if (n < 2 || n_samples < 1 || stride < 1 || md->species) return ORA_EINVAL;
    double acc;
    int st = msd_run(p, theta, md, x, v, x0, n, box, n_eq, n_samples, stride, 1, &acc);
    if (st) return st;
    double mean = acc / n_samples;
    if (msd_out) *msd_out = mean;
    if (k_out) *k_out = 3.0 * KB_EV_PER_K * md->T / mean;
    return ORA_OK;
}

/* Sec. V: one spring per species, each from the msd of its own atoms. */
int ora_msd_fit_species(const ora_eam* p, const double* theta, const ora_md* md,
                        double* x, double* v, const double* x0, int n,
                        const double box[3], long n_eq, long n_samples, int stride,
                        double* msd_s, double* k_out)
{
    if (n < 2 || n_samples < 1 || stride < 1 || !md->species || !species_valid(md, n))
        return ORA_EINVAL;
    double* acc = calloc(md->n_species, sizeof(double));
    int st = msd_run(p, theta, md, x, v, x0, n, box, n_eq, n_samples, stride,
                     md->n_species, acc);
    for (int c = 0; c < md->n_species && !st; c++) {
        double mean = acc[c] / n_samples;
        if (msd_s) msd_s[c] = mean;
        if (k_out) k_out[c] = 3.0 * KB_EV_PER_K * md->T / mean;
    }
    free(acc);
    return st;
}

/* --------------------------------------------------------------- assembly */
/* Einstein-crystal free energy F_E = 3 N k_B T ln(hbar omega / k_B T). */
double ora_einstein_F(int n, double T, double mass, double k)
{
    double omega = sqrt(k / mass);
    return 3.0 * n * KB_EV_PER_K * T * log(HBAR_EV_PS * omega / (KB_EV_PER_K * T));
}

/* Eq. cm: dF_CM = k_B T ln[(N/V) (2 pi k_B T / (N m omega^2))^{3/2}], m omega^2 = k. */
double ora_cm_correction(int n, double V, double T, double mass, double k)
{
    (void)mass;
    double kT = KB_EV_PER_K * T;
    const double pi = 3.14159265358979323846264338327950;
    return kT * log((n / V) * pow(2.0 * pi * kT / (n * k), 1.5));
}

/* Eq. fl plus eq. cm: F_0 = F_E + (mean W_f - mean W_b)/2 + dF_CM, per atom;
 * the error bar is the standard error over seeds of (W_f - W_b)/(2N); the
 * dissipation (eq. Ediss) is -(mean W_f + mean W_b)/2 in this sign convention. */
/* Eq. jarz: dF = -kT ln[(1/n) sum exp(x_s)], x_s = -W_s/kT, written as
 * -kT [x_max + ln sum exp(x_s - x_max) - ln n]. */
double ora_jarzynski(double T, const double* W, int n)
{
    double kT = ora_kB() * T;
    double xmax = -W[0] / kT;
    for (int s = 1; s < n; s++)
        if (-W[s] / kT > xmax) xmax = -W[s] / kT;
    double sum = 0.0;
    for (int s = 0; s < n; s++) sum += exp(-W[s] / kT - xmax);
    return -kT * (xmax + log(sum) - log((double)n));
}

/* Seed statistics of eq. fl: the seed means of W_f and W_b, the standard
 * error over seeds of (W_f - W_b)/(2n) and the dissipation -(mean W_f + mean
 * W_b)/(2n) of eq. Ediss. */
static void work_stats(int n, const double* W_f, const double* W_b, int n_seeds,
                       double* mf_out, double* mb_out, double* se_out, double* ed_out)
{
    double mf = 0.0, mb = 0.0;
    for (int q = 0; q < n_seeds; q++) { mf += W_f[q]; mb += W_b[q]; }
    mf /= n_seeds;
    mb /= n_seeds;
    double se = 0.0;
    if (n_seeds > 1) {
        double mean = 0.5 * (mf - mb) / n, var = 0.0;
        for (int q = 0; q < n_seeds; q++) {
            double d = 0.5 * (W_f[q] - W_b[q]) / n - mean;
            var += d * d;
        }
        var /= (n_seeds - 1);
        se = sqrt(var / n_seeds);
    }
    *mf_out = mf;
    *mb_out = mb;
    *se_out = se;
    *ed_out = -0.5 * (mf + mb) / n;
}

int ora_free_energy(int n, double V, double T, double mass, double k,
                    const double* W_f, const double* W_b, int n_seeds,
                    double* F_per_atom, double* stderr_per_atom,
                    double* Ediss_per_atom)
{
    if (n < 1 || n_seeds < 1 || !(V > 0) || !(T > 0) || !(k > 0) || !(mass > 0))
        return ORA_EINVAL;
    double mf, mb, se, ed;
    work_stats(n, W_f, W_b, n_seeds, &mf, &mb, &se, &ed);
    double F = ora_einstein_F(n, T, mass, k) + 0.5 * (mf - mb) +
               ora_cm_correction(n, V, T, mass, k);
    if (F_per_atom) *F_per_atom = F / n;
    if (stderr_per_atom) *stderr_per_atom = se;
    if (Ediss_per_atom) *Ediss_per_atom = ed;
    return ORA_OK;
}

/* Eq. einstein for independent oscillators with one frequency per species
 * (Sec. V): F_E = sum_i 3 k_B T ln(hbar omega_i / k_B T), omega_i^2 = k_i/m_i. */
double ora_einstein_F_species(int n, const int* species, const double* mass_s,
                              const double* k_s, double T)
{
    double F = 0.0;
    for (int i = 0; i < n; i++) {
        double omega = sqrt(k_s[species[i]] / mass_s[species[i]]);
        F += 3.0 * KB_EV_PER_K * T * log(HBAR_EV_PS * omega / (KB_EV_PER_K * T));
    }
    return F;
}

/* Eq. cm with several species.  The factor 2 pi k_B T / (N m omega^2) of
 * eq. cm is 2 pi sigma^2, sigma^2 the variance per axis of the centre of mass
 * of the Einstein crystal about its site; the centre the dynamics holds fixed
 * is R = sum_i m_i r_i / M, whose variance with independent springs k_i is
 * sigma^2 = k_B T sum_i (m_i / M)^2 / k_i.  The leading N / V stays as
 * printed. */
double ora_cm_correction_species(int n, const int* species, const double* mass_s,
                                 const double* k_s, double V, double T)
{
    double kT = KB_EV_PER_K * T, M = 0.0, s2 = 0.0;
    const double pi = 3.14159265358979323846264338327950;
    for (int i = 0; i < n; i++) M += mass_s[species[i]];
    for (int i = 0; i < n; i++) {
        double w = mass_s[species[i]] / M;
        s2 += w * w * kT / k_s[species[i]];
    }
    return kT * log((n / V) * pow(2.0 * pi * s2, 1.5));
}

/* Eq. fl plus eq. cm with one spring per species (Sec. V). */
int ora_free_energy_species(int n, const int* species, int n_species,
                            const double* mass_s, const double* k_s, double V,
                            double T, const double* W_f, const double* W_b,
                            int n_seeds, double* F_per_atom,
                            double* stderr_per_atom, double* Ediss_per_atom)
{
    if (n < 1 || n_seeds < 1 || !(V > 0) || !(T > 0) || n_species < 1 || !species ||
        !mass_s || !k_s)
        return ORA_EINVAL;
    for (int s = 0; s < n_species; s++)
        if (!(mass_s[s] > 0) || !(k_s[s] > 0)) return ORA_EINVAL;
    for (int i = 0; i < n; i++)
        if (species[i] < 0 || species[i] >= n_species) return ORA_EINVAL;
    double mf, mb, se, ed;
    work_stats(n, W_f, W_b, n_seeds, &mf, &mb, &se, &ed);
    double F = ora_einstein_F_species(n, species, mass_s, k_s, T) + 0.5 * (mf - mb) +
               ora_cm_correction_species(n, species, mass_s, k_s, V, T);
    if (F_per_atom) *F_per_atom = F / n;
    if (stderr_per_atom) *stderr_per_atom = se;
    if (Ediss_per_atom) *Ediss_per_atom = ed;
    return ORA_OK;
}

/* Eq. rs: F_0(T) = F_0(T_0)/lambda + (3/2) N k_B T_0 ln(lambda)/lambda
 *               + [W_{1->lambda} - W_{lambda->1}] / (2 lambda),  lambda = T_0/T.
 * W_{1->lambda}: forward cumulative work where lambda(t) passes lambda;
 * W_{lambda->1}: backward total minus its cumulative work up to lambda; both
 * linearly interpolated in lambda between the bracketing steps.  Cumulative
 * works are averaged over seeds first. */
int ora_rs_free_energy(int n, double T0, double F0_T0, double lambda_f, long t_s,
                       const double* Wcum_f, const double* Wcum_b, int n_seeds,
                       const double* T_grid, int n_T, double* F_per_atom)
{
    if (n < 1 || t_s < 1 || n_seeds < 1 || !(lambda_f > 0 && lambda_f < 1)) return ORA_EINVAL;
    double* wf = calloc(t_s + 1, sizeof(double));
    double* wb = calloc(t_s + 1, sizeof(double));
    for (int q = 0; q < n_seeds; q++)
        for (long k = 0; k <= t_s; k++) {
            wf[k] += Wcum_f[q * (t_s + 1) + k] / n_seeds;
            wb[k] += Wcum_b[q * (t_s + 1) + k] / n_seeds;
        }
    int st = ORA_OK;
    for (int g = 0; g < n_T; g++) {
        double lam = T0 / T_grid[g];
        if (lam > 1.0 || lam < lambda_f) { st = ORA_EINVAL; break; }
        /* forward: lambda decreases from 1 to lambda_f */
        double w_fwd = wf[t_s];
        for (long k = 0; k < t_s; k++) {
            double la = ora_lambda_rs(lambda_f, (double)k / t_s);
            double lb = ora_lambda_rs(lambda_f, (double)(k + 1) / t_s);
            if (lam <= la && lam >= lb) {
                double a = (lam - la) / (lb - la);
                w_fwd = wf[k] + a * (wf[k + 1] - wf[k]);
                break;
            }
        }
        /* backward: lambda increases from lambda_f to 1 */
        double w_b_upto = wb[t_s];
        for (long k = 0; k < t_s; k++) {
            double la = ora_lambda_rs(lambda_f, 1.0 - (double)k / t_s);
            double lb = ora_lambda_rs(lambda_f, 1.0 - (double)(k + 1) / t_s);
            if (lam >= la && lam <= lb) {
                double a = (lam - la) / (lb - la);
                w_b_upto = wb[k] + a * (wb[k + 1] - wb[k]);
                break;
            }
        }
        double w_bwd = wb[t_s] - w_b_upto;
        double F = F0_T0 / lam + 1.5 * n * KB_EV_PER_K * T0 * log(lam) / lam +
                   (w_fwd - w_bwd) / (2.0 * lam);
        F_per_atom[g] = F / n;
    }
    free(wf);
    free(wb);
    return st;
}
