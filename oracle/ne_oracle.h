/*
 * ne_oracle.h -- plain, slow, FP64 CPU oracle of the nonequilibrium free-energy
 * method of Freitas, Asta & de Koning (Frenkel-Ladd and reversible-scaling
 * switching of an EAM crystal under Langevin dynamics).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only
 * the test-suite, the package smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, constant or table
 * generator with the CUDA library; the two are written independently from the
 * paper and meet only through seeded inputs.
 *
 * Units: metal (Angstrom, eV, ps, atomic mass unit, Kelvin).
 * All arrays are caller-owned host memory.  Positions are AoS [n][3].
 * Functions return 0 on success, a negative ORA_E* code on error.
 */
#ifndef NE_ORACLE_H
#define NE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_OK = 0, ORA_EINVAL = -1, ORA_ERANGE = -4, ORA_ENAN = -6 };
enum { ORA_BCC = 0, ORA_FCC = 1, ORA_HCP = 2 };
enum { ORA_PATH_FL = 0, ORA_PATH_RS = 1 };
enum { ORA_H0_EAM = 0, ORA_H0_HARMONIC = 1 };
/* barostat (ora_md.npt): off, isotropic, or one box edge at a time */
enum { ORA_NPT_OFF = 0, ORA_NPT_ISO = 1, ORA_NPT_ANISO = 2 };
/* Philox stream ids (4th counter word, low bits). */
enum { ORA_STREAM_FL = 0, ORA_STREAM_INITV = 1, ORA_STREAM_RS = 2,
       ORA_STREAM_MSD = 3, ORA_STREAM_STEP = 4, ORA_STREAM_BARO = 5 };

/* Analytic Fe-like EAM: Johnson-type exponential pair and density,
 * Finnis-Sinclair embedding F = -B sqrt(rho), quintic taper r_s..r_c. */
typedef struct {
    double A, alpha, beta, B, r_e, r_s, r_c, rho_max;
    int n_knots;
} ora_eam;

/* One Langevin switching trajectory. */
typedef struct {
    double dt;        /* ps */
    double T;         /* K */
    double damp;      /* ps, gamma = 1/damp */
    double mass;      /* eV ps^2 / A^2 */
    double k_spring;  /* Einstein spring, eV/A^2 */
    int lambda_fn;    /* FL: 1 linear, 2 polynomial */
    int path;         /* ORA_PATH_FL / ORA_PATH_RS */
    long t_eq, t_s;   /* steps */
    double lambda_f;  /* RS end point */
    uint64_t seed;
    uint32_t replica;
    int fix_cm;       /* 1: centre of mass held fixed (noise and force means removed) */
    int h0;           /* ORA_H0_EAM, or ORA_H0_HARMONIC (springs k_h0 to the sites) */
    double k_h0;
    /* barostat (reversible-scaling path only, Sec. III.C): ORA_NPT_OFF,
     * ORA_NPT_ISO (the volume) or ORA_NPT_ANISO (each box edge on its own,
     * fix nph aniso of Sec. III.A, for non-cubic cells such as hcp) */
    int npt;
    double P0;        /* target pressure, eV/A^3 */
    double beta_T;    /* compressibility of the coupling, A^3/eV */
    double tau_p;     /* relaxation time of the coupling, ps */
    /* Several species (Sec. V: an A-B solid with one Einstein spring per
     * species).  species == NULL: every atom has mass and k_spring.  Else atom
     * i has mass mass_s[species[i]] and spring k_s[species[i]] (mass and
     * k_spring unused), and the fixed centre of mass is the mass-weighted one:
     * forces and noise are projected in the mass metric.  The springs of
     * ORA_H0_HARMONIC stay k_h0 for every atom. */
    int n_species;
    const int* species;     /* [n], 0 <= species[i] < n_species */
    const double* mass_s;   /* [n_species], eV ps^2 / A^2 */
    const double* k_s;      /* [n_species], eV/A^2 */
} ora_md;

/* constants */
double ora_kB(void);
double ora_hbar(void);
double ora_amu(void);          /* 1 u in eV ps^2/A^2 */

/* crystal: sites r0 [n][3], box lengths; returns n via n_out. */
int ora_create_crystal(int lattice, double a, int nx, int ny, int nz,
                       double* x0, double box[3], int* n_out);
/* Same with the axial ratio of hcp given: c = c_over_a * a (ignored for
 * bcc and fcc); ora_create_crystal uses the ideal sqrt(8/3). */
int ora_create_crystal_ca(int lattice, double a, double c_over_a, int nx, int ny, int nz,
                          double* x0, double box[3], int* n_out);

/* analytic functions and tables */
void ora_eam_analytic(const ora_eam* p, int which /*0 phi,1 f,2 F*/, double x,
                      double* y, double* dy);
void ora_eam_theta(const ora_eam* p, double* theta /* [3][n_knots][2] */);
int ora_hermite(const double* th /* [n][2] */, int n, double xmax, double x,
                double* y, double* dy);

/* neighbour pairs (half list i<j) within rcut, minimum image */
int ora_pairs_brute(const double* x, int n, const double box[3], double rcut,
                    int* pi, int* pj, int max_pairs, int* n_pairs);
int ora_pairs_cells(const double* x, int n, const double box[3], double rcut,
                    int* pi, int* pj, int max_pairs, int* n_pairs);

/* EAM energy, forces and per-atom density from knot parameters theta. */
int ora_eam_energy_forces(const ora_eam* p, const double* theta, const double* x,
                          int n, const double box[3], double* f, double* E,
                          double* rho);
/* dE/dtheta [3][n_knots][2] (same layout as theta). */
/* Configurational virial W = sum_{i<j} r_ij . F_ij = -sum_{i<j} r dU/dr
 * (Sec. III.A zero-pressure condition; P = (N_dof k_B T + W) / (3V)). */
int ora_eam_virial(const ora_eam* p, const double* theta, const double* x, int n,
                   const double box[3], double* W);
/* Diagonal of the virial tensor, W_a = -dU/d eps_a for a scaling of axis a
 * alone; W[0] + W[1] + W[2] is the virial above. */
int ora_eam_virial_axes(const ora_eam* p, const double* theta, const double* x, int n,
                        const double box[3], double W[3]);
int ora_eam_grad_theta(const ora_eam* p, const double* theta, const double* x,
                       int n, const double box[3], double* grad);

void ora_spring(const double* x, const double* x0, int n, double k, double* f,
                double* E);

double ora_lambda_fl(int fn, double tau);
double ora_lambda_rs(double lambda_f, double tau);
/* lambda in force at the start of step s of md's four-phase schedule */
double ora_sched_lambda(const ora_md* md, long s);
/* P = (N_dof k_B T + <W>) / (3V) from n virial samples W, and its standard error */
void ora_pressure(int n_dof, double T, double V, const double* W, int n, double* P, double* err);

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void ora_normals(uint64_t seed, uint32_t replica, uint32_t stream, uint32_t atom,
                 uint64_t step, double z[3]);
/* The same, one call for many: out[4 i ..] = block of ctr[4 i ..] (one key);
 * z[3 a ..] = normals of atoms a = 0 .. n-1 at one (seed, replica, stream, step). */
void ora_philox_many(int n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out);
void ora_normals_many(uint64_t seed, uint32_t replica, uint32_t stream, uint64_t step, int n,
                      double* z);

int ora_init_velocities(const ora_md* md, int n, double* v);

/* FL schedule: t_eq at 0, switch 0->1, t_eq at 1, switch 1->0.
 * RS schedule: t_eq at 1, switch 1->lambda_f, t_eq at lambda_f, switch back.
 * Wcum_f / Wcum_b (nullable): cumulative work after each switch step, t_s+1.
 * trace (nullable): every trace_stride steps, 8 doubles
 *   (step, lambda, dH/dlambda, U0, U_E, T_internal, W_f, W_b).
 * With md->npt (RS path only) the box follows the barostat, isotropic or
 * per axis, and box[] returns the final box. */
int ora_switch_run(const ora_eam* p, const double* theta, const ora_md* md,
                   double* x, double* v, const double* x0, int n,
                   double box[3], double* W_f, double* W_b,
                   double* Wcum_f, double* Wcum_b, double* trace,
                   int trace_stride, int n_trace_max);

/* The first n_steps steps of that schedule (all of it when n_steps >= 2 t_eq
 * + 2 t_s), the same steps, noise and works as ora_switch_run up to there:
 * W_f, W_b the works done so far, Wcum_* filled up to the last switching
 * step reached (entries beyond it untouched). */
int ora_switch_run_prefix(const ora_eam* p, const double* theta, const ora_md* md,
                          double* x, double* v, const double* x0, int n, double box[3],
                          long n_steps, double* W_f, double* W_b, double* Wcum_f,
                          double* Wcum_b);

/* Plain Langevin steps at fixed lambda (FL blend), n_steps, noise stream STEP,
 * starting at global step step0. */
int ora_langevin_steps(const ora_eam* p, const double* theta, const ora_md* md,
                       double lambda, double* x, double* v, const double* x0,
                       int n, const double box[3], long step0, long n_steps);

/* Spring-constant fit from the mean-squared displacement (one species:
 * md->species must be NULL). */
int ora_msd_fit(const ora_eam* p, const double* theta, const ora_md* md, double* x,
                double* v, const double* x0, int n, const double box[3],
                long n_eq, long n_samples, int stride, double* msd_out,
                double* k_out);
/* The same per species (Sec. V): msd_s[s] averages over the atoms of species
 * s, displacements taken relative to the mass-weighted centre of mass, and
 * k_out[s] = 3 k_B T / msd_s[s].  md->species must be set and every species
 * must have atoms. */
int ora_msd_fit_species(const ora_eam* p, const double* theta, const ora_md* md,
                        double* x, double* v, const double* x0, int n,
                        const double box[3], long n_eq, long n_samples, int stride,
                        double* msd_s, double* k_out);

/* Free-energy assembly (host, FP64). */
double ora_einstein_F(int n, double T, double mass, double k);
double ora_cm_correction(int n, double V, double T, double mass, double k);
/* Eq. jarz (Sec. II.A): exp(-dF/kT) = mean exp(-W/kT) over realisations,
 * W the work done on the system. */
double ora_jarzynski(double T, const double* W, int n);
int ora_free_energy(int n, double V, double T, double mass, double k,
                    const double* W_f, const double* W_b, int n_seeds,
                    double* F_per_atom, double* stderr_per_atom,
                    double* Ediss_per_atom);
/* Several species (Sec. V): eq. einstein summed over the atoms with
 * omega_i^2 = k_i / m_i, and eq. cm with the variance of the mass-weighted
 * centre of the Einstein crystal, sigma^2 = k_B T sum_i (m_i/M)^2 / k_i, in
 * place of k_B T / (N m omega^2).  species[i] indexes mass_s and k_s. */
double ora_einstein_F_species(int n, const int* species, const double* mass_s,
                              const double* k_s, double T);
double ora_cm_correction_species(int n, const int* species, const double* mass_s,
                                 const double* k_s, double V, double T);
int ora_free_energy_species(int n, const int* species, int n_species,
                            const double* mass_s, const double* k_s, double V,
                            double T, const double* W_f, const double* W_b,
                            int n_seeds, double* F_per_atom,
                            double* stderr_per_atom, double* Ediss_per_atom);
int ora_rs_free_energy(int n, double T0, double F0_T0, double lambda_f, long t_s,
                       const double* Wcum_f, const double* Wcum_b, int n_seeds,
                       const double* T_grid, int n_T, double* F_per_atom);

#ifdef __cplusplus
}
#endif
#endif
