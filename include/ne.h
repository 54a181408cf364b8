/*
 * ne.h -- C ABI of the GB300 nonequilibrium free-energy library (libne.so).
 *
 * The library runs Langevin molecular dynamics of an EAM crystal whose
 * Hamiltonian is switched in time, and turns the irreversible work into free
 * energies, after Freitas, Asta & de Koning, "Nonequilibrium free-energy
 * calculation of solids using LAMMPS":
 *   - Frenkel-Ladd path (Sec. II.B, eqs. interp, einstein, fl; Sec. III.B):
 *     H(lambda) = (1 - lambda) H_EAM + lambda H_Einstein, forward 0 -> 1 and
 *     backward 1 -> 0, F_0 = F_E + (W_f - W_b)/2 + dF_CM (eq. cm);
 *   - reversible scaling (Sec. II.C, eqs. H_rs, w_irr_rs, rs; Sec. III.C):
 *     H(lambda) = K + lambda U_EAM, giving F(T) for T = T0/lambda.
 *
 * Conventions
 *   Units: metal -- Angstrom, eV, ps, eV ps^2/A^2 for mass, Kelvin.
 *   Positions, velocities, forces: AoS double [n][3], positions unwrapped
 *   (the spring uses r - r0 directly); periodic orthorhombic boxes.
 *   Atom order of a crystal: ((ix*ny+iy)*nz+iz)*nbasis + b.
 *   "_dev" pointers are CUDA device memory owned by the caller; "_host"
 *   pointers are host memory owned by the caller.  "stream" is a cudaStream_t
 *   (NULL = legacy default stream).  Every call that takes a stream is
 *   stream-ordered; calls returning host values synchronise that stream.
 *   Work sign convention: dH/dlambda = U_EAM - U_Einstein on the Frenkel-Ladd
 *   path (the convention under which eq. fl holds as printed) and U_EAM on the
 *   reversible-scaling path (eq. w_irr_rs).
 *
 * Errors: every function returns ne_status; none throws or aborts.  Device
 * kernels never trap: they record problems in a device status word that is
 * read back at the end of each call (NE_ERANGE, NE_ENEIGH, NE_ENAN) and stay
 * inside their buffers whatever the data.  ne_last_error() gives the text.
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter =
 * (atom, step_lo, step_hi, replica << 4 | stream); the same seed, replica and
 * step always give the same noise, so runs are reproducible bit for bit.
 */
#ifndef NE_H
#define NE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NE_OK = 0,
    NE_EINVAL = 1,   /* bad argument (null pointer, size, box too small, ...) */
    NE_ENOMEM = 2,   /* allocation failed or capacity of the context exceeded */
    NE_ECUDA = 3,    /* a CUDA runtime call failed */
    NE_ERANGE = 4,   /* pair distance below 0.2 A, density >= rho_max, or (crystal
                        runner) an atom beyond the displacement its stencil covers */
    NE_ENEIGH = 5,   /* neighbour-list capacity exceeded */
    NE_ENAN = 6,     /* non-finite position, velocity or energy */
    NE_ETIMEOUT = 7, /* a bounded device wait gave up */
    NE_ENOTIMPL = 8
} ne_status;

typedef enum { NE_FP64 = 0, NE_MIXED = 1 } ne_precision;
typedef enum { NE_BCC = 0, NE_FCC = 1, NE_HCP = 2 } ne_lattice;
typedef enum { NE_PATH_FL = 0, NE_PATH_RS = 1 } ne_path;

/* Opaque context: EAM spline tables, neighbour lists, scratch buffers and the
 * device status word.  Not thread-safe: one host thread per context. */
typedef struct ne_ctx ne_ctx;

/* Analytic Fe-like EAM: phi(r) = A exp(-alpha (r/r_e - 1)) s(r),
 * f(r) = exp(-beta (r/r_e - 1)) s(r), F(rho) = -B sqrt(rho), s a quintic
 * taper from r_s to r_c.  Tabulated on n_knots uniform knots: phi and f on
 * [0, r_c], F on [0, rho_max]; each knot holds (value, slope) and the
 * cubic-Hermite interpolant between knots is the potential. */
typedef struct {
    double A, alpha, beta, B, r_e, r_s, r_c, rho_max;
    int n_knots;
} ne_eam_params;

/* One switching trajectory (or, in batched runs, one replica). */
typedef struct {
    double dt;         /* time step, ps */
    double T;          /* thermostat temperature, K */
    double damp;       /* Langevin damping time, ps (gamma = 1/damp; <= 0: NVE) */
    double mass;       /* eV ps^2 / A^2 */
    double k_spring;   /* Einstein spring constant k = m omega^2, eV/A^2 */
    double skin;       /* neighbour-list skin, A (r_c + skin < L/2) */
    int lambda_fn;     /* Frenkel-Ladd lambda(tau): 1 linear, 2 polynomial */
    int path;          /* ne_path */
    long long t_eq;    /* equilibration steps before each switch */
    long long t_s;     /* switching steps */
    double lambda_f;   /* reversible-scaling end point, 0 < lambda_f < 1 */
    unsigned long long seed;
    unsigned replica;  /* < 2^28 */
    int fix_cm;        /* 1: centre of mass fixed (noise and force means removed) */
    ne_precision prec;
    /* Barostat (Sec. III.C: reversible scaling at P = 0), RS path of the
     * multi-kernel runs and of the cluster runner; 0 = fixed box.  npt = 1, isotropic: each step,
     * after the second drift, ln V takes one step of the overdamped Langevin
     * equation whose stationary density is V^(N'+1) exp(-(lambda U + P0 V)/k_B T)
     * (N' = dof/3) at fixed scaled coordinates:
     *   d ln V = m [(dof k_B T + lambda W)/(3V) - P0] dt + sqrt(2 k_B T m dt / V) eta,
     * m = beta_T / tau_p, W the virial of U at the step's start, eta from
     * Philox stream 5; positions and box scale by exp(d ln V / 3) about the
     * origin.  npt = 2, per axis (the paper's fix nph aniso; non-cubic cells
     * such as hcp relax their c/a): each eps_a = ln L_a takes
     *   d eps_a = m [(dof/3 k_B T + lambda W_a)/V - P0] dt + sqrt(2 k_B T m dt / V) eta_a,
     * W_a the a-th diagonal element of the virial, eta_a the a-th normal of
     * the same draw; coordinate a and edge a scale by exp(d eps_a).  The final
     * boxes are read back with ne_ctx_boxes (pass them to the next segment).
     * With P0 = 0, eq. rs gives G(T) at zero pressure. */
    int npt;
    double P0;         /* eV / A^3, >= 0 */
    double beta_T;     /* coupling compressibility, A^3 / eV, > 0 */
    double tau_p;      /* coupling time, ps, > 0 */
    /* Several species (Sec. V: one Einstein spring per species, k_A and k_B
     * for an A-B solid).  n_species 0 or 1: every atom has `mass` and
     * `k_spring` (the fields below are ignored).  2 .. NE_MAX_SPECIES: atom i
     * of the replica has mass mass_s[species_dev[i]] and spring
     * k_s[species_dev[i]] (mass > 0, spring >= 0); species_dev is device
     * memory, one byte per atom of the replica, in its atom order, owned by
     * the caller (an index out of range is reported as NE_EINVAL at the end
     * of the call).  The EAM is the same for every species (an isotope-like
     * mixture).  The fixed centre of mass is the mass-weighted one: the
     * forces lose m_i sum_j F_j / M and the velocity increments of the
     * thermostat, sqrt((1 - c1^2) k_B T / m_i) xi_i, their centre-of-mass
     * velocity sum_j m_j dv_j / M.  With one species both reduce to the plain
     * means.  Supported by the multi-kernel runs, ne_init_velocities,
     * ne_msd_fit_species and the crystal runner. */
    int n_species;
    double mass_s[8];  /* eV ps^2 / A^2 */
    double k_s[8];     /* eV / A^2 */
    const unsigned char* species_dev;
} ne_md_params;

#define NE_MAX_SPECIES 8

/* ------------------------------------------------------------- context */
/* Create a context for up to max_atoms atoms in up to max_replicas replicas.
 * Allocates all device buffers (cudaMalloc) on the current device and builds
 * the spline tables from the analytic parameters.  *out is NULL on failure. */
ne_status ne_ctx_create(const ne_eam_params* eam, int max_atoms, int max_replicas,
                        ne_ctx** out);
ne_status ne_ctx_destroy(ne_ctx* ctx);
/* A second context with the same potential, knot parameters theta and
 * tuning as src and its own buffers for up to max_atoms atoms in up to
 * max_replicas replicas (bookkeeping; the paper has no counterpart).  Calls
 * on different contexts may run at once from different host threads on
 * different streams -- e.g. the crystal runner on one and the multi-kernel
 * path on the other; calls on one context must not overlap.  Synchronises
 * the device.  *out is NULL on failure. */
ne_status ne_ctx_clone(ne_ctx* src, int max_atoms, int max_replicas, ne_ctx** out);

/* Replace the knot parameters theta (device, double [3][n_knots][2]: phi, f,
 * F; (value, slope) per knot) and rebuild the interpolation tables. */
ne_status ne_ctx_set_theta(ne_ctx* ctx, const double* theta_dev, void* stream);
/* Copy the current knot parameters to theta_dev (same layout). */
ne_status ne_ctx_get_theta(ne_ctx* ctx, double* theta_dev, void* stream);

/* Tuning of the pair kernels: threads per atom (1, 2, 4 or 8). */
ne_status ne_ctx_set_tuning(ne_ctx* ctx, int threads_per_atom);

/* CTAs per thread-block cluster of ne_crystal_run_segment (a scheduling
 * choice; the paper has no counterpart).  0 (the default): chosen per call --
 * the smallest C whose CTAs hold each replica, or, when that C is the same
 * for every replica, the C that runs the batch fastest given how many such
 * clusters the device holds at once.  1..16: every replica uses C CTAs
 * (NE_EINVAL at run time if that is too few for a replica).  The CTA sums of
 * a replica depend on C, so results agree across C to rounding only; a fixed
 * C makes a replica's bits independent of the rest of its batch. */
ne_status ne_ctx_set_cluster_size(ne_ctx* ctx, int ctas);

/* Which persistent runner ne_crystal_run_segment uses (a scheduling choice;
 * the paper has no counterpart).  0 (the default): the cluster runner --
 * one thread-block cluster per replica, the whole replica in distributed
 * shared memory -- when every replica of the batch has at most 4096 atoms,
 * else the brick runner for the whole batch: one cooperative launch in which
 * each CTA owns a block of cells of one replica and the CTAs exchange the
 * displacements and F'(rho) through global memory (L2) between two grid
 * barriers a step, so a replica may hold up to the device's CTAs x 384
 * atoms.  1: the cluster runner only (a larger replica is NE_EINVAL).
 * 2: the brick runner for every batch.  The two give the same trajectories
 * to the rounding of the replica sums. */
ne_status ne_ctx_set_runner(ne_ctx* ctx, int runner);

/* Boxes [n_rep][3] (host) at the end of the last multi-kernel run or
 * segment of this context, or of its last crystal-runner call with the
 * barostat, in the order of its replicas: with the barostat
 * (ne_md_params.npt) the boxes it reached, else the boxes passed in.
 * NE_EINVAL if n_rep differs from that run's replica count. */
ne_status ne_ctx_boxes(ne_ctx* ctx, int n_rep, double* boxes_host);

/* Work counters since the context was created (each pointer may be NULL):
 * list_builds -- per-replica neighbour-list builds of the multi-kernel path
 * (one at the start of every run or segment, plus one each time an atom
 * strays more than skin/2 from its list-build position); stencil_visits and
 * pairs -- lattice-stencil entries examined and pairs found inside r_c by
 * ne_crystal_run_segment (pass 1), for algorithmic operation counts;
 * crystal_launches -- kernels launched by ne_crystal_run_segment (one cluster
 * kernel per replica size class a call, plus one lambda-table kernel on the
 * first call of each schedule).  Synchronises the device. */
ne_status ne_ctx_counters(ne_ctx* ctx, long long* list_builds, long long* stencil_visits,
                          long long* pairs, long long* crystal_launches);

/* Device time (ms, host double) of the last ne_crystal_run_segment or
 * ne_crystal_run_segment_cum call on this context: CUDA events recorded on
 * the call's stream just before its first cluster launch and after the last
 * size class has joined back, so the figure is the kernels' own duration,
 * without the call's host work (bookkeeping for the roofline report; the
 * paper has no counterpart).  NE_EINVAL if no such call has run. */
ne_status ne_ctx_last_run_ms(ne_ctx* ctx, double* ms_host);

/* Launch plan of the last ne_crystal_run_segment or
 * ne_crystal_run_segment_cum call on this context (bookkeeping for reports;
 * the paper has no counterpart): runner 1 the cluster runner, 2 the brick
 * runner; threads_per_atom the threads on each atom in the pair passes;
 * ctas the CTAs of the call's launches; cluster_ctas the CTAs per cluster of
 * the cluster runner's largest (0 for the brick runner).  Each pointer may
 * be NULL.  NE_EINVAL if no crystal-runner call has planned a launch. */
ne_status ne_ctx_crystal_plan(ne_ctx* ctx, int* runner, int* threads_per_atom, int* ctas, int* cluster_ctas);

/* Status bits recorded by the last call, and its message (msg may be NULL). */
ne_status ne_last_error(ne_ctx* ctx, int* device_status, char* msg, int msg_len);

/* ------------------------------------------------------------- crystal */
/* Lattice sites r0 (Sec. II.B, eq. einstein) of an nx*ny*nz bcc, fcc or hcp
 * supercell with lattice parameter a.  x0_host: [n][3] with n = 2 (bcc) or 4
 * (fcc, hcp) * nx*ny*nz (may be NULL to query n); box[3] = a*(nx, ny, nz)
 * for bcc and fcc (hcp: see ne_create_crystal_ca).  Atom order
 * ((ix*ny+iy)*nz+iz)*nb+b. */
ne_status ne_create_crystal(ne_lattice lattice, double a, int nx, int ny, int nz,
                            double* x0_host, double box[3], int* n_out);
/* Same with the hcp axial ratio given (c = c_over_a * a, > 0; ignored for
 * bcc and fcc).  hcp uses the orthohexagonal cell with edges (a, sqrt(3) a,
 * c) and four atoms at fractions (0,0,0), (1/2,1/2,0), (0,1/3,1/2),
 * (1/2,5/6,1/2); box = (nx a, ny sqrt(3) a, nz c).  ne_create_crystal uses
 * the ideal sqrt(8/3) for hcp. */
ne_status ne_create_crystal_ca(ne_lattice lattice, double a, double c_over_a, int nx, int ny, int nz,
                               double* x0_host, double box[3], int* n_out);

/* ------------------------------------------------------------ energies */
/* EAM energy U (Sec. II.B, eq. H) and forces at one configuration:
 * U = sum_{i<j} phi(r_ij) + sum_i F(rho_i), rho_i = sum_j f(r_ij).
 * x_dev [n][3]; f_dev [n][3] (may be NULL); e_dev: 1 double; rho_dev [n]
 * (may be NULL).  NE_MIXED evaluates pairs in FP32 with double-float sums
 * (FP64-class precision from FP32 operations). */
ne_status ne_eam_energy_forces(ne_ctx* ctx, ne_precision prec, const double* x_dev,
                               int n, const double box[3], double* f_dev,
                               double* e_dev, double* rho_dev, void* stream);

/* Configurational virial of the EAM at one configuration, for the pressure
 * that fixes the lattice parameter (Sec. III.A: the crystal is brought to
 * zero pressure before switching):
 *   W = sum_{i<j} r_ij . F_ij = -sum_{i<j} r_ij [phi'(r_ij) + (F'(rho_i) +
 *       F'(rho_j)) f'(r_ij)] = -dU/d(eps) under x -> (1+eps) x, box -> (1+eps) box,
 * so that P = (N_dof k_B T + W) / (3 V) at temperature T.  Always FP64.
 * x_dev [n][3] (device, unwrapped positions); w_dev: 1 double (device).
 * NE_ERANGE as ne_eam_energy_forces. */
ne_status ne_eam_virial(ne_ctx* ctx, const double* x_dev, int n, const double box[3], double* w_dev,
                        void* stream);

/* Allocation-free variant of ne_eam_energy_forces, for callers that cannot
 * allocate device memory once they are running -- an engine or framework
 * that has reserved the device memory for its own pool, or a real-time
 * pipeline that forbids cudaMalloc after start-up (it can synchronise the
 * device and can fail).  The paper has no counterpart; it is a deployment
 * convenience.  No context is needed and nothing is allocated: no
 * cudaMalloc, cudaFree or allocating library call.  The spline tables (built
 * from *eam on every call), cell arrays, neighbour lists and per-atom buffers
 * live in one file-scope device array of NE_NOALLOC_SCRATCH_BYTES bytes that
 * every GPU which loads the library holds until the process exits.
 *   Limits: n <= NE_NOALLOC_MAX_ATOMS and eam->n_knots <=
 *   NE_NOALLOC_MAX_KNOTS, else NE_ENOMEM; box edges > 2 r_c, else NE_EINVAL.
 *   Arguments and results as for ne_eam_energy_forces (no rho output).
 *   Each call looks up the device address of the array on the current
 *   device (cudaGetSymbolAddress), so the address stays right after a
 *   cudaDeviceReset; a call whose stream is capturing reuses the address of
 *   that device's last lookup instead, so make the first call on a device
 *   before any stream capture.  Analytic parameters that are not finite
 *   (the NaN placeholders of a potential loaded from a file) are refused
 *   with NE_EINVAL: this entry point tabulates the analytic form only.
 *   All calls on a device share the one array, which keeps the previous
 *   call's contents (the call clears what must start at zero): calls that
 *   overlap on the GPU -- on different streams or host threads -- race and
 *   must be serialised by the caller.  The call synchronises `stream`. */
#define NE_NOALLOC_MAX_ATOMS 2048
#define NE_NOALLOC_MAX_KNOTS 5000
#define NE_NOALLOC_SCRATCH_BYTES (4608u * 1024u)
ne_status ne_eam_energy_forces_noalloc(const ne_eam_params* eam, ne_precision prec,
                                       const double* x_dev, int n, const double box[3],
                                       double* f_dev, double* e_dev, void* stream);

/* Einstein crystal (eq. einstein): U_E = sum_i k/2 |r_i - r0_i|^2 into e_dev
 * (1 double) and F_E = -k (r - r0) into f_dev [n][3] (may be NULL). */
ne_status ne_spring_forces(const double* x_dev, const double* x0_dev, int n, double k,
                           double* f_dev, double* e_dev, void* stream);

/* Backward pass of the EAM energy for automatic differentiation: given the
 * upstream gradient gE = dL/dU, writes gx_dev [n][3] = gE dU/dx = -gE F and
 * gtheta_dev [3][n_knots][2] = gE dU/dtheta for every knot value and slope of
 * phi, f and F.  rho is recomputed, not stored.  NE_MIXED: FP32 pair
 * arithmetic, FP32 per-block bins summed over the blocks in FP64, and the F
 * bins in exact 64-bit fixed point; NE_FP64: FP64 throughout. */
ne_status ne_eam_backward(ne_ctx* ctx, ne_precision prec, const double* x_dev, int n,
                          const double box[3], double gE, double* gx_dev,
                          double* gtheta_dev, void* stream);

/* Same, adding gE dU/dtheta into gtheta_acc_dev [3][n_knots][2] instead of
 * overwriting it, for averages of dU/dtheta over configurations of a run:
 * the free energy's parameter gradient is dF/dtheta = <dU/dtheta> in the
 * EAM ensemble (lambda = 0 of the FL path), and sum_k dlambda_k dU/dtheta(x_k)
 * is the derivative of a switching work at fixed trajectory. */
ne_status ne_eam_backward_acc(ne_ctx* ctx, ne_precision prec, const double* x_dev, int n,
                              const double box[3], double gE, double* gtheta_acc_dev, void* stream);

/* ------------------------------------------------------------- dynamics */
/* The Langevin noise of the path: for atoms 0..n-1 the three normals of one
 * Philox4x32-10 block with key = seed and counter = (atom, step_lo, step_hi,
 * replica << 4 | noise_stream), uniforms (w + 1/2) 2^-32 and two Box-Muller
 * pairs (fourth normal unused); NE_MIXED draws them in FP32 from the top 24
 * bits of each word, as the mixed-precision runs do.  z_dev: double [n][3]. */
ne_status ne_noise(unsigned long long seed, unsigned replica, int noise_stream, long long step,
                   int n, ne_precision prec, double* z_dev, void* stream);

/* Maxwell-Boltzmann velocities at md->T: Philox normals (stream 1, step 0)
 * times sqrt(kT/m), total momentum removed when md->fix_cm, rescaled to
 * exactly T over 3n-3 (fix_cm) or 3n degrees of freedom.  v_dev [n][3]. */
ne_status ne_init_velocities(ne_ctx* ctx, const ne_md_params* md, int n, double* v_dev,
                             void* stream);

/* One Langevin step at fixed positions of the schedule: the Hamiltonian jumps
 * from lambda_k to lambda_k1 at x_k (adding (lambda_k1 - lambda_k) dH/dlambda
 * to *W_dev, the discrete work sum of Sec. II.A), then one BAOAB step of
 * H(lambda_k1) with Philox noise (stream 4, counter step).  md->path selects
 * the Frenkel-Ladd blend or the scaled potential.  Forces are evaluated at
 * x_k and x_{k+1}.  x_dev, v_dev [n][3] updated in place; x0_dev sites. */
ne_status ne_langevin_step(ne_ctx* ctx, const ne_md_params* md, double* x_dev,
                           double* v_dev, const double* x0_dev, int n, const double box[3],
                           long long step, double lambda_k, double lambda_k1,
                           double* W_dev, void* stream);

/* Four-phase switching run (fix ti/spring of Sec. III.B; Sec. III.C for
 * md->path = NE_PATH_RS): t_eq steps at the initial lambda, t_s steps
 * switching, t_eq steps at the final lambda, t_s steps switching back.
 * x_dev, v_dev [n][3] in/out; x0_dev sites.  W_fwd_dev, W_bwd_dev: 1 double
 * each (the two irreversible works).  Wcum_fwd_dev, Wcum_bwd_dev (nullable):
 * t_s+1 doubles, cumulative work after each switching step.  trace_dev
 * (nullable): every trace_stride steps 8 doubles (step, lambda, dH/dlambda,
 * U_EAM, U_E, T_internal, W_f, W_b), floor((2 t_eq + 2 t_s - 1)/stride) + 1
 * rows.  Noise stream 0 (FL) or 2 (RS), counter = step of the run. */
ne_status ne_switch_run(ne_ctx* ctx, const ne_md_params* md, double* x_dev,
                        double* v_dev, const double* x0_dev, int n, const double box[3],
                        double* W_fwd_dev, double* W_bwd_dev, double* Wcum_fwd_dev,
                        double* Wcum_bwd_dev, double* trace_dev, int trace_stride,
                        void* stream);

/* Reversible-scaling run (Sec. III.C): ne_switch_run with path = NE_PATH_RS
 * and lambda from 1 to lambda_f and back; Wcum_*_dev: t_s+1 doubles each. */
ne_status ne_rs_run(ne_ctx* ctx, const ne_md_params* md, double lambda_f, double* x_dev,
                    double* v_dev, const double* x0_dev, int n, const double box[3],
                    double* Wcum_fwd_dev, double* Wcum_bwd_dev, void* stream);

/* Many independent replicas of the four-phase run in one batch (the ten
 * independent realisations of Sec. III.B, generalised to uneven sizes and
 * temperatures).  md[n_rep] host array: per-replica T, k_spring, seed,
 * replica, mass, skin; dt, damp, lambda_fn, path, lambda_f, t_eq, t_s,
 * fix_cm and prec must agree across replicas.  offsets_host[n_rep+1]: atom
 * ranges of the replicas in the concatenated x/v/x0 arrays (device, [N][3]).
 * boxes_host[n_rep][3].  W_fwd_dev, W_bwd_dev: n_rep doubles each. */
ne_status ne_switch_run_batched(ne_ctx* ctx, const ne_md_params* md, int n_rep,
                                const int* offsets_host, double* x_dev, double* v_dev,
                                const double* x0_dev, const double* boxes_host,
                                double* W_fwd_dev, double* W_bwd_dev, void* stream);

/* Steps [step_begin, step_begin + n_steps) of the same four-phase schedule
 * for n_rep replicas (arguments as in ne_switch_run_batched), continuing a
 * run: x_dev, v_dev hold the state at step step_begin (complete velocities)
 * and are advanced in place; W_dev [n_rep][2] (device) accumulates the
 * (forward, backward) work in place.  Running [0, a) then [a, S) gives the
 * same bits as [0, S) -- checkpoint/resume -- as long as every atom stays
 * within skin/2 of its site (the neighbour list is built from the sites).
 * NE_EINVAL if the range leaves [0, 2 t_eq + 2 t_s]. */
ne_status ne_switch_run_segment(ne_ctx* ctx, const ne_md_params* md, int n_rep,
                                const int* offsets_host, double* x_dev, double* v_dev,
                                const double* x0_dev, const double* boxes_host, double* W_dev,
                                long long step_begin, long long n_steps, void* stream);

/* ne_switch_run_segment that also records the cumulative works of the two
 * switches for every replica, for eq. rs over a batch of seeds (Sec. III.C):
 * Wcum_dev (device, double [n_rep][2][t_s + 1]; [r][0] forward, [r][1]
 * backward) gets, for every switching step k of the range, [k + 1] = replica
 * r's W after that step and [0] = 0 at the switch's first step -- the layout
 * of ne_crystal_run_segment_cum.  Errors as ne_switch_run_segment; NE_EINVAL
 * if Wcum_dev is NULL. */
ne_status ne_switch_run_segment_cum(ne_ctx* ctx, const ne_md_params* md, int n_rep,
                                    const int* offsets_host, double* x_dev, double* v_dev,
                                    const double* x0_dev, const double* boxes_host, double* W_dev,
                                    double* Wcum_dev, long long step_begin, long long n_steps,
                                    void* stream);

/* ne_switch_run_segment that also accumulates the parameter gradient along
 * the run (the backward pass of Sec. III.B's switching runs; the paper has no
 * gradient): after the force evaluation at each x_k, k = step_begin ..
 * step_begin + n_steps, gtheta_dev += w_dev[k - step_begin] * dU/dtheta(x_k),
 * summed over the replicas, with the step's own neighbour list and rho (no
 * recomputation; a zero weight skips the step's backward).  w_dev: device,
 * double [n_steps + 1]; gtheta_dev: device, double [3][n_knots][2] (phi, f,
 * F; value and slope per knot), accumulated.  E.g. w = 1 every `stride`
 * steps at lambda = 0 gives sum dU/dtheta for <dU/dtheta> = dF_0/dtheta, and
 * w_k = lambda_k - lambda_(k-stride) over a switch the derivative of W at
 * fixed trajectory.  Mixed precision bins in FP32 per block and sums them in
 * FP64; FP64 adds with FP64 atomics.  Errors as ne_switch_run_segment. */
ne_status ne_switch_run_segment_grad(ne_ctx* ctx, const ne_md_params* md, int n_rep,
                                     const int* offsets_host, double* x_dev, double* v_dev,
                                     const double* x0_dev, const double* boxes_host, double* W_dev,
                                     long long step_begin, long long n_steps, const double* w_dev,
                                     double* gtheta_dev, void* stream);

/* A crystal replica: nx*ny*nz cells of a bcc, fcc or hcp lattice with
 * parameter a (hcp: the orthohexagonal cell of ne_create_crystal_ca); its
 * sites r0 and atom order are those of ne_create_crystal_ca. */
typedef struct {
    ne_lattice lattice;
    double a;
    int nx, ny, nz;
    double c_over_a;  /* hcp only: c / a; 0 = ideal sqrt(8/3) */
} ne_crystal;

/* Persistent batched runner for crystals (mixed precision): steps
 * [step_begin, step_begin + n_steps) of the four-phase schedule (Sec. III.B /
 * III.C) for n_rep crystal replicas, each advanced by one thread-block cluster
 * for the whole range in one launch.  Same semantics as ne_switch_run_segment
 * with x0 = the sites of cr[r]: x_dev, v_dev [N][3] (replicas concatenated in
 * order, each in crystal atom order) hold the state at step_begin and are
 * advanced in place; W_dev [n_rep][2] accumulates (forward, backward) work.
 * md[r].prec must be NE_MIXED; at least 3 cells per axis and box edges
 * > 2 r_c + 1.2 A; replicas above 4096 atoms run on the brick runner
 * (ne_ctx_set_runner), which needs the batch's CTAs (one per 96-768 atoms)
 * to fit the device at once (NE_ENOMEM otherwise); a grid barrier that
 * waits longer than a few seconds gives NE_ETIMEOUT.  The barostat
 * (md[r].npt, reversible-scaling path) runs on both runners: the box and
 * the lattice sites scale with it, ne_ctx_boxes reads the boxes the call
 * reached, and the next segment takes cr[r].a = box edge / cells (and, per
 * axis, c/a) of that box.  Neighbours come from a
 * lattice stencil covering displacements up to D = 2 A from the sites (in a
 * small box it holds two periodic images of some sites, at most one of them
 * within r_c); a replica whose atoms stray further is reported as NE_ERANGE.
 * A replica that raises an error (NE_ERANGE, NE_ENAN, NE_ENEIGH) keeps its
 * x, v and W of step_begin -- its run is void and can be repeated elsewhere
 * (ne_ctx_replica_status names it) -- while the others are advanced.  Noise,
 * work and schedule are those of ne_switch_run_segment.
 * The launch plan (stencils, replica table, cluster size) is built on the
 * first call for a batch and kept in the context; later calls with the same
 * crystals and per-replica parameters only launch, so short segments
 * (checkpoints, cumulative-work chunks) pay no set-up.  The table of lambda
 * over the whole schedule is likewise computed once per schedule. */
ne_status ne_crystal_run_segment(ne_ctx* ctx, const ne_md_params* md, const ne_crystal* cr, int n_rep,
                                 double* x_dev, double* v_dev, double* W_dev, long long step_begin,
                                 long long n_steps, void* stream);

/* ne_crystal_run_segment that also records the cumulative works of the two
 * switches, as ne_rs_run does for eq. rs (Sec. III.C): Wcum_dev (device,
 * double [n_rep][2][t_s + 1]; [r][0] forward, [r][1] backward) gets, for
 * every switching step k of the range, [k + 1] = the replica's W after that
 * step, and [0] = 0 at the switch's first step.  Errors as
 * ne_crystal_run_segment; NE_EINVAL if Wcum_dev is NULL. */
ne_status ne_crystal_run_segment_cum(ne_ctx* ctx, const ne_md_params* md, const ne_crystal* cr, int n_rep,
                                     double* x_dev, double* v_dev, double* W_dev, double* Wcum_dev,
                                     long long step_begin, long long n_steps, void* stream);

/* Outcome per replica of the last ne_crystal_run_segment call that launched
 * (bookkeeping; the paper has no counterpart): out_host[r] (host, n_rep ints)
 * = NE_OK or the error replica r raised (NE_ENAN, NE_ERANGE, ...).  A replica
 * that left the runner's range (a hop or melting at high T) can then be rerun
 * alone on the multi-kernel path while the others keep their results: each
 * replica's trajectory depends only on its own inputs and noise stream.
 * NE_EINVAL if n_rep differs from that call's.  Synchronises the device. */
ne_status ne_ctx_replica_status(ne_ctx* ctx, int n_rep, int* out_host);

/* Timing hook (autotuning and roofline reports): the steps of
 * ne_switch_run_segment launched one by one, with CUDA events on the
 * launching stream around each kernel.  ms_host[4] receives the mean
 * duration (ms) of one launch of: 0 neighbour-list check/build, 1 pass 1
 * (density), 2 pass 2 (forces), 3 fused step; launches_host[4] the number of
 * launches timed.  1 <= n_steps <= 100000.  Same state semantics as
 * ne_switch_run_segment. */
ne_status ne_profile_segment(ne_ctx* ctx, const ne_md_params* md, int n_rep,
                             const int* offsets_host, double* x_dev, double* v_dev,
                             const double* x0_dev, const double* boxes_host, double* W_dev,
                             long long step_begin, long long n_steps, double* ms_host,
                             long long* launches_host, void* stream);

/* Spring constant from the mean-squared displacement (Sec. III.A, eq. msd):
 * n_eq Langevin steps at lambda = 0, then n_samples blocks of stride steps,
 * msd = mean over samples of (1/n) sum |(r_i - r0_i) - (R - R0)|^2 and
 * k = 3 k_B T / msd.  Noise stream 3.  x_dev, v_dev updated; results to host. */
ne_status ne_msd_fit(ne_ctx* ctx, const ne_md_params* md, double* x_dev, double* v_dev,
                     const double* x0_dev, int n, const double box[3], long long n_eq,
                     long long n_samples, int stride, double* msd_host, double* k_host,
                     void* stream);

/* Eq. msd per species (Sec. V: one spring per species), for a replica with
 * species tables (md->n_species >= 2): as ne_msd_fit, the samples taken
 * about the mass-weighted centre, msd_s = mean over samples of
 * (1/N_s) sum over the atoms of species s of |(r_i - r0_i) - (R - R0)|^2,
 * R the mass-weighted centre, and k_s = 3 k_B T / msd_s.  msd_s_host and
 * k_s_host: md->n_species doubles each (either may be NULL; a species with
 * no atom gets 0). */
ne_status ne_msd_fit_species(ne_ctx* ctx, const ne_md_params* md, double* x_dev, double* v_dev,
                             const double* x0_dev, int n, const double box[3], long long n_eq,
                             long long n_samples, int stride, double* msd_s_host, double* k_s_host,
                             void* stream);

/* ne_msd_fit for a batch of replicas at once, each at its own size and
 * temperature (Sec. III.A: the spring of a run comes from the msd at that
 * run's N and T -- e.g. one spring per replica of an uneven batch drawn over
 * 300-1600 K).  md[n_rep]: per-replica T, seed, replica, mass; dt, damp,
 * fix_cm and prec shared.  offsets_host[n_rep+1], x_dev, v_dev, x0_dev and
 * boxes_host as in ne_switch_run_batched.  msd_host, k_host: n_rep doubles
 * each (either may be NULL), k_r = 3 k_B T_r / msd_r.  One species per replica
 * (n_species >= 2: NE_EINVAL; see ne_msd_fit_species). */
ne_status ne_msd_fit_batched(ne_ctx* ctx, const ne_md_params* md, int n_rep, const int* offsets_host,
                             double* x_dev, double* v_dev, const double* x0_dev,
                             const double* boxes_host, long long n_eq, long long n_samples, int stride,
                             double* msd_host, double* k_host, void* stream);

/* ------------------------------------------------------------ assembly */
/* Host only, FP64.  Lambda in force at the start of step `step` of md's
 * four-phase schedule (Sec. III.B, fix ti/spring; Sec. III.C for
 * md->path = NE_PATH_RS), the value every run of this library uses: t_eq
 * steps at lambda_i (FL 0, RS 1), the switch over t_s steps with tau =
 * elapsed steps / t_s (FL: tau, or tau^5 (70 tau^4 - 315 tau^3 + 540 tau^2
 * - 420 tau + 126) for lambda_fn 2; RS: 1 / (1 + tau (1/lambda_f - 1))),
 * t_eq steps at lambda_f (FL 1), the switch back (FL: 1 - lambda(tau); RS:
 * lambda(1 - tau)).  The work of step s is (lambda(s+1) - lambda(s))
 * dH/dlambda(x_s).  0 <= step <= 2 t_eq + 2 t_s, else NE_EINVAL. */
ne_status ne_lambda(const ne_md_params* md, long long step, double* lambda_host);

/* Host only, FP64.  Pressure of an NVT state (Sec. III.A: the crystal is
 * brought to zero pressure before switching) from n_samples configurational
 * virials W_host (ne_eam_virial, eV):
 *   P = (n_dof k_B T + <W>) / (3 V)   (eV/A^3; n_dof = 3N - 3 with the
 *   centre of mass fixed), and its standard error s(W) / sqrt(n) / (3 V)
 * (0 for one sample; stderr_host may be NULL). */
ne_status ne_pressure(int n_dof, double T, double V, const double* W_host, int n_samples,
                      double* P_host, double* stderr_host);

/* Host only, FP64.  Jarzynski's equality (eq. jarz, Sec. II.A): the
 * free-energy difference from the exponential average of the work done on
 * the system over independent realisations started in equilibrium,
 *   dF = -k_B T ln[(1/n) sum_s exp(-W_s / k_B T)],
 * evaluated with the smallest W factored out (no overflow).  W_host
 * [n_seeds] in eV (work done on the system: for this library's switching
 * works, W = -W_fwd or -W_bwd); *dF_out in eV.  Exact in the limit of many
 * realisations, biased upward by roughly the dissipation when few are
 * available (Sec. II.A). */
ne_status ne_jarzynski(double T, const double* W_host, int n_seeds, double* dF_out);

/* Host only, FP64.  Frenkel-Ladd free energy per atom (eq. fl + eq. cm):
 * F_0 = F_E + (mean W_f - mean W_b)/2 + dF_CM, F_E = 3 N k_B T ln(hbar w /
 * k_B T), dF_CM = k_B T ln[(N/V)(2 pi k_B T/(N k))^{3/2}]; stderr over seeds
 * of (W_f - W_b)/(2N); Ediss = -(mean W_f + mean W_b)/(2N) (eq. Ediss). */
ne_status ne_free_energy(int n, double V, double T, double mass, double k,
                         const double* W_fwd_host, const double* W_bwd_host, int n_seeds,
                         double* F_per_atom, double* stderr_per_atom,
                         double* Ediss_per_atom);

/* Host only, FP64.  Eq. fl + eq. cm for a solid of several species with one
 * Einstein spring per species (Sec. V: k_A, k_B for an A-B compound).
 * species_host [n] gives each atom's species, 0 <= species[i] < n_species;
 * mass_s_host and k_s_host [n_species] its mass (eV ps^2/A^2) and spring
 * (eV/A^2).  F_E = sum_i 3 k_B T ln(hbar w_i / k_B T), w_i^2 = k_i/m_i.  The
 * fixed centre of mass is the mass-weighted one, so the factor
 * 2 pi k_B T/(N k) of eq. cm becomes 2 pi sigma^2, sigma^2 = k_B T
 * sum_i (m_i/M)^2 / k_i (the per-axis variance of that centre in the
 * Einstein crystal), with eq. cm's leading N/V kept.  With one species this
 * is ne_free_energy.  W_*_host [n_seeds]; outputs per atom as in
 * ne_free_energy (each nullable).  NE_EINVAL for a species index out of
 * range or a non-positive mass or spring.  The switching runs themselves
 * are single-species in this library. */
ne_status ne_free_energy_species(int n, const int* species_host, int n_species,
                                 const double* mass_s_host, const double* k_s_host,
                                 double V, double T, const double* W_fwd_host,
                                 const double* W_bwd_host, int n_seeds,
                                 double* F_per_atom, double* stderr_per_atom,
                                 double* Ediss_per_atom);

/* Host only, FP64.  Eq. rs on a temperature grid: F_0(T) = F_0(T0)/l +
 * (3/2) N k_B T0 ln(l)/l + [W_{1->l} - W_{l->1}]/(2 l), l = T0/T, from the
 * seed-averaged cumulative works Wcum_*_host [n_seeds][t_s+1].  F0_T0 is the
 * total free energy at T0 (eV); F_per_atom [n_T]. */
ne_status ne_rs_free_energy(int n, double T0, double F0_T0, double lambda_f,
                            long long t_s, const double* Wcum_fwd_host,
                            const double* Wcum_bwd_host, int n_seeds,
                            const double* T_grid_host, int n_T, double* F_per_atom);

#ifdef __cplusplus
}
#endif
#endif
