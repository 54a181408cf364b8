// ne_api.cu -- the C ABI of libne.so (include/ne.h): context and buffers,
// batch set-up, the run loops (captured in CUDA graphs), status mapping and
// the host-side free-energy assembly.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ne.h"
#include "ne_cluster.cuh"
#include "ne_internal.cuh"

static_assert(NE_MAX_SPECIES == NE_MAX_SPECIES_DEV, "species table size");

namespace {

const double kB = 8.617333262e-5;      // eV/K
const double HBAR = 6.582119569e-4;    // eV ps
const double PI = 3.14159265358979323846;

template <typename T>
cudaError_t dalloc(T** p, size_t n)
{
    return cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
}

}  // namespace

// Launch plan of a crystal-runner batch, cached in the context: built on the
// first call for a batch and reused while the batch stays the same, so a call
// is a memset, the launches and the status read.
struct CrGroup {
    int b, e;     // replicas [b, e) of the sorted table: one size class
    int C;        // CTAs per cluster
    size_t smem;  // dynamic shared memory per CTA
    int k_lo;     // first spline interval held in shared memory
};
struct CrPlan {
    bool valid = false;
    std::vector<double> key;
    std::vector<XRep> xs;  // replica table, sorted by size class (uploaded to ctx->xrep)
    std::vector<CrGroup> groups;
    std::vector<float4> sv;
    std::vector<float> sd;
    // brick runner (replicas larger than a cluster holds): one cooperative
    // launch of n_cta CTAs, tpa threads per atom, CTA -> replica table
    bool brick = false;
    bool npt = false;  // a replica has the barostat
    int tpa = 0, n_cta = 0, k_lo = 0;
    size_t smem = 0;
    std::vector<int> cta_rep;
};

struct ne_ctx {
    ne_eam_params eam{};
    int max_atoms = 0, max_rep = 0, tiles_cap = 0, cells_cap = 0, tpa = 4;
    int cluster_c = 0;  // crystal runner: CTAs per cluster (0: chosen per batch)
    int last_nrep = 0;  // replicas of the last multi-kernel run (ne_ctx_boxes)
    int last_nrep_cr = 0;  // replicas of the last crystal-runner call (ne_ctx_replica_status)
    double* theta = nullptr;
    float4* pf32 = nullptr;
    ned4* pf64 = nullptr;
    float4* F32 = nullptr;
    ned4* F64 = nullptr;
    float4 *pos32 = nullptr, *posF = nullptr, *pbuild = nullptr, *f32 = nullptr;
    double *f64 = nullptr, *dF64 = nullptr, *rho = nullptr, *xi64 = nullptr;
    float* xi32 = nullptr;
    int *nbr = nullptr, *ncnt = nullptr, *sl = nullptr, *scnt = nullptr;
    int *cellof = nullptr, *sorted = nullptr, *cstart = nullptr, *cfill = nullptr;
    double *partA = nullptr, *partB = nullptr, *tot = nullptr, *W = nullptr, *scratch = nullptr;
    unsigned* tile_done = nullptr;
    int *flags = nullptr, *building = nullptr, *status = nullptr, *tile_rep = nullptr;
    int* rep_status = nullptr;  // crystal runner: status bits per replica of the last call (= status + 1)
    int* status_host = nullptr; // pinned host copy of the status word
    RepDev* rep = nullptr;
    long long* step_ctr = nullptr;
    unsigned long long* rebuilds = nullptr;
    unsigned long long* work = nullptr;  // crystal runner: [0] stencil entries visited, [1] pairs < r_c
    XRep* xrep = nullptr;
    double* lam_tab = nullptr;  // lambda of each step of the crystal runner's schedule
    long long lam_cap = 0;
    Sched lam_sched{};          // the schedule lam_tab holds
    bool lam_valid = false;
    CrPlan plan;                // launch plan of the last crystal-runner batch
    int runner = 0;             // 0 automatic, 1 cluster runner only, 2 brick runner for every batch
    ne::BrickBufs bb{};         // brick runner's exchange buffers (allocated on first use)
    int* cta_rep = nullptr;     // brick runner: replica of each CTA
    int bb_ctas = 0;            // CTAs the partials buffer holds
    double* cr_boxes = nullptr; // crystal runner with the barostat: each replica's box at the call's end
    bool boxes_from_runner = false;
    cudaEvent_t ev_run[2] = {}; // around the cluster launches of the last crystal-runner call
    bool run_timed = false;
    cudaStream_t gst[16] = {};  // crystal runner: one stream per replica size class
    cudaEvent_t gev[17] = {};
    float4* st_vec = nullptr;
    float* st_dist = nullptr;
    float* bins = nullptr;
    int bins_blocks = 0;
    std::vector<RepDev> rep_h;
    std::vector<int> tile_rep_h;
    int last_bits = 0;
    long long cr_launches = 0;  // kernels launched by ne_crystal_run_segment
    std::string msg;
    Tables tab{};
};

namespace {

ne_status fail(ne_ctx* c, ne_status st, const std::string& m)
{
    if (c) c->msg = m;
    return st;
}

#define NE_CU(call)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(ctx, NE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

// ------------------------------------------------------------ potential
// The analytic Fe-like EAM and its knot parameters (value and slope at each
// knot); the embedding slope at rho = 0 is infinite, so that knot takes the
// secant slope to its neighbour.
void taper(const ne_eam_params& p, double r, double& s, double& ds)
{
    if (r <= p.r_s) { s = 1.0; ds = 0.0; return; }
    if (r >= p.r_c) { s = 0.0; ds = 0.0; return; }
    const double w = p.r_c - p.r_s, x = (r - p.r_s) / w, om = 1.0 - x;
    s = om * om * om * (1.0 + x * (3.0 + 6.0 * x));
    ds = -30.0 * x * x * om * om / w;
}

void analytic(const ne_eam_params& p, int fn, double x, double& y, double& dy)
{
    if (fn == 2) {
        y = -p.B * std::sqrt(x);
        dy = -0.5 * p.B / std::sqrt(x);
        return;
    }
    double s, ds;
    taper(p, x, s, ds);
    const double c = fn == 0 ? p.alpha : p.beta;
    const double e = (fn == 0 ? p.A : 1.0) * std::exp(-c * (x / p.r_e - 1.0));
    y = e * s;
    dy = e * (ds - c / p.r_e * s);
}

std::vector<double> make_theta(const ne_eam_params& p)
{
    const int nk = p.n_knots;
    std::vector<double> th((size_t)6 * nk);
    for (int fn = 0; fn < 3; ++fn) {
        const double h = (fn == 2 ? p.rho_max : p.r_c) / (nk - 1);
        for (int k = 0; k < nk; ++k) {
            double y, dy;
            if (fn == 2 && k == 0) {
                double y1, d1;
                analytic(p, 2, h, y1, d1);
                y = 0.0;
                dy = y1 / h;
            } else {
                analytic(p, fn, k * h, y, dy);
            }
            th[((size_t)fn * nk + k) * 2] = y;
            th[((size_t)fn * nk + k) * 2 + 1] = dy;
        }
    }
    return th;
}

void fill_tables(ne_ctx* ctx)
{
    Tables& t = ctx->tab;
    const ne_eam_params& p = ctx->eam;
    t.pf32 = ctx->pf32;
    t.pf64 = ctx->pf64;
    t.F32 = ctx->F32;
    t.F64 = ctx->F64;
    t.nk = p.n_knots;
    t.h_r = p.r_c / (p.n_knots - 1);
    t.inv_h_r = (p.n_knots - 1) / p.r_c;
    t.h_rho = p.rho_max / (p.n_knots - 1);
    t.inv_h_rho = (p.n_knots - 1) / p.rho_max;
    t.r_c = p.r_c;
    t.rho_max = p.rho_max;
    t.inv_h_rf = (float)t.inv_h_r;
    t.rcf = (float)p.r_c;
    t.rc2f = (float)(p.r_c * p.r_c);
    t.rmin2f = (float)(NE_RMIN * NE_RMIN);
    t.inv_h_rhof = (float)t.inv_h_rho;
}

// ------------------------------------------------------------ batches
struct RunArgs {
    double* x;
    double* v;
    const double* x0;
    double* W;
    double* Wcum;
    double* trace;
    int trace_stride, trace_rows;
    double* rho;
};

// Species tables of one replica (Sec. V): per-species mass, spring, noise
// amplitude and half-step factor, the atoms' species read back and checked
// (every index in range) and the total mass formed on the host.
ne_status species_tables(ne_ctx* ctx, const ne_md_params& m, int n, double c1, RepDev& R, cudaStream_t st)
{
    if (m.n_species < 2 || m.n_species > NE_MAX_SPECIES || !m.species_dev)
        return fail(ctx, NE_EINVAL, "species: 2 .. NE_MAX_SPECIES species and a device species array");
    for (int q = 0; q < m.n_species; ++q)
        if (!(m.mass_s[q] > 0) || !(m.k_s[q] >= 0))
            return fail(ctx, NE_EINVAL, "species: masses must be positive and springs non-negative");
    std::vector<unsigned char> sp(n);
    NE_CU(cudaMemcpyAsync(sp.data(), m.species_dev, (size_t)n, cudaMemcpyDeviceToHost, st));
    NE_CU(cudaStreamSynchronize(st));
    double M = 0.0;
    for (int a = 0; a < n; ++a) {
        if (sp[a] >= m.n_species) return fail(ctx, NE_EINVAL, "species index out of range");
        M += m.mass_s[sp[a]];
    }
    R.nsp = m.n_species;
    R.sp = m.species_dev;
    R.M = M;
    for (int q = 0; q < m.n_species; ++q) {
        R.ms[q] = m.mass_s[q];
        R.ks[q] = m.k_s[q];
        R.c2s[q] = std::sqrt((1.0 - c1 * c1) * kB * m.T / m.mass_s[q]);
        R.hdts[q] = 0.5 * m.dt / m.mass_s[q];
    }
    return NE_OK;
}

ne_status setup_batch(ne_ctx* ctx, int n_rep, const int* off, const double* boxes,
                      const ne_md_params* md, int md_stride, double skin_override, DevBatch& B,
                      const RunArgs& a, cudaStream_t st, bool geometry = true)
{
    if (n_rep < 1 || n_rep > ctx->max_rep) return fail(ctx, NE_ENOMEM, "replica count exceeds the context");
    if (off[0] != 0) return fail(ctx, NE_EINVAL, "offsets must start at 0");
    const int n_tot = off[n_rep];
    if (n_tot > ctx->max_atoms) return fail(ctx, NE_ENOMEM, "atom count exceeds the context");
    ctx->rep_h.assign(n_rep, RepDev{});
    ctx->tile_rep_h.clear();
    int cells = 0, npt_any = 0;
    const double rc = ctx->eam.r_c;
    for (int r = 0; r < n_rep; ++r) {
        const ne_md_params& m = md[(size_t)r * md_stride];
        RepDev& R = ctx->rep_h[r];
        const int n = off[r + 1] - off[r];
        if (n < 2) return fail(ctx, NE_EINVAL, "every replica needs at least 2 atoms");
        const double skin = skin_override >= 0 ? skin_override : m.skin;
        if (!(skin >= 0)) return fail(ctx, NE_EINVAL, "skin must be >= 0");
        const double rl = rc + skin;
        // with the barostat the cells keep an edge >= r_c + skin down to a
        // 10 % linear contraction of the box (further is reported as NE_ERANGE)
        const double shrink = m.npt ? 0.9 : 1.0;
        for (int d = 0; d < 3; ++d) {
            R.L[d] = boxes[3 * r + d];
            if (geometry && !(R.L[d] > 2.0 * rl))
                return fail(ctx, NE_EINVAL, "box edge must exceed 2 (r_c + skin)");
            R.invL[d] = 1.0 / R.L[d];
            R.nc[d] = geometry ? (int)std::min(std::floor(shrink * R.L[d] / rl), 1024.0) : 0;
        }
        // cells of edge >= r_c + skin; fewer (larger) cells when the box is
        // sparse, so the cell count stays below 2n + 27
        while ((long long)R.nc[0] * R.nc[1] * R.nc[2] > 2ll * n + 27) {
            int d = R.nc[0] >= R.nc[1] && R.nc[0] >= R.nc[2] ? 0 : (R.nc[1] >= R.nc[2] ? 1 : 2);
            R.nc[d] -= 1;
        }
        if (R.nc[0] < 3 || R.nc[1] < 3 || R.nc[2] < 3) R.nc[0] = R.nc[1] = R.nc[2] = 0;
        R.k = m.k_spring;
        R.m = m.mass;
        if (!(m.mass > 0)) return fail(ctx, NE_EINVAL, "mass must be positive");
        const double gamma = m.damp > 0 ? 1.0 / m.damp : 0.0;
        R.c1 = std::exp(-gamma * m.dt);
        R.c2 = std::sqrt((1.0 - R.c1 * R.c1) * kB * m.T / m.mass);
        R.hdt_m = 0.5 * m.dt / m.mass;
        R.kT = kB * m.T;
        R.rlist2 = rl * rl;
        R.half_skin2 = (float)(0.25 * skin * skin);
        R.off = off[r];
        R.n = n;
        R.tile0 = (int)ctx->tile_rep_h.size();
        R.ntile = (n + NE_TILE - 1) / NE_TILE;
        for (int t = 0; t < R.ntile; ++t) ctx->tile_rep_h.push_back(r);
        R.cell_off = cells;
        cells += R.nc[0] * R.nc[1] * R.nc[2];
        R.dof = m.fix_cm ? 3 * n - 3 : 3 * n;
        R.seed = m.seed;
        R.replica = m.replica;
        if (m.replica >= (1u << 28)) return fail(ctx, NE_EINVAL, "replica id must be < 2^28");
        R.npt = m.npt;
        R.P0 = m.P0;
        R.mp = m.npt ? m.beta_T / m.tau_p : 0.0;
        npt_any |= m.npt;
        if (m.n_species >= 2) {
            ne_status sst = species_tables(ctx, m, n, R.c1, R, st);
            if (sst) return sst;
        } else if (m.n_species < 0 || m.n_species > NE_MAX_SPECIES) {
            return fail(ctx, NE_EINVAL, "n_species must be 0 .. NE_MAX_SPECIES");
        }
    }
    ctx->last_nrep = n_rep;
    ctx->boxes_from_runner = false;
    int species_all = 1;
    for (int r = 0; r < n_rep; ++r) species_all &= ctx->rep_h[r].nsp >= 2;
    const int n_tiles = (int)ctx->tile_rep_h.size();
    if (n_tiles > ctx->tiles_cap) return fail(ctx, NE_ENOMEM, "tile capacity exceeded");
    if (cells > ctx->cells_cap) return fail(ctx, NE_ENOMEM, "cell capacity exceeded");
    NE_CU(cudaMemcpyAsync(ctx->rep, ctx->rep_h.data(), sizeof(RepDev) * n_rep, cudaMemcpyHostToDevice, st));
    NE_CU(cudaMemcpyAsync(ctx->tile_rep, ctx->tile_rep_h.data(), sizeof(int) * n_tiles,
                          cudaMemcpyHostToDevice, st));
    NE_CU(cudaMemsetAsync(ctx->tile_done, 0, sizeof(unsigned) * n_rep, st));
    NE_CU(cudaMemsetAsync(ctx->flags, 0, sizeof(int) * n_rep, st));
    NE_CU(cudaMemsetAsync(ctx->status, 0, sizeof(int), st));
    NE_CU(cudaMemsetAsync(ctx->tot, 0, sizeof(double) * NTOT * n_rep, st));
    B = DevBatch{};
    B.n_rep = n_rep;
    B.n_tot = n_tot;
    B.n_tiles = n_tiles;
    B.tpa = ctx->tpa;
    B.rep = ctx->rep;
    B.tile_rep = ctx->tile_rep;
    B.x = a.x;
    B.v = a.v;
    B.x0 = a.x0;
    B.pos32 = ctx->pos32;
    B.posF = ctx->posF;
    B.pbuild = ctx->pbuild;
    B.f32 = ctx->f32;
    B.f64 = ctx->f64;
    B.dF64 = ctx->dF64;
    B.rho = a.rho;
    B.xi32 = ctx->xi32;
    B.xi64 = ctx->xi64;
    B.nbr = ctx->nbr;
    B.ncnt = ctx->ncnt;
    B.sl = ctx->sl;
    B.scnt = ctx->scnt;
    B.cellof = ctx->cellof;
    B.sorted = ctx->sorted;
    B.cstart = ctx->cstart;
    B.cfill = ctx->cfill;
    B.partA = ctx->partA;
    B.partB = ctx->partB;
    B.tot = ctx->tot;
    B.tile_done = ctx->tile_done;
    B.W = a.W;
    B.Wcum = a.Wcum;
    B.trace = a.trace;
    B.trace_stride = a.trace_stride > 0 ? a.trace_stride : 1;
    B.trace_rows = a.trace_rows;
    B.flags = ctx->flags;
    B.building = ctx->building;
    B.rebuilds = ctx->rebuilds;
    B.status = ctx->status;
    B.tab = ctx->tab;
    B.npt_any = npt_any;
    B.species_any = species_all;
    return NE_OK;
}

// Read the device status word back and map it to the ABI's codes.
ne_status finish(ne_ctx* ctx, cudaStream_t st)
{
    NE_CU(cudaGetLastError());
    // the status word lands in pinned host memory: the copy is a plain DMA
    NE_CU(cudaMemcpyAsync(ctx->status_host, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    NE_CU(cudaStreamSynchronize(st));
    const int bits = *ctx->status_host;
    ctx->last_bits = bits;
    if (bits & ST_ENAN) return fail(ctx, NE_ENAN, "non-finite position, velocity or energy");
    if (bits & ST_ERANGE) return fail(ctx, NE_ERANGE, "pair distance below 0.2 A, density >= rho_max, or an atom beyond the crystal runner's stencil range");
    if (bits & ST_ENEIGH) return fail(ctx, NE_ENEIGH, "neighbour-list capacity exceeded");
    if (bits & ST_ETIMEOUT) return fail(ctx, NE_ETIMEOUT, "bounded device wait gave up");
    if (bits & ST_EINVAL) return fail(ctx, NE_EINVAL, "crystal runner: shared-memory layout larger than the launch's allocation");
    ctx->msg = "ok";
    return NE_OK;
}

// Forces at the current x of every replica: list (re)build when flagged,
// pass 1, pass 2 (with the noise of step s when want_noise).
void force_eval(const DevBatch& B, const Sched& S, bool mixed, const long long* ctr, int j,
                int want_noise, int force_build, cudaStream_t st)
{
    ne::launch_nl_build(B, force_build, 0, st);
    ne::launch_density(B, mixed, ctr, j, st);
    ne::launch_force(B, S, mixed, ctr, j, want_noise, st);
}

// One fused step of the schedule (device step = *ctr + j).
// Optional parameter gradient along a run: after the force evaluation at
// x_k, gtheta += w[k - s_off] dU/dtheta(x_k) (the step's own list and rho).
struct GradAcc {
    double* gtheta;
    const double* w;
    float* bins;
    int nbb;
    long long s_off;
};

void grad_at(const DevBatch& B, bool mixed, const GradAcc* ga, const long long* ctr, int j, cudaStream_t st)
{
    if (ga) ne::launch_backward(B, mixed, 0.0, nullptr, ga->gtheta, ga->bins, ga->nbb, true, st, ga->w, ctr, j,
                                ga->s_off, false);
}

void one_step(const DevBatch& B, const Sched& S, bool mixed, const long long* ctr, int j, int first,
              cudaStream_t st, const GradAcc* ga = nullptr)
{
    force_eval(B, S, mixed, ctr, j, 1, 0, st);
    grad_at(B, mixed, ga, ctr, j, st);
    ne::launch_step(B, S, mixed, ctr, j, first ? 0 : 1, 1, st);
    if (B.npt_any) ne::launch_npt_box(B, S, ctr, j, st);
}

// Run steps [0, n_steps) of schedule S from the state held in B, then the
// closing half kick.  Chunks of G steps are captured once into a CUDA graph
// and replayed; the step index lives in device memory, so one graph serves
// every chunk.
ne_status run_steps(ne_ctx* ctx, const DevBatch& B, const Sched& S, bool mixed, long long s_begin,
                    long long n_steps, cudaStream_t st, double* msd_acc = nullptr,
                    long long msd_from = 0, int msd_stride = 0, const GradAcc* ga = nullptr)
{
    long long* ctr = ctx->step_ctr;
    NE_CU(cudaMemcpyAsync(ctr, &s_begin, sizeof(long long), cudaMemcpyHostToDevice, st));
    NE_CU(cudaStreamSynchronize(st));
    // list from the lattice sites (from the positions when a barostat may
    // have changed the box since the sites were made)
    ne::launch_nl_build(B, 1, B.npt_any ? 0 : 1, st);
    ne::launch_prep(B, S, mixed, ctr, st);
    long long s = 0;
    // first step: no closing kick
    if (n_steps > 0) {
        one_step(B, S, mixed, ctr, 0, 1, st, ga);
        ne::launch_advance(ctr, 1, st);
        s = 1;
        if (msd_acc && msd_stride > 0 && s > msd_from && (s - msd_from) % msd_stride == 0)
            ne::launch_msd_sample(B, msd_acc, st);
    }
    const int G = 32;
    const bool use_graph = !msd_acc && n_steps - s >= 4 * G;
    if (use_graph) {
        cudaGraph_t graph;
        cudaGraphExec_t exec;
        cudaStream_t cs;
        NE_CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaEvent_t ev;
        NE_CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        NE_CU(cudaEventRecord(ev, st));
        NE_CU(cudaStreamWaitEvent(cs, ev, 0));
        NE_CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        for (int j = 0; j < G; ++j) one_step(B, S, mixed, ctr, j, 0, cs, ga);
        ne::launch_advance(ctr, G, cs);
        cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        if (ce != cudaSuccess) {
            cudaStreamDestroy(cs);
            cudaEventDestroy(ev);
            return fail(ctx, NE_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        }
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            cudaStreamDestroy(cs);
            cudaEventDestroy(ev);
            return fail(ctx, NE_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        }
        const long long reps = (n_steps - s) / G;
        for (long long q = 0; q < reps; ++q) {
            ce = cudaGraphLaunch(exec, st);
            if (ce != cudaSuccess) break;
        }
        s += reps * G;
        cudaGraphExecDestroy(exec);
        cudaStreamDestroy(cs);
        cudaEventDestroy(ev);
        if (ce != cudaSuccess) return fail(ctx, NE_ECUDA, std::string("graph launch: ") + cudaGetErrorString(ce));
    }
    for (; s < n_steps; ++s) {
        one_step(B, S, mixed, ctr, 0, 0, st, ga);
        ne::launch_advance(ctr, 1, st);
        if (msd_acc && msd_stride > 0 && s + 1 > msd_from && (s + 1 - msd_from) % msd_stride == 0)
            ne::launch_msd_sample(B, msd_acc, st);
    }
    // closing half kick of the last step
    force_eval(B, S, mixed, ctr, 0, 0, 0, st);
    grad_at(B, mixed, ga, ctr, 0, st);
    ne::launch_step(B, S, mixed, ctr, 0, 1, 0, st);
    NE_CU(cudaGetLastError());
    return NE_OK;
}

// Per-kernel timing: the same steps launched one by one with CUDA events
// around each kernel on the launching stream.  kinds: 0 list build,
// 1 pass 1 (density), 2 pass 2 (forces), 3 fused step.
ne_status profile_steps(ne_ctx* ctx, const DevBatch& B, const Sched& S, bool mixed, long long s_begin,
                        long long n_steps, double* ms, long long* counts, cudaStream_t st)
{
    long long* ctr = ctx->step_ctr;
    NE_CU(cudaMemcpyAsync(ctr, &s_begin, sizeof(long long), cudaMemcpyHostToDevice, st));
    NE_CU(cudaStreamSynchronize(st));
    ne::launch_nl_build(B, 1, 1, st);
    ne::launch_prep(B, S, mixed, ctr, st);
    std::vector<cudaEvent_t> ev(2 * 4 * (size_t)n_steps);
    for (auto& e : ev) NE_CU(cudaEventCreate(&e));
    for (long long s = 0; s < n_steps; ++s) {
        cudaEvent_t* e = &ev[8 * s];
        NE_CU(cudaEventRecord(e[0], st));
        ne::launch_nl_build(B, 0, 0, st);
        NE_CU(cudaEventRecord(e[1], st));
        NE_CU(cudaEventRecord(e[2], st));
        ne::launch_density(B, mixed, ctr, 0, st);
        NE_CU(cudaEventRecord(e[3], st));
        NE_CU(cudaEventRecord(e[4], st));
        ne::launch_force(B, S, mixed, ctr, 0, 1, st);
        NE_CU(cudaEventRecord(e[5], st));
        NE_CU(cudaEventRecord(e[6], st));
        ne::launch_step(B, S, mixed, ctr, 0, s == 0 ? 0 : 1, 1, st);
        NE_CU(cudaEventRecord(e[7], st));
        ne::launch_advance(ctr, 1, st);
    }
    force_eval(B, S, mixed, ctr, 0, 0, 0, st);
    ne::launch_step(B, S, mixed, ctr, 0, 1, 0, st);
    NE_CU(cudaStreamSynchronize(st));
    for (int k = 0; k < 4; ++k) {
        ms[k] = 0.0;
        counts[k] = n_steps;
    }
    for (long long s = 0; s < n_steps; ++s)
        for (int k = 0; k < 4; ++k) {
            float t = 0.f;
            NE_CU(cudaEventElapsedTime(&t, ev[8 * s + 2 * k], ev[8 * s + 2 * k + 1]));
            ms[k] += t;
        }
    for (int k = 0; k < 4; ++k) ms[k] /= (double)(n_steps > 0 ? n_steps : 1);
    for (auto& e : ev) cudaEventDestroy(e);
    return NE_OK;
}

Sched make_sched(const ne_md_params& m)
{
    Sched S{};
    S.kind = SCHED_SWITCH;
    S.t_eq = m.t_eq;
    S.t_s = m.t_s;
    S.lambda_f = m.lambda_f;
    S.dt = m.dt;
    S.path = m.path;
    S.fn = m.lambda_fn;
    S.stream = m.path == NE_PATH_FL ? STREAM_FL : STREAM_RS;
    S.fix_cm = m.fix_cm;
    return S;
}

ne_status check_md(ne_ctx* ctx, const ne_md_params* m)
{
    if (!m) return fail(ctx, NE_EINVAL, "md params are NULL");
    if (!(m->dt > 0) || !(m->T > 0) || !(m->mass > 0)) return fail(ctx, NE_EINVAL, "dt, T and mass must be positive");
    if (m->path != NE_PATH_FL && m->path != NE_PATH_RS) return fail(ctx, NE_EINVAL, "unknown path");
    if (m->lambda_fn != 1 && m->lambda_fn != 2) return fail(ctx, NE_EINVAL, "lambda_fn must be 1 or 2");
    if (m->path == NE_PATH_RS && !(m->lambda_f > 0 && m->lambda_f < 1))
        return fail(ctx, NE_EINVAL, "lambda_f must lie in (0, 1)");
    if (m->prec != NE_FP64 && m->prec != NE_MIXED) return fail(ctx, NE_EINVAL, "unknown precision");
    if (m->npt < 0 || m->npt > 2) return fail(ctx, NE_EINVAL, "npt must be 0, 1 or 2");
    if (m->npt && m->path != NE_PATH_RS)
        return fail(ctx, NE_EINVAL, "the barostat runs on the reversible-scaling path (the Einstein crystal has no pressure)");
    if (m->npt && (!(m->beta_T > 0) || !(m->tau_p > 0) || !(m->P0 >= 0)))
        return fail(ctx, NE_EINVAL, "barostat: beta_T > 0, tau_p > 0 and P0 >= 0 required");
    return NE_OK;
}

}  // namespace

// =============================================================== C ABI
extern "C" {

ne_status ne_ctx_create(const ne_eam_params* eam, int max_atoms, int max_replicas, ne_ctx** out)
{
    if (out) *out = nullptr;
    if (!eam || !out || max_atoms < 2 || max_replicas < 1) return NE_EINVAL;
    if (eam->n_knots < 4 || !(eam->r_c > 0) || !(eam->rho_max > 0) || !(eam->r_s < eam->r_c))
        return NE_EINVAL;
    ne_ctx* ctx = new (std::nothrow) ne_ctx();
    if (!ctx) return NE_ENOMEM;
    ctx->eam = *eam;
    ctx->max_atoms = max_atoms;
    ctx->max_rep = max_replicas;
    ctx->tiles_cap = max_atoms / NE_TILE + max_replicas + 1;
    ctx->cells_cap = max_atoms + 64 * max_replicas;
    const size_t N = (size_t)max_atoms, R = (size_t)max_replicas, nk = (size_t)eam->n_knots;
    bool ok = true;
    auto A = [&](cudaError_t e) { ok = ok && e == cudaSuccess; };
    A(dalloc(&ctx->theta, 6 * nk));
    A(dalloc(&ctx->pf32, 2 * nk));
    A(dalloc(&ctx->pf64, 2 * nk));
    A(dalloc(&ctx->F32, nk));
    A(dalloc(&ctx->F64, nk));
    A(dalloc(&ctx->pos32, N));
    A(dalloc(&ctx->posF, N));
    A(dalloc(&ctx->pbuild, N));
    A(dalloc(&ctx->f32, N));
    A(dalloc(&ctx->f64, 3 * N));
    A(dalloc(&ctx->dF64, N));
    A(dalloc(&ctx->rho, N));
    A(dalloc(&ctx->xi64, 3 * N));
    A(dalloc(&ctx->xi32, 3 * N));
    A(dalloc(&ctx->nbr, N * NE_NMAX));
    A(dalloc(&ctx->ncnt, N));
    A(dalloc(&ctx->sl, N * NE_SMAX));
    A(dalloc(&ctx->scnt, N * 8));
    A(dalloc(&ctx->cellof, N));
    A(dalloc(&ctx->sorted, N));
    A(dalloc(&ctx->cstart, (size_t)ctx->cells_cap + R));
    A(dalloc(&ctx->cfill, (size_t)ctx->cells_cap));
    A(dalloc(&ctx->partA, (size_t)ctx->tiles_cap * NPA));
    A(dalloc(&ctx->partB, (size_t)ctx->tiles_cap * NPB));
    A(dalloc(&ctx->tot, R * NTOT));
    A(dalloc(&ctx->W, 2 * R));
    A(dalloc(&ctx->scratch, 4 * R + 16));
    A(dalloc(&ctx->tile_done, R));
    A(dalloc(&ctx->flags, R));
    A(dalloc(&ctx->building, R));
    A(dalloc(&ctx->status, 1 + R));  // the status word, then one per replica (crystal runner)
    if (ok) ctx->rep_status = ctx->status + 1;
    A(dalloc(&ctx->tile_rep, (size_t)ctx->tiles_cap));
    A(dalloc(&ctx->rep, R));
    A(dalloc(&ctx->step_ctr, 1));
    A(dalloc(&ctx->rebuilds, 1));
    A(dalloc(&ctx->xrep, R));
    A(dalloc(&ctx->work, 2));
    A(dalloc(&ctx->cr_boxes, 3 * R));
    A(cudaMallocHost((void**)&ctx->status_host, sizeof(int)));
    if (ok) ok = cudaMemset(ctx->work, 0, 2 * sizeof(unsigned long long)) == cudaSuccess;
    A(dalloc(&ctx->st_vec, R * 4 * NE_STENCIL_MAX));
    A(dalloc(&ctx->st_dist, R * 4 * NE_STENCIL_MAX));
    if (ok) ok = cudaMemset(ctx->rebuilds, 0, sizeof(unsigned long long)) == cudaSuccess;
    if (!ok) {
        ne_ctx_destroy(ctx);
        return NE_ENOMEM;
    }
    fill_tables(ctx);
    std::vector<double> th = make_theta(*eam);
    if (cudaMemcpy(ctx->theta, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        ne_ctx_destroy(ctx);
        return NE_ECUDA;
    }
    ne::launch_tables(ctx->theta, eam->n_knots, eam->r_c, eam->rho_max, ctx->pf32, ctx->pf64, ctx->F32,
                      ctx->F64, 0);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        ne_ctx_destroy(ctx);
        return NE_ECUDA;
    }
    ctx->msg = "ok";
    *out = ctx;
    return NE_OK;
}

ne_status ne_ctx_destroy(ne_ctx* ctx)
{
    if (!ctx) return NE_EINVAL;
    void* ptrs[] = {ctx->theta, ctx->pf32, ctx->pf64, ctx->F32, ctx->F64, ctx->pos32, ctx->posF,
                    ctx->pbuild, ctx->f32, ctx->f64, ctx->dF64, ctx->rho, ctx->xi64, ctx->xi32,
                    ctx->nbr, ctx->ncnt, ctx->sl, ctx->scnt, ctx->cellof, ctx->sorted, ctx->cstart,
                    ctx->cfill, ctx->partA, ctx->partB, ctx->tot, ctx->W, ctx->scratch,
                    ctx->tile_done, ctx->flags, ctx->building, ctx->status, ctx->tile_rep, ctx->rep, ctx->step_ctr, ctx->rebuilds, ctx->xrep, ctx->work, ctx->st_vec, ctx->st_dist, ctx->lam_tab,
                    ctx->bins};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (ctx->status_host) cudaFreeHost(ctx->status_host);
    for (int g = 0; g < 16; ++g)
        if (ctx->gst[g]) cudaStreamDestroy(ctx->gst[g]);
    for (int g = 0; g < 17; ++g)
        if (ctx->gev[g]) cudaEventDestroy(ctx->gev[g]);
    for (int g = 0; g < 2; ++g)
        if (ctx->ev_run[g]) cudaEventDestroy(ctx->ev_run[g]);
    void* bptrs[] = {ctx->bb.u4, ctx->bb.fp, ctx->bb.part, ctx->bb.vir, ctx->bb.bar, ctx->bb.abortf, ctx->cta_rep,
                     ctx->cr_boxes};
    for (void* p : bptrs)
        if (p) cudaFree(p);
    delete ctx;
    return NE_OK;
}

ne_status ne_ctx_clone(ne_ctx* src, int max_atoms, int max_replicas, ne_ctx** out)
{
    if (out) *out = nullptr;
    if (!src || !out) return NE_EINVAL;
    ne_ctx* c = nullptr;
    ne_status s = ne_ctx_create(&src->eam, max_atoms, max_replicas, &c);
    if (s) return s;
    c->tpa = src->tpa;
    c->cluster_c = src->cluster_c;
    s = ne_ctx_set_theta(c, src->theta, nullptr);
    if (!s && cudaDeviceSynchronize() != cudaSuccess) s = NE_ECUDA;
    if (s) {
        ne_ctx_destroy(c);
        return s;
    }
    *out = c;
    return NE_OK;
}

ne_status ne_ctx_set_theta(ne_ctx* ctx, const double* theta_dev, void* stream)
{
    if (!ctx || !theta_dev) return NE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int nk = ctx->eam.n_knots;
    NE_CU(cudaMemcpyAsync(ctx->theta, theta_dev, sizeof(double) * 6 * nk, cudaMemcpyDeviceToDevice, st));
    ne::launch_tables(ctx->theta, nk, ctx->eam.r_c, ctx->eam.rho_max, ctx->pf32, ctx->pf64, ctx->F32,
                      ctx->F64, st);
    NE_CU(cudaGetLastError());
    return NE_OK;
}

ne_status ne_ctx_get_theta(ne_ctx* ctx, double* theta_dev, void* stream)
{
    if (!ctx || !theta_dev) return NE_EINVAL;
    NE_CU(cudaMemcpyAsync(theta_dev, ctx->theta, sizeof(double) * 6 * ctx->eam.n_knots,
                          cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return NE_OK;
}

ne_status ne_ctx_set_tuning(ne_ctx* ctx, int tpa)
{
    if (!ctx) return NE_EINVAL;
    if (tpa != 1 && tpa != 2 && tpa != 4 && tpa != 8) return fail(ctx, NE_EINVAL, "threads_per_atom must be 1, 2, 4 or 8");
    ctx->tpa = tpa;
    return NE_OK;
}

ne_status ne_ctx_set_cluster_size(ne_ctx* ctx, int ctas)
{
    if (!ctx) return NE_EINVAL;
    if (ctas < 0 || ctas > 16) return fail(ctx, NE_EINVAL, "cluster size must be 0 (automatic) or 1..16");
    ctx->cluster_c = ctas;
    return NE_OK;
}

ne_status ne_ctx_set_runner(ne_ctx* ctx, int runner)
{
    if (!ctx) return NE_EINVAL;
    if (runner < 0 || runner > 2) return fail(ctx, NE_EINVAL, "runner must be 0 (automatic), 1 (cluster) or 2 (brick)");
    ctx->runner = runner;
    return NE_OK;
}

ne_status ne_ctx_boxes(ne_ctx* ctx, int n_rep, double* boxes_host)
{
    if (!ctx || !boxes_host || n_rep < 1) return NE_EINVAL;
    if (n_rep != ctx->last_nrep) return fail(ctx, NE_EINVAL, "replica count differs from the last run");
    if (ctx->boxes_from_runner) {
        if (cudaMemcpy(boxes_host, ctx->cr_boxes, sizeof(double) * 3 * (size_t)n_rep, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return fail(ctx, NE_ECUDA, "reading the boxes failed");
        return NE_OK;
    }
    std::vector<RepDev> r(n_rep);
    if (cudaMemcpy(r.data(), ctx->rep, sizeof(RepDev) * n_rep, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(ctx, NE_ECUDA, "reading the boxes failed");
    for (int q = 0; q < n_rep; ++q)
        for (int d = 0; d < 3; ++d) boxes_host[3 * q + d] = r[q].L[d];
    return NE_OK;
}

ne_status ne_ctx_replica_status(ne_ctx* ctx, int n_rep, int* out_host)
{
    if (!ctx || !out_host || n_rep < 1) return NE_EINVAL;
    if (n_rep != ctx->last_nrep_cr) return fail(ctx, NE_EINVAL, "replica count differs from the last crystal-runner call");
    std::vector<int> bits(n_rep);
    if (cudaMemcpy(bits.data(), ctx->rep_status, sizeof(int) * n_rep, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(ctx, NE_ECUDA, "reading the replica status failed");
    for (int r = 0; r < n_rep; ++r) {
        const int b = bits[r];
        out_host[r] = (b & ST_ENAN) ? NE_ENAN : (b & ST_ERANGE) ? NE_ERANGE : (b & ST_ENEIGH) ? NE_ENEIGH
                    : (b & ST_ETIMEOUT) ? NE_ETIMEOUT : NE_OK;
    }
    return NE_OK;
}

ne_status ne_ctx_counters(ne_ctx* ctx, long long* list_builds, long long* stencil_visits, long long* pairs,
                          long long* crystal_launches)
{
    if (!ctx) return NE_EINVAL;
    unsigned long long v[3] = {0, 0, 0};
    if (cudaMemcpy(&v[0], ctx->rebuilds, sizeof(v[0]), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&v[1], ctx->work, 2 * sizeof(v[0]), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(ctx, NE_ECUDA, "reading the counters failed");
    if (list_builds) *list_builds = (long long)v[0];
    if (stencil_visits) *stencil_visits = (long long)v[1];
    if (pairs) *pairs = (long long)v[2];
    if (crystal_launches) *crystal_launches = ctx->cr_launches;
    return NE_OK;
}

ne_status ne_ctx_crystal_plan(ne_ctx* ctx, int* runner, int* threads_per_atom, int* ctas, int* cluster_ctas)
{
    if (!ctx) return NE_EINVAL;
    const CrPlan& P = ctx->plan;
    if (!P.valid) return fail(ctx, NE_EINVAL, "no crystal-runner launch has been planned on this context");
    int r = 2, tpa = P.tpa, n = P.n_cta, cc = 0;
    if (!P.brick) {
        r = 1;
        tpa = ne::cluster_threads_per_atom();
        n = 0;
        for (const CrGroup& G : P.groups) {
            n += (G.e - G.b) * G.C;
            cc = std::max(cc, G.C);
        }
    }
    if (runner) *runner = r;
    if (threads_per_atom) *threads_per_atom = tpa;
    if (ctas) *ctas = n;
    if (cluster_ctas) *cluster_ctas = cc;
    return NE_OK;
}

ne_status ne_ctx_last_run_ms(ne_ctx* ctx, double* ms_host)
{
    if (!ctx || !ms_host) return NE_EINVAL;
    if (!ctx->run_timed) return fail(ctx, NE_EINVAL, "no crystal-runner call has run on this context");
    float ms = 0.f;
    if (cudaEventSynchronize(ctx->ev_run[1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, ctx->ev_run[0], ctx->ev_run[1]) != cudaSuccess)
        return fail(ctx, NE_ECUDA, "reading the run's events failed");
    *ms_host = (double)ms;
    return NE_OK;
}

ne_status ne_last_error(ne_ctx* ctx, int* device_status, char* msg, int msg_len)
{
    if (!ctx) return NE_EINVAL;
    if (device_status) *device_status = ctx->last_bits;
    if (msg && msg_len > 0) {
        std::strncpy(msg, ctx->msg.c_str(), (size_t)msg_len - 1);
        msg[msg_len - 1] = 0;
    }
    return NE_OK;
}

// Cell edges and basis (fractions of the edges) of a lattice; hcp is the
// orthohexagonal cell (a, sqrt(3) a, c).
static bool lattice_cell(ne_lattice lattice, double a, double c_over_a, double cell[3], int* nb,
                         const double (**basis)[3])
{
    static const double bcc[2][3] = {{0, 0, 0}, {0.5, 0.5, 0.5}};
    static const double fcc[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
    static const double hcp[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0, 1.0 / 3.0, 0.5}, {0.5, 5.0 / 6.0, 0.5}};
    cell[0] = cell[1] = cell[2] = a;
    if (lattice == NE_BCC) {
        *nb = 2;
        *basis = bcc;
    } else if (lattice == NE_FCC) {
        *nb = 4;
        *basis = fcc;
    } else if (lattice == NE_HCP) {
        if (!(c_over_a > 0)) return false;
        *nb = 4;
        *basis = hcp;
        cell[1] = std::sqrt(3.0) * a;
        cell[2] = c_over_a * a;
    } else {
        return false;
    }
    return true;
}

ne_status ne_create_crystal_ca(ne_lattice lattice, double a, double c_over_a, int nx, int ny, int nz,
                               double* x0_host, double box[3], int* n_out)
{
    if (!(a > 0) || nx < 1 || ny < 1 || nz < 1) return NE_EINVAL;
    double cell[3];
    int nb;
    const double(*basis)[3];
    if (!lattice_cell(lattice, a, lattice == NE_HCP ? c_over_a : 1.0, cell, &nb, &basis)) return NE_EINVAL;
    long long n = (long long)nb * nx * ny * nz;
    if (n > (1ll << 30)) return NE_EINVAL;
    if (x0_host) {
        long long i = 0;
        for (int ix = 0; ix < nx; ++ix)
            for (int iy = 0; iy < ny; ++iy)
                for (int iz = 0; iz < nz; ++iz)
                    for (int b = 0; b < nb; ++b, ++i) {
                        x0_host[3 * i] = cell[0] * (ix + basis[b][0]);
                        x0_host[3 * i + 1] = cell[1] * (iy + basis[b][1]);
                        x0_host[3 * i + 2] = cell[2] * (iz + basis[b][2]);
                    }
    }
    if (box) {
        box[0] = cell[0] * nx;
        box[1] = cell[1] * ny;
        box[2] = cell[2] * nz;
    }
    if (n_out) *n_out = (int)n;
    return NE_OK;
}

ne_status ne_create_crystal(ne_lattice lattice, double a, int nx, int ny, int nz, double* x0_host,
                            double box[3], int* n_out)
{
    return ne_create_crystal_ca(lattice, a, std::sqrt(8.0 / 3.0), nx, ny, nz, x0_host, box, n_out);
}

ne_status ne_eam_energy_forces(ne_ctx* ctx, ne_precision prec, const double* x_dev, int n,
                               const double box[3], double* f_dev, double* e_dev, double* rho_dev,
                               void* stream)
{
    if (!ctx || !x_dev || !box || n < 2 || (!f_dev && !e_dev && !rho_dev)) return NE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    ne_md_params m{};
    m.dt = 1e-3;
    m.T = 1.0;
    m.mass = 1.0;
    m.prec = prec;
    int off[2] = {0, n};
    RunArgs a{};
    a.x = const_cast<double*>(x_dev);
    a.rho = rho_dev;
    DevBatch B;
    ne_status s = setup_batch(ctx, 1, off, box, &m, 0, 0.0, B, a, st);
    if (s) return s;
    const bool mixed = prec == NE_MIXED;
    Sched S{};
    S.kind = SCHED_FIXED;
    ne::launch_nl_build(B, 1, 0, st);
    if (mixed) ne::launch_wrap32(B, st);
    ne::launch_density(B, mixed, ctx->step_ctr, 0, st);
    ne::launch_force(B, S, mixed, ctx->step_ctr, 0, 0, st);
    ne::launch_export(B, mixed, f_dev, e_dev, st);
    return finish(ctx, st);
}

ne_status ne_eam_virial(ne_ctx* ctx, const double* x_dev, int n, const double box[3], double* w_dev,
                        void* stream)
{
    if (!ctx || !x_dev || !box || n < 2 || !w_dev) return NE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    ne_md_params m{};
    m.dt = 1e-3;
    m.T = 1.0;
    m.mass = 1.0;
    m.prec = NE_FP64;
    int off[2] = {0, n};
    RunArgs a{};
    a.x = const_cast<double*>(x_dev);
    DevBatch B;
    ne_status s = setup_batch(ctx, 1, off, box, &m, 0, 0.0, B, a, st);
    if (s) return s;
    ne::launch_nl_build(B, 1, 0, st);
    ne::launch_density(B, false, ctx->step_ctr, 0, st);
    ne::launch_virial(B, w_dev, st);
    return finish(ctx, st);
}

ne_status ne_spring_forces(const double* x_dev, const double* x0_dev, int n, double k, double* f_dev,
                           double* e_dev, void* stream)
{
    if (!x_dev || !x0_dev || n < 1 || (!f_dev && !e_dev)) return NE_EINVAL;
    ne::launch_spring(x_dev, x0_dev, n, k, f_dev, e_dev, nullptr, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? NE_OK : NE_ECUDA;
}

static ne_status backward_impl(ne_ctx* ctx, ne_precision prec, const double* x_dev, int n, const double box[3],
                               double gE, double* gx_dev, double* gtheta_dev, bool accumulate, void* stream)
{
    if (!ctx || !x_dev || !box || n < 2 || !gtheta_dev) return NE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    ne_md_params m{};
    m.dt = 1e-3;
    m.T = 1.0;
    m.mass = 1.0;
    int off[2] = {0, n};
    RunArgs a{};
    a.x = const_cast<double*>(x_dev);
    a.rho = ctx->rho;
    DevBatch B;
    ne_status s = setup_batch(ctx, 1, off, box, &m, 0, 0.0, B, a, st);
    if (s) return s;
    const bool mixed = prec == NE_MIXED;
    Sched S{};
    S.kind = SCHED_FIXED;
    ne::launch_nl_build(B, 1, 0, st);
    if (mixed) ne::launch_wrap32(B, st);
    ne::launch_density(B, mixed, ctx->step_ctr, 0, st);
    ne::launch_force(B, S, mixed, ctx->step_ctr, 0, 0, st);
    if (gx_dev) ne::launch_export(B, mixed, gx_dev, nullptr, st);
    if (mixed && !ne::backward_fits(ctx->eam.n_knots))
        return fail(ctx, NE_EINVAL, "mixed backward: n_knots too large for one block's shared-memory bins");
    int nbb = ne::backward_bin_blocks(B);
    if (mixed && nbb > ctx->bins_blocks) {
        if (ctx->bins) cudaFree(ctx->bins);
        ctx->bins = nullptr;
        ctx->bins_blocks = 0;
        NE_CU(cudaMalloc((void**)&ctx->bins, ne::backward_bins_bytes(ctx->eam.n_knots, nbb)));
        ctx->bins_blocks = nbb;
    }
    ne::launch_backward(B, mixed, gE, gx_dev, gtheta_dev, ctx->bins, nbb, accumulate, st);
    if (gx_dev) ne::launch_scale(gx_dev, 3 * n, -gE, st);  // dU/dx = -F times gE
    return finish(ctx, st);
}

ne_status ne_eam_backward(ne_ctx* ctx, ne_precision prec, const double* x_dev, int n, const double box[3],
                          double gE, double* gx_dev, double* gtheta_dev, void* stream)
{
    return backward_impl(ctx, prec, x_dev, n, box, gE, gx_dev, gtheta_dev, false, stream);
}

ne_status ne_eam_backward_acc(ne_ctx* ctx, ne_precision prec, const double* x_dev, int n, const double box[3],
                              double gE, double* gtheta_acc_dev, void* stream)
{
    return backward_impl(ctx, prec, x_dev, n, box, gE, nullptr, gtheta_acc_dev, true, stream);
}

ne_status ne_noise(unsigned long long seed, unsigned replica, int noise_stream, long long step, int n,
                   ne_precision prec, double* z_dev, void* stream)
{
    if (!z_dev || n < 1 || noise_stream < 0 || noise_stream > 15 || step < 0 || replica >= (1u << 28))
        return NE_EINVAL;
    ne::launch_noise(seed, replica, noise_stream, step, n, prec == NE_MIXED, z_dev, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? NE_OK : NE_ECUDA;
}

ne_status ne_init_velocities(ne_ctx* ctx, const ne_md_params* md, int n, double* v_dev, void* stream)
{
    if (!ctx || !v_dev || n < 2) return NE_EINVAL;
    ne_status s = check_md(ctx, md);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    int off[2] = {0, n};
    double box[3] = {1.0, 1.0, 1.0};
    RunArgs a{};
    a.v = v_dev;
    DevBatch B;
    s = setup_batch(ctx, 1, off, box, md, 0, 0.0, B, a, st, false);
    if (s) return s;
    ne::launch_init_velocities(B, md->fix_cm, st);
    return finish(ctx, st);
}

ne_status ne_langevin_step(ne_ctx* ctx, const ne_md_params* md, double* x_dev, double* v_dev,
                           const double* x0_dev, int n, const double box[3], long long step,
                           double lambda_k, double lambda_k1, double* W_dev, void* stream)
{
    if (!ctx || !x_dev || !v_dev || !x0_dev || !box || n < 2 || step < 0) return NE_EINVAL;
    ne_status s = check_md(ctx, md);
    if (s) return s;
    if (md->npt) return fail(ctx, NE_EINVAL, "the barostat runs in the switching runs (ne_switch_run_segment, ne_rs_run)");
    cudaStream_t st = (cudaStream_t)stream;
    int off[2] = {0, n};
    RunArgs a{};
    a.x = x_dev;
    a.v = v_dev;
    a.x0 = x0_dev;
    a.W = W_dev ? W_dev : ctx->W;
    if (!W_dev) NE_CU(cudaMemsetAsync(ctx->W, 0, sizeof(double), st));
    DevBatch B;
    s = setup_batch(ctx, 1, off, box, md, 0, -1.0, B, a, st);
    if (s) return s;
    Sched S = make_sched(*md);
    S.kind = SCHED_FIXED;
    S.lam_a = lambda_k;
    S.lam_b = lambda_k1;
    S.s0 = step;
    S.stream = STREAM_STEP;
    s = run_steps(ctx, B, S, md->prec == NE_MIXED, step, 1, st);
    if (s) return s;
    return finish(ctx, st);
}

ne_status ne_switch_run_batched(ne_ctx* ctx, const ne_md_params* md, int n_rep, const int* offsets_host,
                                double* x_dev, double* v_dev, const double* x0_dev, const double* boxes_host,
                                double* W_fwd_dev, double* W_bwd_dev, void* stream);

static ne_status check_batch(ne_ctx* ctx, const ne_md_params* md, int n_rep, const int* off)
{
    for (int r = 0; r < n_rep; ++r) {
        ne_status s = check_md(ctx, &md[r]);
        if (s) return s;
        const ne_md_params &a = md[0], &b = md[r];
        if (a.dt != b.dt || a.damp != b.damp || a.lambda_fn != b.lambda_fn || a.path != b.path ||
            a.lambda_f != b.lambda_f || a.t_eq != b.t_eq || a.t_s != b.t_s || a.fix_cm != b.fix_cm ||
            a.prec != b.prec)
            return fail(ctx, NE_EINVAL, "replicas must share dt, damp, schedule, path, fix_cm and precision");
        if (off[r + 1] <= off[r]) return fail(ctx, NE_EINVAL, "offsets must increase");
    }
    if (md[0].t_s < 1 || md[0].t_eq < 0) return fail(ctx, NE_EINVAL, "t_s >= 1 and t_eq >= 0 required");
    return NE_OK;
}

// Steps [s_begin, s_begin + n_steps) of the four-phase schedule for n_rep
// replicas; W [n_rep][2] accumulates (forward, backward) work in place.
static ne_status segment_impl(ne_ctx* ctx, const ne_md_params* md, int n_rep, const int* off, double* x,
                              double* v, const double* x0, const double* boxes, double* W, double* wcum,
                              double* trace, int trace_stride, long long s_begin, long long n_steps,
                              cudaStream_t st, const double* gw = nullptr, double* gtheta = nullptr)
{
    const long long S_total = 2 * md[0].t_eq + 2 * md[0].t_s;
    if (s_begin < 0 || n_steps < 0 || s_begin + n_steps > S_total)
        return fail(ctx, NE_EINVAL, "step range outside the schedule");
    RunArgs a{};
    a.x = x;
    a.v = v;
    a.x0 = x0;
    a.W = W;
    a.Wcum = wcum;
    a.trace = trace;
    a.trace_stride = trace_stride;
    a.trace_rows = trace ? (int)((S_total - 1) / (trace_stride > 0 ? trace_stride : 1) + 1) : 0;
    a.rho = gtheta ? ctx->rho : nullptr;  // the backward pass reads rho (FP64) of each step
    DevBatch B;
    ne_status s = setup_batch(ctx, n_rep, off, boxes, md, 1, -1.0, B, a, st);
    if (s) return s;
    Sched S = make_sched(md[0]);
    if (n_steps == 0) return finish(ctx, st);
    const bool mixed = md[0].prec == NE_MIXED;
    GradAcc ga{gtheta, gw, nullptr, 0, s_begin};
    if (gtheta) {
        if (mixed && !ne::backward_fits(ctx->eam.n_knots))
            return fail(ctx, NE_EINVAL, "mixed backward: n_knots too large for one block's shared-memory bins");
        ga.nbb = ne::backward_bin_blocks(B);
        if (mixed && ga.nbb > ctx->bins_blocks) {
            if (ctx->bins) cudaFree(ctx->bins);
            ctx->bins = nullptr;
            ctx->bins_blocks = 0;
            NE_CU(cudaMalloc((void**)&ctx->bins, ne::backward_bins_bytes(ctx->eam.n_knots, ga.nbb)));
            ctx->bins_blocks = ga.nbb;
        }
        ga.bins = ctx->bins;
        // the backward kernel's shared-memory attribute, once, outside any capture
        if (mixed) NE_CU(ne::prepare_backward(B));
    }
    s = run_steps(ctx, B, S, mixed, s_begin, n_steps, st, nullptr, 0, 0, gtheta ? &ga : nullptr);
    if (s) return s;
    return finish(ctx, st);
}

static ne_status switch_run_impl(ne_ctx* ctx, const ne_md_params* md, int n_rep, const int* off,
                                 double* x, double* v, const double* x0, const double* boxes,
                                 double* W_fwd, double* W_bwd, double* Wcum_f, double* Wcum_b,
                                 double* trace, int trace_stride, cudaStream_t st)
{
    if (!ctx || !md || !off || !x || !v || !x0 || !boxes || n_rep < 1) return NE_EINVAL;
    if (n_rep > ctx->max_rep) return fail(ctx, NE_ENOMEM, "replica count exceeds the context");
    ne_status s = check_batch(ctx, md, n_rep, off);
    if (s) return s;
    const long long S_total = 2 * md[0].t_eq + 2 * md[0].t_s;
    double* wcum = nullptr;
    const size_t ncum = (size_t)(md[0].t_s + 1);
    if (Wcum_f || Wcum_b) {
        if (n_rep != 1) return fail(ctx, NE_EINVAL, "cumulative work is recorded for single runs");
        NE_CU(cudaMalloc((void**)&wcum, sizeof(double) * 2 * ncum));
        NE_CU(cudaMemsetAsync(wcum, 0, sizeof(double) * 2 * ncum, st));
    }
    NE_CU(cudaMemsetAsync(ctx->W, 0, sizeof(double) * 2 * n_rep, st));
    s = segment_impl(ctx, md, n_rep, off, x, v, x0, boxes, ctx->W, wcum, trace, trace_stride, 0, S_total, st);
    if (!s) {
        // W layout [n_rep][2] -> caller's W_fwd[n_rep], W_bwd[n_rep]
        if (W_fwd) cudaMemcpy2DAsync(W_fwd, sizeof(double), ctx->W, 2 * sizeof(double), sizeof(double), n_rep,
                                     cudaMemcpyDeviceToDevice, st);
        if (W_bwd) cudaMemcpy2DAsync(W_bwd, sizeof(double), ctx->W + 1, 2 * sizeof(double), sizeof(double), n_rep,
                                     cudaMemcpyDeviceToDevice, st);
        if (Wcum_f) cudaMemcpyAsync(Wcum_f, wcum, sizeof(double) * ncum, cudaMemcpyDeviceToDevice, st);
        if (Wcum_b) cudaMemcpyAsync(Wcum_b, wcum + ncum, sizeof(double) * ncum, cudaMemcpyDeviceToDevice, st);
        s = finish(ctx, st);
    }
    if (wcum) {
        cudaStreamSynchronize(st);
        cudaFree(wcum);
    }
    return s;
}

ne_status ne_switch_run_segment_grad(ne_ctx* ctx, const ne_md_params* md, int n_rep, const int* offsets_host,
                                     double* x_dev, double* v_dev, const double* x0_dev, const double* boxes_host,
                                     double* W_dev, long long step_begin, long long n_steps, const double* w_dev,
                                     double* gtheta_dev, void* stream)
{
    if (!ctx || !md || !offsets_host || !x_dev || !v_dev || !x0_dev || !boxes_host || !W_dev || n_rep < 1 ||
        !w_dev || !gtheta_dev)
        return NE_EINVAL;
    if (n_rep > ctx->max_rep) return fail(ctx, NE_ENOMEM, "replica count exceeds the context");
    ne_status s = check_batch(ctx, md, n_rep, offsets_host);
    if (s) return s;
    return segment_impl(ctx, md, n_rep, offsets_host, x_dev, v_dev, x0_dev, boxes_host, W_dev, nullptr, nullptr,
                        0, step_begin, n_steps, (cudaStream_t)stream, w_dev, gtheta_dev);
}

ne_status ne_switch_run_segment_cum(ne_ctx* ctx, const ne_md_params* md, int n_rep, const int* offsets_host,
                                    double* x_dev, double* v_dev, const double* x0_dev, const double* boxes_host,
                                    double* W_dev, double* Wcum_dev, long long step_begin, long long n_steps,
                                    void* stream)
{
    if (!ctx || !md || !offsets_host || !x_dev || !v_dev || !x0_dev || !boxes_host || !W_dev || !Wcum_dev ||
        n_rep < 1)
        return NE_EINVAL;
    if (n_rep > ctx->max_rep) return fail(ctx, NE_ENOMEM, "replica count exceeds the context");
    ne_status s = check_batch(ctx, md, n_rep, offsets_host);
    if (s) return s;
    return segment_impl(ctx, md, n_rep, offsets_host, x_dev, v_dev, x0_dev, boxes_host, W_dev, Wcum_dev, nullptr,
                        0, step_begin, n_steps, (cudaStream_t)stream);
}

ne_status ne_switch_run_segment(ne_ctx* ctx, const ne_md_params* md, int n_rep, const int* offsets_host,
                                double* x_dev, double* v_dev, const double* x0_dev, const double* boxes_host,
                                double* W_dev, long long step_begin, long long n_steps, void* stream)
{
    if (!ctx || !md || !offsets_host || !x_dev || !v_dev || !x0_dev || !boxes_host || !W_dev || n_rep < 1)
        return NE_EINVAL;
    if (n_rep > ctx->max_rep) return fail(ctx, NE_ENOMEM, "replica count exceeds the context");
    ne_status s = check_batch(ctx, md, n_rep, offsets_host);
    if (s) return s;
    return segment_impl(ctx, md, n_rep, offsets_host, x_dev, v_dev, x0_dev, boxes_host, W_dev, nullptr, nullptr,
                        0, step_begin, n_steps, (cudaStream_t)stream);
}

ne_status ne_switch_run(ne_ctx* ctx, const ne_md_params* md, double* x_dev, double* v_dev,
                        const double* x0_dev, int n, const double box[3], double* W_fwd_dev,
                        double* W_bwd_dev, double* Wcum_fwd_dev, double* Wcum_bwd_dev, double* trace_dev,
                        int trace_stride, void* stream)
{
    if (n < 2 || !box) return NE_EINVAL;
    int off[2] = {0, n};
    return switch_run_impl(ctx, md, 1, off, x_dev, v_dev, x0_dev, box, W_fwd_dev, W_bwd_dev, Wcum_fwd_dev,
                           Wcum_bwd_dev, trace_dev, trace_stride, (cudaStream_t)stream);
}

ne_status ne_rs_run(ne_ctx* ctx, const ne_md_params* md, double lambda_f, double* x_dev, double* v_dev,
                    const double* x0_dev, int n, const double box[3], double* Wcum_fwd_dev,
                    double* Wcum_bwd_dev, void* stream)
{
    if (!md) return NE_EINVAL;
    ne_md_params m = *md;
    m.path = NE_PATH_RS;
    m.lambda_f = lambda_f;
    if (n < 2 || !box) return NE_EINVAL;
    int off[2] = {0, n};
    return switch_run_impl(ctx, &m, 1, off, x_dev, v_dev, x0_dev, box, nullptr, nullptr, Wcum_fwd_dev,
                           Wcum_bwd_dev, nullptr, 0, (cudaStream_t)stream);
}

ne_status ne_switch_run_batched(ne_ctx* ctx, const ne_md_params* md, int n_rep, const int* offsets_host,
                                double* x_dev, double* v_dev, const double* x0_dev, const double* boxes_host,
                                double* W_fwd_dev, double* W_bwd_dev, void* stream)
{
    return switch_run_impl(ctx, md, n_rep, offsets_host, x_dev, v_dev, x0_dev, boxes_host, W_fwd_dev,
                           W_bwd_dev, nullptr, nullptr, nullptr, 0, (cudaStream_t)stream);
}

// the packed neighbour code of a stencil entry, carried in the .w of its
// lattice vector as the float with the same bits
static float code_bits(int code)
{
    float f;
    std::memcpy(&f, &code, sizeof f);
    return f;
}

static ne_status crystal_segment_impl(ne_ctx* ctx, const ne_md_params* md, const ne_crystal* cr, int n_rep,
                                      double* x_dev, double* v_dev, double* W_dev, double* Wcum_dev,
                                      long long step_begin, long long n_steps, void* stream);

ne_status ne_crystal_run_segment(ne_ctx* ctx, const ne_md_params* md, const ne_crystal* cr, int n_rep,
                                 double* x_dev, double* v_dev, double* W_dev, long long step_begin,
                                 long long n_steps, void* stream)
{
    return crystal_segment_impl(ctx, md, cr, n_rep, x_dev, v_dev, W_dev, nullptr, step_begin, n_steps, stream);
}

ne_status ne_crystal_run_segment_cum(ne_ctx* ctx, const ne_md_params* md, const ne_crystal* cr, int n_rep,
                                     double* x_dev, double* v_dev, double* W_dev, double* Wcum_dev,
                                     long long step_begin, long long n_steps, void* stream)
{
    if (!Wcum_dev) return NE_EINVAL;
    return crystal_segment_impl(ctx, md, cr, n_rep, x_dev, v_dev, W_dev, Wcum_dev, step_begin, n_steps, stream);
}

// Key of a crystal-runner launch plan: everything the plan is built from
// (crystals, the per-replica parameters that enter XRep, the fixed cluster
// size), field by field so that struct padding never enters the comparison.
static std::vector<double> plan_key(ne_ctx* ctx, const ne_md_params* md, const ne_crystal* cr, int n_rep)
{
    std::vector<double> k;
    k.reserve(3 + 19 * (size_t)n_rep);
    k.push_back((double)n_rep);
    k.push_back((double)ctx->cluster_c);
    k.push_back((double)ctx->runner);
    for (int r = 0; r < n_rep; ++r) {
        const double rec[] = {(double)cr[r].lattice, cr[r].a, cr[r].c_over_a, (double)cr[r].nx, (double)cr[r].ny,
                              (double)cr[r].nz, md[r].k_spring, md[r].mass, md[r].dt, md[r].damp, md[r].T,
                              (double)(md[r].seed & 0xffffffffull), (double)(md[r].seed >> 32), (double)md[r].replica,
                              (double)md[r].npt, md[r].P0, md[r].beta_T, md[r].tau_p, (double)md[r].fix_cm};
        k.insert(k.end(), rec, rec + sizeof rec / sizeof rec[0]);
    }
    return k;
}

static bool same_sched(const Sched& a, const Sched& b)
{
    return a.t_eq == b.t_eq && a.t_s == b.t_s && a.lambda_f == b.lambda_f && a.lam_a == b.lam_a &&
           a.lam_b == b.lam_b && a.s0 == b.s0 && a.dt == b.dt && a.kind == b.kind && a.path == b.path &&
           a.fn == b.fn && a.stream == b.stream && a.fix_cm == b.fix_cm;
}

// Build the launch plan of a batch (stencils, replica table, cluster size,
// size classes and their shared memory) and upload its device part.  Runs
// on a call whose key differs from the cached plan's; later calls with the
// same batch launch at once.
static ne_status build_plan(ne_ctx* ctx, const ne_md_params* md, const ne_crystal* cr, int n_rep, cudaStream_t st)
{
    CrPlan& P = ctx->plan;
    P.valid = false;
    std::vector<int> off(n_rep + 1, 0);
    for (int r = 0; r < n_rep; ++r) {
        double cell[3];
        int nb;
        const double(*basis)[3];
        const double ca = cr[r].c_over_a > 0 ? cr[r].c_over_a : std::sqrt(8.0 / 3.0);
        if (!lattice_cell(cr[r].lattice, cr[r].a, ca, cell, &nb, &basis) || !(cr[r].a > 0) || cr[r].nx < 3 ||
            cr[r].ny < 3 || cr[r].nz < 3 || cr[r].c_over_a < 0)
            return fail(ctx, NE_EINVAL, "crystal: bcc/fcc/hcp, a > 0, c/a >= 0 and at least 3 cells per axis");
        const long long nn = (long long)nb * cr[r].nx * cr[r].ny * cr[r].nz;
        if (nn > (1 << 24)) return fail(ctx, NE_EINVAL, "crystal: too many atoms");
        off[r + 1] = off[r] + (int)nn;
    }
    if (off[n_rep] > ctx->max_atoms) return fail(ctx, NE_ENOMEM, "atom count exceeds the context");
    // the cluster runner holds up to 4096 atoms a replica; larger replicas,
    // or every batch when the context says so, go to the brick runner
    bool brick = ctx->runner == 2;
    for (int r = 0; r < n_rep; ++r) brick = brick || off[r + 1] - off[r] > 4096;
    if (brick && ctx->runner == 1)
        return fail(ctx, NE_EINVAL, "cluster runner: at most 4096 atoms per replica (the runner setting excludes the brick runner)");
    const double rc = ctx->eam.r_c;
    std::vector<XRep> xr(n_rep);
    std::vector<float4>& sv = P.sv;  // (lattice vector, neighbour code as float bits)
    std::vector<float>& sd = P.sd;   // |lattice vector|
    sv.clear();
    sd.clear();
    for (int r = 0; r < n_rep; ++r) {
        const ne_md_params& m = md[r];
        XRep& X = xr[r];
        X = XRep{};
        const double(*basis)[3];
        lattice_cell(cr[r].lattice, cr[r].a, cr[r].c_over_a > 0 ? cr[r].c_over_a : std::sqrt(8.0 / 3.0), X.cell,
                     &X.nb, &basis);
        for (int b = 0; b < X.nb; ++b)
            for (int d = 0; d < 3; ++d) X.basis[b][d] = basis[b][d];
        X.nx = cr[r].nx;
        X.ny = cr[r].ny;
        X.nz = cr[r].nz;
        X.n = off[r + 1] - off[r];
        X.off = off[r];
        X.k = m.k_spring;
        X.kf = (float)m.k_spring;
        X.mf = (float)m.mass;
        X.hdt_mf = (float)(0.5 * m.dt / m.mass);
        const double gamma = m.damp > 0 ? 1.0 / m.damp : 0.0;
        const double c1 = std::exp(-gamma * m.dt);
        X.c1f = (float)c1;
        X.c2f = (float)std::sqrt((1.0 - c1 * c1) * kB * m.T / m.mass);
        X.seed = m.seed;
        X.replica = m.replica;
        if (m.replica >= (1u << 28)) return fail(ctx, NE_EINVAL, "replica id must be < 2^28");
        X.npt = m.npt;
        X.dof = m.fix_cm ? 3 * X.n - 3 : 3 * X.n;
        X.P0 = m.P0;
        X.mp = m.npt ? m.beta_T / m.tau_p : 0.0;
        X.kT = kB * m.T;
        X.box0[0] = X.cell[0] * X.nx;
        X.box0[1] = X.cell[1] * X.ny;
        X.box0[2] = X.cell[2] * X.nz;
        if (m.n_species >= 2) {
            // one spring and mass per species (Sec. V): the tables of the
            // multi-kernel path in FP32, the species checked on the host
            RepDev R{};
            ne_status sst = species_tables(ctx, m, X.n, c1, R, st);
            if (sst) return sst;
            X.nsp = R.nsp;
            X.sp = R.sp;
            X.invM = (float)(1.0 / R.M);
            for (int q = 0; q < R.nsp; ++q) {
                X.kfs[q] = (float)R.ks[q];
                X.hdts[q] = (float)R.hdts[q];
                X.c2fs[q] = (float)R.c2s[q];
                X.mfs[q] = (float)R.ms[q];
            }
        } else if (m.n_species < 0 || m.n_species > NE_MAX_SPECIES) {
            return fail(ctx, NE_EINVAL, "n_species must be 0 .. NE_MAX_SPECIES");
        }
        // stencil: sites within r_c + 2D of each basis site, sorted by distance,
        // D = 2 A.  In a small box r_c + 2D can pass L/2 and the stencil then
        // holds two periodic images of some sites; two images are L > 2 r_c
        // apart, so at most one of them lies within r_c and every pair inside
        // the cutoff is still counted exactly once.
        const double Lmin = std::min(X.cell[0] * X.nx, std::min(X.cell[1] * X.ny, X.cell[2] * X.nz));
        if (0.5 * Lmin - rc < 0.6) return fail(ctx, NE_EINVAL, "box too small for the crystal runner (needs L/2 > r_c + 0.6 A)");
        const double D = 2.0;
        X.D = (float)D;
        const double Rst = rc + 2.0 * D;
        const int M = (int)std::ceil(Rst / std::min(X.cell[0], std::min(X.cell[1], X.cell[2]))) + 1;
        // neighbour code of a stencil entry (dx, dy, dz, b2): bits 0-15 the
        // offset (dx + M) * (ny + 2M) + dy + M into the xy table of wrapped
        // cells, bits 16-31 b2 * (nz + 2M) + dz + M into the z table, whose
        // entries also carry the start of basis site b2 in the basis-major
        // copy of the replica
        const int LY = X.ny + 2 * M, LZ = X.nz + 2 * M;
        if ((X.nx + 2 * M) * LY >= (1 << 16) || X.nb * LZ >= (1 << 16))
            return fail(ctx, NE_EINVAL, "crystal runner: box shape outside the stencil code range");
        // a replica with the same lattice, cell counts and margin as an
        // earlier one of the batch shares its stencil
        int same = -1;
        for (int q = 0; q < r && same < 0; ++q)
            if (cr[q].lattice == cr[r].lattice && cr[q].a == cr[r].a && cr[q].c_over_a == cr[r].c_over_a &&
                cr[q].nx == cr[r].nx && cr[q].ny == cr[r].ny && cr[q].nz == cr[r].nz)
                same = q;
        if (same >= 0) {
            X.st_cnt = xr[same].st_cnt;
            X.st_margin = xr[same].st_margin;
            X.st_off = xr[same].st_off;
            continue;
        }
        std::vector<std::vector<std::pair<double, std::pair<float4, int>>>> per(X.nb);
        for (int b = 0; b < X.nb; ++b) {
            for (int dx = -M; dx <= M; ++dx)
                for (int dy = -M; dy <= M; ++dy)
                    for (int dz = -M; dz <= M; ++dz)
                        for (int b2 = 0; b2 < X.nb; ++b2) {
                            if (dx == 0 && dy == 0 && dz == 0 && b2 == b) continue;
                            const double ex = X.cell[0] * (dx + basis[b2][0] - basis[b][0]);
                            const double ey = X.cell[1] * (dy + basis[b2][1] - basis[b][1]);
                            const double ez = X.cell[2] * (dz + basis[b2][2] - basis[b][2]);
                            const double d = std::sqrt(ex * ex + ey * ey + ez * ez);
                            if (d >= Rst) continue;
                            const int code = ((dx + M) * LY + dy + M) | ((b2 * LZ + dz + M) << 16);
                            per[b].push_back({d, {make_float4((float)ex, (float)ey, (float)ez, code_bits(code)), code}});
                        }
            std::stable_sort(per[b].begin(), per[b].end(), [](const auto& p, const auto& q) {
                return p.first < q.first || (p.first == q.first && p.second.second < q.second.second);
            });
        }
        size_t cnt = 0;
        for (int b = 0; b < X.nb; ++b) cnt = std::max(cnt, per[b].size());
        cnt += NE_STENCIL_PAD;  // a runner may read a few entries past its scan bound
        if (cnt > NE_STENCIL_MAX) return fail(ctx, NE_EINVAL, "stencil too large");
        X.st_cnt = (int)cnt;
        X.st_margin = M;
        X.st_off = (int)sv.size();
        for (int b = 0; b < X.nb; ++b)
            for (size_t q = 0; q < cnt; ++q) {
                if (q < per[b].size()) {
                    sv.push_back(per[b][q].second.first);
                    sd.push_back((float)per[b][q].first);
                } else {  // padding: a site 1.7e4 A away (outside any cutoff), in the atom's own cell
                    sv.push_back(make_float4(1e4f, 1e4f, 1e4f, code_bits((M * LY + M) | (M << 16))));
                    sd.push_back(1e30f);
                }
            }
    }
    if (sv.size() > (size_t)ctx->max_rep * 4 * NE_STENCIL_MAX) return fail(ctx, NE_ENOMEM, "stencil capacity exceeded");
    int dev = 0, smem_max = 0;
    NE_CU(cudaGetDevice(&dev));
    NE_CU(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    // a crystal-runner CTA takes all of its SM's tensor memory, so no two may
    // share an SM: their shared memory is at least half of the SM's
    int smem_sm = 0;
    NE_CU(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    const size_t smem_floor = (size_t)smem_sm / 2 + 1024;
    const int nk = ctx->eam.n_knots;
    // shared memory of a launch over replicas rs: replica state, stencil,
    // lists and sums, then as many r intervals of the (phi, f) tables,
    // counted down from r_c, as fit (k_lo: first interval held)
    auto launch_smem = [&](const std::vector<int>& rs, size_t& smem, int& k_lo) -> bool {
        int gn = 0, gnb = 0, glut = 0;
        for (int r : rs) {
            gn = std::max(gn, xr[r].n);
            gnb = std::max(gnb, xr[r].nb * xr[r].st_cnt);
            const int Mr = xr[r].st_margin;
            // the kernel's wrapped-cell tables: (x, y) and, per basis site, z
            glut = std::max(glut, (xr[r].nx + 2 * Mr) * (xr[r].ny + 2 * Mr) + xr[r].nb * (xr[r].nz + 2 * Mr));
        }
        const size_t base = (ne::cluster_smem_bytes(gn, gnb, glut, P.npt) + 15) & ~(size_t)15;
        if (base > (size_t)smem_max) return false;
        const long long fit = ((long long)smem_max - (long long)base) / (2 * (long long)sizeof(float4));
        const int n_int = (int)std::min<long long>(nk - 1, fit);
        k_lo = nk - 1 - n_int;
        smem = std::max(base + (size_t)n_int * 2 * sizeof(float4), smem_floor);
        return smem <= (size_t)smem_max;
    };
    P.npt = false;
    for (int r = 0; r < n_rep; ++r) P.npt = P.npt || xr[r].npt != 0;
    if (brick) {
        // Brick runner: the largest threads-per-atom (8, 4, 3, 2, 1: each
        // divides the 768 threads into whole warps of one pair lane) at which
        // every replica's blocks of cells, one CTA each, fit the device at once
        int gnb = 0, glut = 0;
        for (int r = 0; r < n_rep; ++r) {
            gnb = std::max(gnb, xr[r].nb * xr[r].st_cnt);
            const int Mr = xr[r].st_margin;
            glut = std::max(glut, (xr[r].nx + 2 * Mr) * (xr[r].ny + 2 * Mr) + xr[r].nb * (xr[r].nz + 2 * Mr));
        }
        P.brick = false;
        for (int tpa : {8, 4, 3, 2, 1}) {
            const size_t base = (ne::brick_smem_bytes(tpa, gnb, glut, P.npt) + 15) & ~(size_t)15;
            if (base > (size_t)smem_max) continue;
            const long long fit = ((long long)smem_max - (long long)base) / (2 * (long long)sizeof(float4));
            const int n_int = (int)std::min<long long>(nk - 1, fit);
            const size_t smem = std::max(base + (size_t)n_int * 2 * sizeof(float4), smem_floor);
            if (smem > (size_t)smem_max) continue;
            const int per = ne::brick_atoms_per_cta(tpa);
            std::vector<int> cr_(n_rep);
            int total = 0;
            for (int r = 0; r < n_rep; ++r) {
                int C = (xr[r].n + per - 1) / per;
                while ((((xr[r].n + C - 1) / C) + xr[r].nb - 1) / xr[r].nb * xr[r].nb > per) ++C;
                cr_[r] = C;
                total += C;
            }
            const int cap = ne::brick_max_ctas(tpa, smem, P.npt);
            if (total > cap) continue;
            P.brick = true;
            P.tpa = tpa;
            P.n_cta = total;
            P.smem = smem;
            P.k_lo = nk - 1 - n_int;
            P.cta_rep.clear();
            for (int r = 0; r < n_rep; ++r) {
                xr[r].cta0 = (int)P.cta_rep.size();
                xr[r].ncta = cr_[r];
                xr[r].widx = r;
                for (int q = 0; q < cr_[r]; ++q) P.cta_rep.push_back(r);
            }
            break;
        }
        if (!P.brick)
            return fail(ctx, NE_ENOMEM, "brick runner: the batch needs more CTAs than the device holds at once");
        // exchange buffers, sized for the context (once)
        if (!ctx->bb.u4) {
            const size_t N = (size_t)ctx->max_atoms;
            NE_CU(cudaMalloc((void**)&ctx->bb.u4, sizeof(float4) * 2 * N));
            NE_CU(cudaMalloc((void**)&ctx->bb.fp, sizeof(float) * N));
            NE_CU(cudaMalloc((void**)&ctx->bb.bar, sizeof(unsigned) * 2));
            NE_CU(cudaMalloc((void**)&ctx->bb.abortf, sizeof(int)));
        }
        if (P.n_cta > ctx->bb_ctas) {
            if (ctx->bb.part) cudaFree(ctx->bb.part);
            if (ctx->bb.vir) cudaFree(ctx->bb.vir);
            if (ctx->cta_rep) cudaFree(ctx->cta_rep);
            ctx->bb.part = nullptr;
            ctx->bb.vir = nullptr;
            ctx->cta_rep = nullptr;
            ctx->bb_ctas = 0;
            NE_CU(cudaMalloc((void**)&ctx->bb.part, sizeof(float) * 2 * 16 * (size_t)P.n_cta));
            NE_CU(cudaMalloc((void**)&ctx->bb.vir, sizeof(float) * 6 * (size_t)P.n_cta));
            NE_CU(cudaMalloc((void**)&ctx->cta_rep, sizeof(int) * (size_t)P.n_cta));
            ctx->bb_ctas = P.n_cta;
        }
        P.xs = xr;
        P.groups.clear();
        NE_CU(cudaMemcpyAsync(ctx->xrep, P.xs.data(), sizeof(XRep) * n_rep, cudaMemcpyHostToDevice, st));
        NE_CU(cudaMemcpyAsync(ctx->cta_rep, P.cta_rep.data(), sizeof(int) * P.cta_rep.size(), cudaMemcpyHostToDevice, st));
        NE_CU(cudaMemcpyAsync(ctx->st_vec, sv.data(), sizeof(float4) * sv.size(), cudaMemcpyHostToDevice, st));
        NE_CU(cudaMemcpyAsync(ctx->st_dist, sd.data(), sizeof(float) * sd.size(), cudaMemcpyHostToDevice, st));
        P.key = plan_key(ctx, md, cr, n_rep);
        P.valid = true;
        return NE_OK;
    }
    P.brick = false;
    // Cluster size per replica: the smallest C whose CTAs hold it, unless the
    // caller fixed C (ne_ctx_set_cluster_size).  When every replica needs the
    // same smallest C, a larger C is taken if the device then runs the batch
    // in fewer waves or with fewer atoms per CTA: clusters must fit inside one
    // GPC, so the number of co-resident clusters (cudaOccupancyMaxActiveClusters)
    // is not 152 / C.  The estimate is waves x (atoms per CTA + 96), the
    // constant being the per-step cost that does not scale with the atoms.
    std::vector<int> csel(n_rep);
    bool uniform = true;
    for (int r = 0; r < n_rep; ++r) {
        csel[r] = ne::cluster_size_for(xr[r].n, xr[r].nb);
        uniform = uniform && csel[r] == csel[0];
    }
    if (ctx->cluster_c > 0) {
        for (int r = 0; r < n_rep; ++r) {
            if (ctx->cluster_c < csel[r])
                return fail(ctx, NE_EINVAL, "crystal runner: the fixed cluster size is too small for a replica");
            csel[r] = ctx->cluster_c;
        }
    } else if (uniform) {
        std::vector<int> all(n_rep);
        for (int r = 0; r < n_rep; ++r) all[r] = r;
        size_t smem = 0;
        int k_lo = 0;
        if (!launch_smem(all, smem, k_lo)) return fail(ctx, NE_EINVAL, "replica too large for the crystal runner");
        int best = csel[0];
        double best_t = -1.0;
        for (int C = csel[0]; C <= 16; ++C) {
            const int act = ne::cluster_max_active(C, smem);
            if (act < 1) continue;
            int A = 0;
            for (int r = 0; r < n_rep; ++r) A = std::max(A, ne::cluster_atoms_for(xr[r].n, C, xr[r].nb));
            const double t = (double)((n_rep + act - 1) / act) * (A + 96);
            if (best_t < 0.0 || t < 0.97 * best_t) {
                best = C;
                best_t = t;
            }
        }
        for (int r = 0; r < n_rep; ++r) csel[r] = best;
    }
    // Replicas grouped by cluster size, each group one launch on its own
    // stream, largest replicas first.
    std::vector<int> order(n_rep);
    for (int r = 0; r < n_rep; ++r) order[r] = r;
    auto csize = [&](int r) { return csel[r]; };
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) {
        return csize(p) > csize(q) || (csize(p) == csize(q) && xr[p].n > xr[q].n);
    });
    P.xs.assign(n_rep, XRep{});
    for (int q = 0; q < n_rep; ++q) {
        P.xs[q] = xr[order[q]];
        P.xs[q].widx = order[q];
    }
    P.groups.clear();
    for (int q = 0; q < n_rep;) {
        int e = q;
        while (e < n_rep && csize(order[e]) == csize(order[q])) ++e;
        CrGroup g{};
        g.b = q;
        g.e = e;
        g.C = csize(order[q]);
        std::vector<int> rs;
        for (int t = q; t < e; ++t) rs.push_back(order[t]);
        if (!launch_smem(rs, g.smem, g.k_lo)) return fail(ctx, NE_EINVAL, "replica too large for the crystal runner");
        P.groups.push_back(g);
        q = e;
    }
    if (P.groups.size() > 16) return fail(ctx, NE_EINVAL, "crystal runner: at most 16 size classes per call");
    if (P.groups.size() > 1 && !ctx->gev[0]) {
        for (int g = 0; g < 17; ++g) NE_CU(cudaEventCreateWithFlags(&ctx->gev[g], cudaEventDisableTiming));
        for (int g = 0; g < 16; ++g) NE_CU(cudaStreamCreateWithFlags(&ctx->gst[g], cudaStreamNonBlocking));
    }
    // the host vectors stay in the plan until the next rebuild, which comes
    // after this call's closing synchronisation: the copies never outlive them
    NE_CU(cudaMemcpyAsync(ctx->xrep, P.xs.data(), sizeof(XRep) * n_rep, cudaMemcpyHostToDevice, st));
    NE_CU(cudaMemcpyAsync(ctx->st_vec, sv.data(), sizeof(float4) * sv.size(), cudaMemcpyHostToDevice, st));
    NE_CU(cudaMemcpyAsync(ctx->st_dist, sd.data(), sizeof(float) * sd.size(), cudaMemcpyHostToDevice, st));
    P.key = plan_key(ctx, md, cr, n_rep);
    P.valid = true;
    return NE_OK;
}

// lambda(s) of every step of the schedule, s = 0 .. 2 t_eq + 2 t_s + 1,
// computed once per schedule (FP64) and read by the persistent kernel
static ne_status lambda_table(ne_ctx* ctx, const Sched& S, cudaStream_t st)
{
    if (ctx->lam_valid && same_sched(ctx->lam_sched, S)) return NE_OK;
    const long long need = 2 * S.t_eq + 2 * S.t_s + 2;
    ctx->lam_valid = false;
    if (need > ctx->lam_cap) {
        // every earlier call ended with a synchronisation of its stream, so
        // no kernel still reads the old table
        if (ctx->lam_tab) cudaFree(ctx->lam_tab);
        ctx->lam_tab = nullptr;
        ctx->lam_cap = 0;
        NE_CU(cudaMalloc((void**)&ctx->lam_tab, sizeof(double) * (size_t)need));
        ctx->lam_cap = need;
    }
    NE_CU(ne::launch_lambda_table(S, 0, need, ctx->lam_tab, st));
    ++ctx->cr_launches;
    ctx->lam_sched = S;
    ctx->lam_valid = true;
    return NE_OK;
}

static ne_status crystal_segment_impl(ne_ctx* ctx, const ne_md_params* md, const ne_crystal* cr, int n_rep,
                                      double* x_dev, double* v_dev, double* W_dev, double* Wcum_dev,
                                      long long step_begin, long long n_steps, void* stream)
{
    if (!ctx || !md || !cr || !x_dev || !v_dev || !W_dev || n_rep < 1) return NE_EINVAL;
    if (n_rep > ctx->max_rep) return fail(ctx, NE_ENOMEM, "replica count exceeds the context");
    std::vector<int> off(n_rep + 1, 0);
    for (int r = 0; r < n_rep; ++r) {
        const int nb = cr[r].lattice == NE_BCC ? 2 : 4;
        if (cr[r].nx < 1 || cr[r].ny < 1 || cr[r].nz < 1 || cr[r].nx > 4096 || cr[r].ny > 4096 || cr[r].nz > 4096)
            return fail(ctx, NE_EINVAL, "crystal: at least 3 cells per axis");
        off[r + 1] = off[r] + (int)std::min<long long>((long long)nb * cr[r].nx * cr[r].ny * cr[r].nz, 1 << 20);
    }
    ne_status s = check_batch(ctx, md, n_rep, off.data());
    if (s) return s;
    if (md[0].prec != NE_MIXED) return fail(ctx, NE_EINVAL, "the crystal runner is mixed precision; use ne_switch_run_segment for FP64");

    const long long S_total = 2 * md[0].t_eq + 2 * md[0].t_s;
    if (step_begin < 0 || n_steps < 0 || step_begin + n_steps > S_total)
        return fail(ctx, NE_EINVAL, "step range outside the schedule");
    cudaStream_t st = (cudaStream_t)stream;
    // a batch with species tables is planned on every call: its species
    // arrays are read back and checked each time
    bool species = false;
    for (int r = 0; r < n_rep; ++r) species = species || md[r].n_species >= 2;
    if (species || !ctx->plan.valid || ctx->plan.key != plan_key(ctx, md, cr, n_rep)) {
        s = build_plan(ctx, md, cr, n_rep, st);
        if (s) return s;
    }
    const CrPlan& P = ctx->plan;
    // the status word and the per-replica words that follow it
    NE_CU(cudaMemsetAsync(ctx->status, 0, sizeof(int) * (size_t)(1 + n_rep), st));
    ctx->last_nrep_cr = n_rep;
    Sched S = make_sched(md[0]);
    s = lambda_table(ctx, S, st);
    if (s) return s;
    if (!ctx->ev_run[0]) {
        NE_CU(cudaEventCreate(&ctx->ev_run[0]));
        NE_CU(cudaEventCreate(&ctx->ev_run[1]));
    }
    NE_CU(cudaEventRecord(ctx->ev_run[0], st));
    if (P.brick) {
        const long long n_tot = [&] {
            long long t = 0;
            for (const XRep& X : P.xs) t = std::max<long long>(t, (long long)X.off + X.n);
            return t;
        }();
        NE_CU(ne::launch_brick(P.tpa, ctx->xrep, ctx->cta_rep, P.n_cta, P.smem, ctx->st_vec, ctx->st_dist, x_dev,
                               v_dev, W_dev, ctx->status, S, step_begin, n_steps, ctx->tab, ctx->work, P.k_lo,
                               ctx->lam_tab + step_begin, Wcum_dev, ctx->bb, n_tot, st, P.npt, ctx->cr_boxes));
        ++ctx->cr_launches;
        NE_CU(cudaEventRecord(ctx->ev_run[1], st));
        ctx->run_timed = true;
        if (P.npt) {  // ne_ctx_boxes reads the boxes this call reached
            ctx->boxes_from_runner = true;
            ctx->last_nrep = n_rep;
        }
        return finish(ctx, st);
    }
    const bool multi = P.groups.size() > 1;
    if (multi) NE_CU(cudaEventRecord(ctx->gev[16], st));
    for (size_t g = 0; g < P.groups.size(); ++g) {
        const CrGroup& G = P.groups[g];
        cudaStream_t gs = multi ? ctx->gst[g] : st;
        if (multi) NE_CU(cudaStreamWaitEvent(gs, ctx->gev[16], 0));
        NE_CU(ne::launch_cluster(ctx->xrep + G.b, G.e - G.b, G.C, G.smem, ctx->st_vec, ctx->st_dist, x_dev, v_dev,
                                 W_dev, ctx->status, S, step_begin, n_steps, ctx->tab, ctx->work, G.k_lo,
                                 ctx->lam_tab + step_begin, Wcum_dev, gs, P.npt, ctx->cr_boxes));
        ++ctx->cr_launches;
        if (multi) {
            NE_CU(cudaEventRecord(ctx->gev[g], gs));
            NE_CU(cudaStreamWaitEvent(st, ctx->gev[g], 0));
        }
    }
    NE_CU(cudaEventRecord(ctx->ev_run[1], st));
    ctx->run_timed = true;
    if (P.npt) {  // ne_ctx_boxes reads the boxes this call reached
        ctx->boxes_from_runner = true;
        ctx->last_nrep = n_rep;
    }
    return finish(ctx, st);
}

ne_status ne_profile_segment(ne_ctx* ctx, const ne_md_params* md, int n_rep, const int* offsets_host,
                             double* x_dev, double* v_dev, const double* x0_dev, const double* boxes_host,
                             double* W_dev, long long step_begin, long long n_steps, double* ms_host,
                             long long* launches_host, void* stream)
{
    if (!ctx || !md || !offsets_host || !x_dev || !v_dev || !x0_dev || !boxes_host || !W_dev || !ms_host ||
        !launches_host || n_rep < 1 || n_steps < 1 || n_steps > 100000)
        return NE_EINVAL;
    if (n_rep > ctx->max_rep) return fail(ctx, NE_ENOMEM, "replica count exceeds the context");
    ne_status s = check_batch(ctx, md, n_rep, offsets_host);
    if (s) return s;
    const long long S_total = 2 * md[0].t_eq + 2 * md[0].t_s;
    if (step_begin < 0 || step_begin + n_steps > S_total) return fail(ctx, NE_EINVAL, "step range outside the schedule");
    cudaStream_t st = (cudaStream_t)stream;
    RunArgs a{};
    a.x = x_dev;
    a.v = v_dev;
    a.x0 = x0_dev;
    a.W = W_dev;
    DevBatch B;
    s = setup_batch(ctx, n_rep, offsets_host, boxes_host, md, 1, -1.0, B, a, st);
    if (s) return s;
    Sched S = make_sched(md[0]);
    s = profile_steps(ctx, B, S, md[0].prec == NE_MIXED, step_begin, n_steps, ms_host, launches_host, st);
    if (s) return s;
    return finish(ctx, st);
}

ne_status ne_msd_fit_batched(ne_ctx* ctx, const ne_md_params* md, int n_rep, const int* offsets_host,
                             double* x_dev, double* v_dev, const double* x0_dev, const double* boxes_host,
                             long long n_eq, long long n_samples, int stride, double* msd_host, double* k_host,
                             void* stream)
{
    if (!ctx || !md || n_rep < 1 || !offsets_host || !x_dev || !v_dev || !x0_dev || !boxes_host || n_eq < 0 ||
        n_samples < 1 || stride < 1)
        return NE_EINVAL;
    if (n_rep > ctx->max_rep) return fail(ctx, NE_ENOMEM, "replica count exceeds the context");
    for (int r = 0; r < n_rep; ++r) {
        ne_status s = check_md(ctx, &md[r]);
        if (s) return s;
        if (md[r].npt) return fail(ctx, NE_EINVAL, "the barostat runs in the switching runs (ne_switch_run_segment, ne_rs_run)");
        if (md[r].n_species >= 2) return fail(ctx, NE_EINVAL, "several species: use ne_msd_fit_species");
        if (md[r].dt != md[0].dt || md[r].damp != md[0].damp || md[r].fix_cm != md[0].fix_cm ||
            md[r].prec != md[0].prec)
            return fail(ctx, NE_EINVAL, "replicas must share dt, damp, fix_cm and precision");
        if (offsets_host[r + 1] - offsets_host[r] < 2) return fail(ctx, NE_EINVAL, "offsets must increase by at least 2");
    }
    if (offsets_host[0] != 0) return fail(ctx, NE_EINVAL, "offsets must start at 0");
    cudaStream_t st = (cudaStream_t)stream;
    RunArgs a{};
    a.x = x_dev;
    a.v = v_dev;
    a.x0 = x0_dev;
    a.W = ctx->W;
    DevBatch B;
    ne_status s = setup_batch(ctx, n_rep, offsets_host, boxes_host, md, 1, -1.0, B, a, st);
    if (s) return s;
    Sched S = make_sched(md[0]);
    S.kind = SCHED_FIXED;
    S.path = NE_PATH_FL;
    S.lam_a = S.lam_b = 0.0;
    S.s0 = -1;
    S.stream = STREAM_MSD;
    double* acc = ctx->scratch;  // one msd sum per replica
    NE_CU(cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)n_rep, st));
    s = run_steps(ctx, B, S, md[0].prec == NE_MIXED, 0, n_eq + n_samples * stride, st, acc, n_eq, stride);
    if (s) return s;
    std::vector<double> sum(n_rep, 0.0);
    NE_CU(cudaMemcpyAsync(sum.data(), acc, sizeof(double) * (size_t)n_rep, cudaMemcpyDeviceToHost, st));
    s = finish(ctx, st);
    if (s) return s;
    for (int r = 0; r < n_rep; ++r) {
        const double msd = sum[r] / (double)n_samples;
        if (msd_host) msd_host[r] = msd;
        if (k_host) k_host[r] = 3.0 * kB * md[r].T / msd;
    }
    return NE_OK;
}

ne_status ne_msd_fit_species(ne_ctx* ctx, const ne_md_params* md, double* x_dev, double* v_dev,
                             const double* x0_dev, int n, const double box[3], long long n_eq,
                             long long n_samples, int stride, double* msd_s_host, double* k_s_host, void* stream)
{
    if (!ctx || !md || !x_dev || !v_dev || !x0_dev || !box || n < 2 || n_eq < 0 || n_samples < 1 || stride < 1)
        return NE_EINVAL;
    ne_status s = check_md(ctx, md);
    if (s) return s;
    if (md->n_species < 2) return fail(ctx, NE_EINVAL, "ne_msd_fit_species needs species tables (n_species >= 2)");
    if (md->npt) return fail(ctx, NE_EINVAL, "the barostat runs in the switching runs (ne_switch_run_segment, ne_rs_run)");
    cudaStream_t st = (cudaStream_t)stream;
    const int off[2] = {0, n};
    RunArgs a{};
    a.x = x_dev;
    a.v = v_dev;
    a.x0 = x0_dev;
    a.W = ctx->W;
    DevBatch B;
    s = setup_batch(ctx, 1, off, box, md, 0, -1.0, B, a, st);
    if (s) return s;
    const RepDev& R = ctx->rep_h[0];
    Sched S = make_sched(*md);
    S.kind = SCHED_FIXED;
    S.path = NE_PATH_FL;
    S.lam_a = S.lam_b = 0.0;
    S.s0 = -1;
    S.stream = STREAM_MSD;
    double* acc = ctx->scratch;  // one msd sum per species
    NE_CU(cudaMemsetAsync(acc, 0, sizeof(double) * NE_MAX_SPECIES, st));
    s = run_steps(ctx, B, S, md->prec == NE_MIXED, 0, n_eq + n_samples * stride, st, acc, n_eq, stride);
    if (s) return s;
    double sum[NE_MAX_SPECIES] = {};
    NE_CU(cudaMemcpyAsync(sum, acc, sizeof(sum), cudaMemcpyDeviceToHost, st));
    s = finish(ctx, st);
    if (s) return s;
    std::vector<int> cnt(NE_MAX_SPECIES, 0);
    {
        std::vector<unsigned char> sp(n);
        NE_CU(cudaMemcpy(sp.data(), md->species_dev, (size_t)n, cudaMemcpyDeviceToHost));
        for (int q = 0; q < n; ++q) ++cnt[sp[q]];
    }
    for (int q = 0; q < R.nsp; ++q) {
        const double msd = cnt[q] ? sum[q] / (double)n_samples : 0.0;
        if (msd_s_host) msd_s_host[q] = msd;
        if (k_s_host) k_s_host[q] = msd > 0 ? 3.0 * kB * md->T / msd : 0.0;
    }
    return NE_OK;
}

ne_status ne_msd_fit(ne_ctx* ctx, const ne_md_params* md, double* x_dev, double* v_dev, const double* x0_dev,
                     int n, const double box[3], long long n_eq, long long n_samples, int stride,
                     double* msd_host, double* k_host, void* stream)
{
    if (!ctx || !md || !box || n < 2) return NE_EINVAL;
    const int off[2] = {0, n};
    return ne_msd_fit_batched(ctx, md, 1, off, x_dev, v_dev, x0_dev, box, n_eq, n_samples, stride, msd_host,
                              k_host, stream);
}

// ------------------------------------------------------------ assembly
ne_status ne_free_energy(int n, double V, double T, double mass, double k, const double* W_fwd,
                         const double* W_bwd, int n_seeds, double* F_per_atom, double* stderr_per_atom,
                         double* Ediss_per_atom)
{
    if (n < 1 || n_seeds < 1 || !W_fwd || !W_bwd || !(V > 0) || !(T > 0) || !(mass > 0) || !(k > 0))
        return NE_EINVAL;
    double wf = 0, wb = 0;
    for (int q = 0; q < n_seeds; ++q) {
        wf += W_fwd[q];
        wb += W_bwd[q];
    }
    wf /= n_seeds;
    wb /= n_seeds;
    const double kT = kB * T, w = std::sqrt(k / mass);
    const double FE = 3.0 * n * kT * std::log(HBAR * w / kT);            // Einstein crystal
    const double dcm = kT * std::log(n / V * std::pow(2.0 * PI * kT / (n * k), 1.5));  // eq. cm
    if (F_per_atom) *F_per_atom = (FE + 0.5 * (wf - wb) + dcm) / n;
    if (stderr_per_atom) {
        double se = 0.0;
        if (n_seeds > 1) {
            double m = 0.5 * (wf - wb) / n, ss = 0.0;
            for (int q = 0; q < n_seeds; ++q) {
                double d = 0.5 * (W_fwd[q] - W_bwd[q]) / n - m;
                ss += d * d;
            }
            se = std::sqrt(ss / (n_seeds - 1) / n_seeds);
        }
        *stderr_per_atom = se;
    }
    if (Ediss_per_atom) *Ediss_per_atom = -0.5 * (wf + wb) / n;
    return NE_OK;
}

ne_status ne_free_energy_species(int n, const int* species, int n_species, const double* mass_s,
                                 const double* k_s, double V, double T, const double* W_fwd,
                                 const double* W_bwd, int n_seeds, double* F_per_atom,
                                 double* stderr_per_atom, double* Ediss_per_atom)
{
    if (n < 1 || n_seeds < 1 || n_species < 1 || !species || !mass_s || !k_s || !W_fwd || !W_bwd ||
        !(V > 0) || !(T > 0))
        return NE_EINVAL;
    for (int s = 0; s < n_species; ++s)
        if (!(mass_s[s] > 0) || !(k_s[s] > 0)) return NE_EINVAL;
    std::vector<long long> count(n_species, 0);
    for (int i = 0; i < n; ++i) {
        if (species[i] < 0 || species[i] >= n_species) return NE_EINVAL;
        ++count[species[i]];
    }
    const double kT = kB * T;
    // F_E: one oscillator frequency per species; the fixed centre is the
    // mass-weighted one, with per-axis variance kT sum_s N_s m_s^2 / k_s / M^2.
    double FE = 0.0, M = 0.0, m2k = 0.0;
    for (int s = 0; s < n_species; ++s) {
        if (!count[s]) continue;
        const double Ns = (double)count[s], w = std::sqrt(k_s[s] / mass_s[s]);
        FE += 3.0 * Ns * kT * std::log(HBAR * w / kT);
        M += Ns * mass_s[s];
        m2k += Ns * mass_s[s] * mass_s[s] / k_s[s];
    }
    const double sigma2 = kT * m2k / (M * M);
    const double dcm = kT * std::log(n / V * std::pow(2.0 * PI * sigma2, 1.5));
    double wf = 0, wb = 0;
    for (int q = 0; q < n_seeds; ++q) {
        wf += W_fwd[q];
        wb += W_bwd[q];
    }
    wf /= n_seeds;
    wb /= n_seeds;
    if (F_per_atom) *F_per_atom = (FE + 0.5 * (wf - wb) + dcm) / n;
    if (stderr_per_atom) {
        double se = 0.0;
        if (n_seeds > 1) {
            double m = 0.5 * (wf - wb) / n, ss = 0.0;
            for (int q = 0; q < n_seeds; ++q) {
                double d = 0.5 * (W_fwd[q] - W_bwd[q]) / n - m;
                ss += d * d;
            }
            se = std::sqrt(ss / (n_seeds - 1) / n_seeds);
        }
        *stderr_per_atom = se;
    }
    if (Ediss_per_atom) *Ediss_per_atom = -0.5 * (wf + wb) / n;
    return NE_OK;
}

ne_status ne_lambda(const ne_md_params* md, long long step, double* lambda_host)
{
    if (!md || !lambda_host) return NE_EINVAL;
    if (md->path != NE_PATH_FL && md->path != NE_PATH_RS) return NE_EINVAL;
    if (md->path == NE_PATH_FL && md->lambda_fn != 1 && md->lambda_fn != 2) return NE_EINVAL;
    if (md->path == NE_PATH_RS && !(md->lambda_f > 0 && md->lambda_f < 1)) return NE_EINVAL;
    if (md->t_s < 1 || md->t_eq < 0 || step < 0 || step > 2 * md->t_eq + 2 * md->t_s) return NE_EINVAL;
    *lambda_host = ne_sched_lambda(make_sched(*md), step);
    return NE_OK;
}

ne_status ne_pressure(int n_dof, double T, double V, const double* W_host, int n_samples, double* P_host,
                      double* stderr_host)
{
    if (n_dof < 0 || !(T >= 0) || !(V > 0) || !W_host || n_samples < 1 || !P_host) return NE_EINVAL;
    double mean = 0.0;
    for (int q = 0; q < n_samples; ++q) mean += W_host[q];
    mean /= n_samples;
    double ss = 0.0;
    for (int q = 0; q < n_samples; ++q) ss += (W_host[q] - mean) * (W_host[q] - mean);
    *P_host = (n_dof * kB * T + mean) / (3.0 * V);
    if (stderr_host)
        *stderr_host = n_samples > 1 ? std::sqrt(ss / (n_samples - 1)) / std::sqrt((double)n_samples) / (3.0 * V) : 0.0;
    return NE_OK;
}

ne_status ne_jarzynski(double T, const double* W_host, int n_seeds, double* dF_out)
{
    if (!W_host || n_seeds < 1 || !(T > 0) || !dF_out) return NE_EINVAL;
    const double kT = kB * T;
    double wmin = W_host[0];
    for (int q = 1; q < n_seeds; ++q) wmin = std::min(wmin, W_host[q]);
    double acc = 0.0;  // every term exp(-(W - W_min)/kT) <= 1
    for (int q = 0; q < n_seeds; ++q) acc += std::exp(-(W_host[q] - wmin) / kT);
    *dF_out = wmin - kT * std::log(acc / n_seeds);
    return NE_OK;
}

ne_status ne_rs_free_energy(int n, double T0, double F0_T0, double lambda_f, long long t_s,
                            const double* Wf, const double* Wb, int n_seeds, const double* T_grid, int n_T,
                            double* F_per_atom)
{
    if (n < 1 || t_s < 1 || n_seeds < 1 || !Wf || !Wb || !T_grid || !F_per_atom || !(lambda_f > 0 && lambda_f < 1))
        return NE_EINVAL;
    const size_t m = (size_t)t_s + 1;
    std::vector<double> cf(m, 0.0), cb(m, 0.0), lf(m), lb(m);
    for (int q = 0; q < n_seeds; ++q)
        for (size_t k = 0; k < m; ++k) {
            cf[k] += Wf[q * m + k] / n_seeds;
            cb[k] += Wb[q * m + k] / n_seeds;
        }
    for (size_t k = 0; k < m; ++k) {
        lf[k] = ne_lambda_rs(lambda_f, (double)k / t_s);
        lb[k] = ne_lambda_rs(lambda_f, 1.0 - (double)k / t_s);
    }
    for (int g = 0; g < n_T; ++g) {
        const double l = T0 / T_grid[g];
        if (l > 1.0 || l < lambda_f) return NE_EINVAL;
        // forward: lambda falls from 1 to lambda_f; backward rises back
        size_t kf = 0;
        while (kf + 1 < m - 1 && lf[kf + 1] > l) ++kf;
        double af = (l - lf[kf]) / (lf[kf + 1] - lf[kf]);
        const double w1l = cf[kf] + af * (cf[kf + 1] - cf[kf]);
        size_t kb = 0;
        while (kb + 1 < m - 1 && lb[kb + 1] < l) ++kb;
        double ab = (l - lb[kb]) / (lb[kb + 1] - lb[kb]);
        const double wl1 = cb[m - 1] - (cb[kb] + ab * (cb[kb + 1] - cb[kb]));
        const double F = F0_T0 / l + 1.5 * n * kB * T0 * std::log(l) / l + (w1l - wl1) / (2.0 * l);
        F_per_atom[g] = F / n;
    }
    return NE_OK;
}

}  // extern "C"

// dU/dx = -F scaled by the upstream gradient (used by ne_eam_backward).
__global__ void k_scale(double* p, int n, double s)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) p[q] *= s;
}

namespace ne {
void launch_scale(double* p, int n, double s, cudaStream_t st) { k_scale<<<64, 256, 0, st>>>(p, n, s); }
}  // namespace ne
