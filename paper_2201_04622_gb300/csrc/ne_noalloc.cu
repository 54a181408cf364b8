// ne_noalloc.cu -- ne_eam_energy_forces_noalloc: the EAM energy and forces of
// one configuration without any device allocation.
//
// Some callers cannot call cudaMalloc once they are running: an MD engine or
// framework that has reserved the device memory for its own pool, or a
// real-time pipeline that forbids allocation after start-up (cudaMalloc can
// synchronise the device and can fail when memory is fragmented).  For them
// this entry point takes its scratch -- spline tables, cell arrays,
// neighbour lists, per-atom buffers and sums -- from one file-scope
// __device__ array of fixed size, NE_NOALLOC_SCRATCH_BYTES, which every GPU
// that loads the library holds until the process exits.  It runs the same
// kernels as ne_eam_energy_forces.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/ne.h"
#include "ne_internal.cuh"

namespace {

constexpr int NA = NE_NOALLOC_MAX_ATOMS;
constexpr int NK = NE_NOALLOC_MAX_KNOTS;
constexpr int TPA = 4;
constexpr int TILES = (NA + NE_TILE - 1) / NE_TILE;
constexpr int CELLS = 2 * NA + 27;

constexpr size_t up(size_t b) { return (b + 255) / 256 * 256; }

// byte offsets of the sub-buffers inside the scratch array
constexpr size_t O_THETA = 0;
constexpr size_t O_PF32 = O_THETA + up(sizeof(double) * 6 * NK);
constexpr size_t O_PF64 = O_PF32 + up(sizeof(float4) * 2 * NK);
constexpr size_t O_F32 = O_PF64 + up(sizeof(ned4) * 2 * NK);
constexpr size_t O_F64 = O_F32 + up(sizeof(float4) * NK);
constexpr size_t O_POS32 = O_F64 + up(sizeof(ned4) * NK);
constexpr size_t O_POSF = O_POS32 + up(sizeof(float4) * NA);
constexpr size_t O_PBUILD = O_POSF + up(sizeof(float4) * NA);
constexpr size_t O_FORCE32 = O_PBUILD + up(sizeof(float4) * NA);
constexpr size_t O_FORCE64 = O_FORCE32 + up(sizeof(float4) * NA);
constexpr size_t O_DF64 = O_FORCE64 + up(sizeof(double) * 3 * NA);
constexpr size_t O_NBR = O_DF64 + up(sizeof(double) * NA);
constexpr size_t O_NCNT = O_NBR + up(sizeof(int) * (size_t)NA * NE_NMAX);
constexpr size_t O_SL = O_NCNT + up(sizeof(int) * NA);
constexpr size_t O_SCNT = O_SL + up(sizeof(int) * (size_t)NA * NE_SMAX);
constexpr size_t O_CELLOF = O_SCNT + up(sizeof(int) * NA * TPA);
constexpr size_t O_SORTED = O_CELLOF + up(sizeof(int) * NA);
constexpr size_t O_CSTART = O_SORTED + up(sizeof(int) * NA);
constexpr size_t O_CFILL = O_CSTART + up(sizeof(int) * (CELLS + 1));
constexpr size_t O_PARTA = O_CFILL + up(sizeof(int) * CELLS);
constexpr size_t O_PARTB = O_PARTA + up(sizeof(double) * TILES * NPA);
constexpr size_t O_TOT = O_PARTB + up(sizeof(double) * TILES * NPB);
constexpr size_t O_REP = O_TOT + up(sizeof(double) * NTOT);
constexpr size_t O_TILEREP = O_REP + up(sizeof(RepDev));
constexpr size_t O_SMALL = O_TILEREP + up(sizeof(int) * TILES);
// small words: tile_done, flags, building, status (ints), rebuilds, step counter (8 bytes)
constexpr size_t O_END = O_SMALL + 256;
static_assert(O_END <= NE_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds NE_NOALLOC_SCRATCH_BYTES");

// The scratch itself.  In host code this name is only a stand-in for the
// symbol; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[NE_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
unsigned char* g_addr[256] = {};

// Device address of the scratch on the current device (with that device
// current).  Looked up again on every call made outside a stream capture --
// a cudaDeviceReset reloads the module, and the array may then sit at another
// address -- and kept per device for calls made while `st` is capturing,
// where the last address looked up is used.
cudaError_t scratch_address(cudaStream_t st, unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    bool capturing = true;  // an error of the query counts as capturing
    if (cudaStreamIsCapturing(st, &cap) == cudaSuccess) capturing = cap != cudaStreamCaptureStatusNone;
    else (void)cudaGetLastError();
    std::lock_guard<std::mutex> lk(g_mu);
    if (!capturing || !g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = (unsigned char*)p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// Knot parameters (value, slope) of the analytic Fe-like EAM evaluated on
// the device: phi and f on [0, r_c], F on [0, rho_max]; the embedding slope
// at rho = 0 (infinite) is replaced by the secant slope to the next knot.
__global__ void k_theta(ne_eam_params p, double* theta)
{
    const int nk = p.n_knots;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    for (int fn = 0; fn < 3; ++fn) {
        const double h = (fn == 2 ? p.rho_max : p.r_c) / (nk - 1);
        const double x = k * h;
        double y, dy;
        if (fn == 2) {
            if (k == 0) {
                y = 0.0;
                dy = -p.B * sqrt(h) / h;
            } else {
                y = -p.B * sqrt(x);
                dy = -0.5 * p.B / sqrt(x);
            }
        } else {
            double s = 1.0, ds = 0.0;
            if (x >= p.r_c) {
                s = 0.0;
            } else if (x > p.r_s) {
                const double w = p.r_c - p.r_s, t = (x - p.r_s) / w, om = 1.0 - t;
                s = om * om * om * (1.0 + t * (3.0 + 6.0 * t));
                ds = -30.0 * t * t * om * om / w;
            }
            const double c = fn == 0 ? p.alpha : p.beta;
            const double e = (fn == 0 ? p.A : 1.0) * exp(-c * (x / p.r_e - 1.0));
            y = e * s;
            dy = e * (ds - c / p.r_e * s);
        }
        theta[((size_t)fn * nk + k) * 2] = y;
        theta[((size_t)fn * nk + k) * 2 + 1] = dy;
    }
}

}  // namespace

extern "C" ne_status ne_eam_energy_forces_noalloc(const ne_eam_params* eam, ne_precision prec,
                                                  const double* x_dev, int n, const double box[3],
                                                  double* f_dev, double* e_dev, void* stream)
{
    if (!eam || !x_dev || !box || n < 2 || (!f_dev && !e_dev)) return NE_EINVAL;
    if (prec != NE_FP64 && prec != NE_MIXED) return NE_EINVAL;
    if (eam->n_knots < 4 || !(eam->r_c > 0) || !(eam->rho_max > 0) || !(eam->r_s < eam->r_c)) return NE_EINVAL;
    // the potential is built from the analytic parameters alone: placeholders
    // (NaN, as a file-loaded potential carries) are refused, not tabulated
    if (!std::isfinite(eam->A) || !std::isfinite(eam->alpha) || !std::isfinite(eam->beta) ||
        !std::isfinite(eam->B) || !(eam->r_e > 0) || !std::isfinite(eam->r_c) || !std::isfinite(eam->rho_max))
        return NE_EINVAL;
    if (n > NE_NOALLOC_MAX_ATOMS || eam->n_knots > NE_NOALLOC_MAX_KNOTS) return NE_ENOMEM;
    const double rc = eam->r_c;
    for (int d = 0; d < 3; ++d)
        if (!(box[d] > 2.0 * rc)) return NE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    if (scratch_address(st, &base) != cudaSuccess) return NE_ECUDA;

    // ---- one replica: host-side description on the stack
    RepDev R{};
    for (int d = 0; d < 3; ++d) {
        R.L[d] = box[d];
        R.invL[d] = 1.0 / box[d];
        R.nc[d] = (int)std::min(std::floor(box[d] / rc), 1024.0);
    }
    while ((long long)R.nc[0] * R.nc[1] * R.nc[2] > 2ll * n + 27) {
        int d = R.nc[0] >= R.nc[1] && R.nc[0] >= R.nc[2] ? 0 : (R.nc[1] >= R.nc[2] ? 1 : 2);
        R.nc[d] -= 1;
    }
    if (R.nc[0] < 3 || R.nc[1] < 3 || R.nc[2] < 3) R.nc[0] = R.nc[1] = R.nc[2] = 0;
    R.m = 1.0;
    R.c1 = 1.0;
    R.rlist2 = rc * rc;
    R.off = 0;
    R.n = n;
    R.tile0 = 0;
    R.ntile = (n + NE_TILE - 1) / NE_TILE;
    R.cell_off = 0;
    R.dof = 3 * n;
    int tile_rep[TILES] = {};

    // ---- batch view of the scratch
    const int nk = eam->n_knots;
    DevBatch B{};
    B.n_rep = 1;
    B.n_tot = n;
    B.n_tiles = R.ntile;
    B.tpa = TPA;
    B.rep = (const RepDev*)(base + O_REP);
    B.tile_rep = (const int*)(base + O_TILEREP);
    B.x = const_cast<double*>(x_dev);
    B.pos32 = (float4*)(base + O_POS32);
    B.posF = (float4*)(base + O_POSF);
    B.pbuild = (float4*)(base + O_PBUILD);
    B.f32 = (float4*)(base + O_FORCE32);
    B.f64 = (double*)(base + O_FORCE64);
    B.dF64 = (double*)(base + O_DF64);
    B.nbr = (int*)(base + O_NBR);
    B.ncnt = (int*)(base + O_NCNT);
    B.sl = (int*)(base + O_SL);
    B.scnt = (int*)(base + O_SCNT);
    B.cellof = (int*)(base + O_CELLOF);
    B.sorted = (int*)(base + O_SORTED);
    B.cstart = (int*)(base + O_CSTART);
    B.cfill = (int*)(base + O_CFILL);
    B.partA = (double*)(base + O_PARTA);
    B.partB = (double*)(base + O_PARTB);
    B.tot = (double*)(base + O_TOT);
    int* small = (int*)(base + O_SMALL);
    B.tile_done = (unsigned*)(small + 0);
    B.flags = small + 1;
    B.building = small + 2;
    B.status = small + 3;
    B.rebuilds = (unsigned long long*)(base + O_SMALL + 16);
    long long* step_ctr = (long long*)(base + O_SMALL + 24);
    B.trace_stride = 1;
    Tables& t = B.tab;
    t.pf32 = (const float4*)(base + O_PF32);
    t.pf64 = (const ned4*)(base + O_PF64);
    t.F32 = (const float4*)(base + O_F32);
    t.F64 = (const ned4*)(base + O_F64);
    t.nk = nk;
    t.h_r = rc / (nk - 1);
    t.inv_h_r = (nk - 1) / rc;
    t.h_rho = eam->rho_max / (nk - 1);
    t.inv_h_rho = (nk - 1) / eam->rho_max;
    t.r_c = rc;
    t.rho_max = eam->rho_max;
    t.inv_h_rf = (float)t.inv_h_r;
    t.rcf = (float)rc;
    t.rc2f = (float)(rc * rc);
    t.rmin2f = (float)(NE_RMIN * NE_RMIN);
    t.inv_h_rhof = (float)t.inv_h_rho;

    // ---- what must start at zero (the scratch keeps the previous call's contents)
    if (cudaMemcpyAsync(base + O_REP, &R, sizeof(RepDev), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(base + O_TILEREP, tile_rep, sizeof(int) * R.ntile, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(base + O_SMALL, 0, 256, st) != cudaSuccess ||
        cudaMemsetAsync(base + O_TOT, 0, sizeof(double) * NTOT, st) != cudaSuccess)
        return NE_ECUDA;

    // ---- tables, list, pass 1, pass 2, export (the kernels of ne_eam_energy_forces)
    double* theta = (double*)(base + O_THETA);
    k_theta<<<(nk + 255) / 256, 256, 0, st>>>(*eam, theta);
    ne::launch_tables(theta, nk, rc, eam->rho_max, (float4*)(base + O_PF32), (ned4*)(base + O_PF64),
                      (float4*)(base + O_F32), (ned4*)(base + O_F64), st);
    const bool mixed = prec == NE_MIXED;
    Sched S{};
    S.kind = SCHED_FIXED;
    ne::launch_nl_build(B, 1, 0, st);
    if (mixed) ne::launch_wrap32(B, st);
    ne::launch_density(B, mixed, step_ctr, 0, st);
    ne::launch_force(B, S, mixed, step_ctr, 0, 0, st);
    ne::launch_export(B, mixed, f_dev, e_dev, st);
    if (cudaGetLastError() != cudaSuccess) return NE_ECUDA;
    int bits = 0;
    if (cudaMemcpyAsync(&bits, B.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return NE_ECUDA;
    if (bits & ST_ENAN) return NE_ENAN;
    if (bits & ST_ERANGE) return NE_ERANGE;
    if (bits & ST_ENEIGH) return NE_ENEIGH;
    return NE_OK;
}
