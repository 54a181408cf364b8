// ne_internal.cuh -- device-side layouts and helpers shared by the kernels of
// libne.so (not part of the public ABI; see include/ne.h).
//
// Data layout in HBM (all replicas of a batch concatenated, atom-major):
//   x, v, x0            double [N][3]   caller-owned, unwrapped positions
//   pos32               float4 [N]      FP32 copy of x wrapped into the box
//   posF                float4 [N]      (x, y, z, F'(rho)) written by pass 1
//   pbuild              float4 [N]      wrapped positions at the last list build
//   f32 / f64           EAM forces, float4 [N] (mixed) or double [N][3]
//   dF64                double [N]      F'(rho) (FP64 path)
//   xi32 / xi64         Langevin normals of the current step, [N][3]
//   nbr, ncnt           candidate list within r_c + skin, int, lane-interleaved:
//                       entry k of atom i at ((k / TPA) * N + i) * TPA + k % TPA
//   sl, scnt            per-step short list (r < r_c) in the same layout, one
//                       count per (atom, lane)
//   partA / partB       per-tile FP64 partial sums (pass 1+2 / step kernel)
//   tot                 per-replica totals formed by the last tile of pass 2
// A tile is NE_TILE consecutive atoms of one replica; tiles never straddle
// replicas, so every per-replica sum is a fixed-order sum of tile partials.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// 32-byte aligned quadruple of doubles (one spline interval in FP64)
struct __align__(32) ned4 {
    double x, y, z, w;
};

#define NE_TILE 64
#define NE_MAX_SPECIES_DEV 8  // species per replica (NE_MAX_SPECIES of the public header)
#define NE_NMAX 256   // candidate neighbours per atom (r < r_c + skin)
#define NE_SMAX 128   // neighbours per atom inside r_c
#define NE_RMIN 0.2   // A: shorter pair distances are reported as NE_ERANGE (atoms may overlap at lambda -> 1)

// device status bits
enum { ST_ERANGE = 1, ST_ENEIGH = 2, ST_ENAN = 4, ST_ETIMEOUT = 8, ST_EINVAL = 16 };

// Philox stream ids (low 4 bits of the 4th counter word)
enum { STREAM_FL = 0, STREAM_INITV = 1, STREAM_RS = 2, STREAM_MSD = 3, STREAM_STEP = 4, STREAM_BARO = 5 };

// tile partials of pass 1 / pass 2 (at x_k)
enum { PA_UEMB = 0, PA_UPAIR, PA_F0X, PA_F0Y, PA_F0Z, PA_XIX, PA_XIY, PA_XIZ, PA_VIR, PA_VXX, PA_VYY, PA_VZZ, NPA };
// tile partials of the step kernel (at x_{k+1}; KE of the completed velocity)
enum { PB_UE = 0, PB_UX, PB_UY, PB_UZ, PB_U2, PB_KE, NPB };
// per-replica totals
enum { TOT_UEMB = 0, TOT_UPAIR, TOT_F0X, TOT_F0Y, TOT_F0Z, TOT_XIX, TOT_XIY, TOT_XIZ, TOT_VIR,
       TOT_VXX, TOT_VYY, TOT_VZZ, TOT_UE, TOT_UX, TOT_UY, TOT_UZ, TOT_U2, TOT_KE, NTOT };
static_assert((int)TOT_VIR == (int)PA_VIR && (int)TOT_UE == (int)NPA, "totals: pass-2 partials first, then the step's");

struct RepDev {
    double L[3], invL[3];
    double k;        // Einstein spring
    double c1, c2;   // Ornstein-Uhlenbeck coefficients
    double hdt_m;    // dt / (2 m)
    double kT;
    double m;
    double rlist2;   // (r_c + skin)^2
    float half_skin2;
    int off, n, tile0, ntile;
    int nc[3];       // cells per axis; 0 = all pairs
    int cell_off;
    int dof;
    unsigned long long seed;
    unsigned replica;
    int npt;         // barostat (RS path): 1 isotropic, 2 one equation per box edge
    double P0, mp;   // target pressure, mobility beta_T / tau_p
    // Several species (Sec. V): nsp = 0 -- every atom has m and k above;
    // nsp >= 2 -- atom a has species sp[a] (validated on the host) with mass
    // ms, spring ks, noise amplitude c2s and half-step factor hdts of its
    // species; M is the replica's total mass.  With species tables the
    // step kernel's sum PB_UX.. holds sum_j k_j u_j and pass 2's PA_XIX..
    // holds sum_j m_j c2_j xi_j: the sums the mass-weighted centre-of-mass
    // constraint needs.
    int nsp;
    const unsigned char* sp;
    double M;
    double ms[NE_MAX_SPECIES_DEV], ks[NE_MAX_SPECIES_DEV], c2s[NE_MAX_SPECIES_DEV], hdts[NE_MAX_SPECIES_DEV];
};

// Schedule of a run, shared by the replicas of one launch.
enum { SCHED_SWITCH = 0, SCHED_FIXED = 1 };
struct Sched {
    long long t_eq, t_s;
    double lambda_f;
    double lam_a, lam_b;   // SCHED_FIXED: lambda before / after the jump
    long long s0;          // SCHED_FIXED: step of the jump
    double dt;
    int kind, path, fn, stream, fix_cm;
};

struct Tables {
    // phi and f interleaved per interval: [nk-1][2] (phi, f), cubic in u
    const float4* pf32;
    const ned4* pf64;
    const float4* F32;     // embedding, [nk-1]
    const ned4* F64;
    int nk;
    double h_r, inv_h_r, h_rho, inv_h_rho;
    double r_c, rho_max;
    float inv_h_rf, rcf, rc2f, rmin2f, inv_h_rhof;
};

struct DevBatch {
    int n_rep, n_tot, n_tiles, tpa;
    const RepDev* rep;
    const int* tile_rep;
    double* x;
    double* v;
    const double* x0;
    float4* pos32;
    float4* posF;
    float4* pbuild;
    float4* f32;
    double* f64;
    double* dF64;
    double* rho;       // nullable: per-atom density output
    float* xi32;
    double* xi64;
    int* nbr;
    int* ncnt;
    int* sl;
    int* scnt;
    int* cellof;
    int* sorted;
    int* cstart;
    int* cfill;
    double* partA;
    double* partB;
    double* tot;
    unsigned* tile_done;
    double* W;         // [n_rep][2]
    double* Wcum;      // nullable, [n_rep][2][t_s + 1]
    double* trace;     // nullable, [rows][8], single replica
    int trace_stride, trace_rows;
    int* flags;        // [n_rep] list rebuild requested (set by the step kernel)
    int* building;     // [n_rep] rebuild in progress this step
    unsigned long long* rebuilds;  // count of replica list builds
    int* status;
    Tables tab;
    int npt_any;       // some replica has the barostat on
    int species_any;   // every replica has species tables (msd sampling per species)
};

// ------------------------------------------------------------------ lambda
// Sec. III.B: lambda = tau (function 1) or tau^5 (70 tau^4 - 315 tau^3 +
// 540 tau^2 - 420 tau + 126) (function 2); Sec. III.C: 1/(1 + tau(1/lf - 1)).
__host__ __device__ inline double ne_lambda_fl(int fn, double t)
{
    if (fn == 1) return t;
    double t2 = t * t;
    return t2 * t2 * t * (126.0 + t * (-420.0 + t * (540.0 + t * (-315.0 + t * 70.0))));
}

__host__ __device__ inline double ne_lambda_rs(double lf, double t)
{
    return 1.0 / (1.0 + t * (1.0 / lf - 1.0));
}

// Lambda in force at the start of global step s of the four-phase schedule.
__host__ __device__ inline double ne_sched_lambda(const Sched& S, long long s)
{
    if (S.kind == SCHED_FIXED) return s <= S.s0 ? S.lam_a : S.lam_b;
    const bool fl = S.path == 0;
    const double li = fl ? 0.0 : 1.0, lf = fl ? 1.0 : S.lambda_f;
    if (s <= S.t_eq) return li;
    long long s1 = s - S.t_eq;
    if (s1 <= S.t_s) {
        double tau = (double)s1 / (double)S.t_s;
        return fl ? ne_lambda_fl(S.fn, tau) : ne_lambda_rs(S.lambda_f, tau);
    }
    long long s2 = s1 - S.t_s;
    if (s2 <= S.t_eq) return lf;
    long long s3 = s2 - S.t_eq;
    if (s3 <= S.t_s) {
        double tau = (double)s3 / (double)S.t_s;
        return fl ? 1.0 - ne_lambda_fl(S.fn, tau) : ne_lambda_rs(S.lambda_f, 1.0 - tau);
    }
    return li;
}

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds, each two
// 32x32 -> 64-bit products mixed into the other words with the round key;
// the key advances by the Weyl increments between rounds.
__device__ __forceinline__ uint4 ne_philox(uint4 c, uint2 k)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += W0;
        k.y += W1;
    }
    return c;
}

__device__ __forceinline__ uint4 ne_philox_block(unsigned long long seed, unsigned replica,
                                                 unsigned stream, unsigned atom,
                                                 unsigned long long step)
{
    uint4 c = make_uint4(atom, (uint32_t)step, (uint32_t)(step >> 32), (replica << 4) | (stream & 15u));
    uint2 k = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    return ne_philox(c, k);
}

// Three standard normals from one Philox block by Box-Muller, uniforms
// (w + 1/2) 2^-32; the fourth normal is not used.
__device__ __forceinline__ void ne_normals64(uint4 w, double z[3])
{
    const double s = 2.3283064365386963e-10;  // 2^-32
    double u0 = ((double)w.x + 0.5) * s, u1 = ((double)w.y + 0.5) * s;
    double u2 = ((double)w.z + 0.5) * s, u3 = ((double)w.w + 0.5) * s;
    double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
    double s1, c1, s3, c3;
    sincospi(2.0 * u1, &s1, &c1);
    sincospi(2.0 * u3, &s3, &c3);
    z[0] = r0 * c1;
    z[1] = r0 * s1;
    z[2] = r1 * c3;
}

// FP32 variant: the top 24 bits of each word give u = (w>>8 + 1/2) 2^-24.
__device__ __forceinline__ void ne_normals32(uint4 w, float z[3])
{
    const float s = 5.9604644775390625e-8f;  // 2^-24
    float u0 = ((float)(w.x >> 8) + 0.5f) * s, u1 = ((float)(w.y >> 8) + 0.5f) * s;
    float u2 = ((float)(w.z >> 8) + 0.5f) * s, u3 = ((float)(w.w >> 8) + 0.5f) * s;
    float r0 = sqrtf(-2.0f * logf(u0)), r1 = sqrtf(-2.0f * logf(u2));
    float s1, c1, s3, c3;
    sincospif(2.0f * u1, &s1, &c1);
    sincospif(2.0f * u3, &s3, &c3);
    z[0] = r0 * c1;
    z[1] = r0 * s1;
    z[2] = r1 * c3;
}

// ------------------------------------------------------------------ misc
__device__ __forceinline__ int ne_nbr_index(int k, int i, int n_tot, int tpa)
{
    return ((k / tpa) * n_tot + i) * tpa + (k % tpa);
}

// double-float (hi + lo, |lo| <= ulp(hi) / 2) sum of two such numbers from
// FP32 operations (TwoSum of the high parts, the low parts added to its error)
struct dff {
    float hi, lo;
};

__device__ __forceinline__ dff dff_add(dff a, dff b)
{
    const float s = a.hi + b.hi, bp = s - a.hi;
    float e = (a.hi - (s - bp)) + (b.hi - bp);
    e += a.lo + b.lo;
    const float h = s + e;
    return {h, e - (h - s)};
}

// sum over the warp of a double-float (fixed xor tree: every lane gets it)
__device__ __forceinline__ dff dff_warp_sum(dff v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = dff_add(v, {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
    return v;
}

// Sum of quantity q over tiles [t0, t0 + nt) of a tile-partials array (nq
// values a tile), by one warp: lane l adds tiles t0 + l, t0 + l + 32, ...
// in order, then a fixed xor-shuffle tree; every lane returns the total, and
// the order depends only on nt, never on scheduling.  Called by all 32 lanes.
__device__ __forceinline__ double ne_warp_tile_sum(const double* part, int nq, int q, int t0, int nt)
{
    const int l = threadIdx.x & 31;
    double acc = 0.0;
    for (int t = l; t < nt; t += 32) acc += __ldcg(&part[(size_t)(t0 + t) * nq + q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

__device__ __forceinline__ void ne_set_status(int* status, int bits)
{
    atomicOr(status, bits);
}

// Fixed-order block sum of NV doubles per thread into out[NV] (thread 0).
template <int NV>
__device__ inline void ne_block_sum(double (&val)[NV], double* out, double* scratch)
{
    // scratch: blockDim.x * NV doubles
    const int t = threadIdx.x;
    for (int q = 0; q < NV; ++q) scratch[q * blockDim.x + t] = val[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int q = 0; q < NV; ++q) scratch[q * blockDim.x + t] += scratch[q * blockDim.x + t + w];
        __syncthreads();
    }
    if (t == 0)
        for (int q = 0; q < NV; ++q) out[q] = scratch[q * blockDim.x];
    __syncthreads();
}

// Launch helpers (defined in the kernel translation units).
namespace ne {
void launch_tables(const double* theta, int nk, double r_c, double rho_max, float4* pf32,
                   ned4* pf64, float4* F32, ned4* F64, cudaStream_t st);
void launch_nl_build(const DevBatch& B, int force, int from_sites, cudaStream_t st);
void launch_density(const DevBatch& B, bool mixed, const long long* step_base, int j,
                    cudaStream_t st);
void launch_force(const DevBatch& B, const Sched& S, bool mixed, const long long* step_base,
                  int j, int want_noise, cudaStream_t st);
void launch_step(const DevBatch& B, const Sched& S, bool mixed, const long long* step_base,
                 int j, int do_close, int do_open, cudaStream_t st);
void launch_prep(const DevBatch& B, const Sched& S, bool mixed, const long long* step_base,
                 cudaStream_t st);
void launch_advance(long long* step_base, long long by, cudaStream_t st);
void launch_wrap32(const DevBatch& B, cudaStream_t st);
void launch_noise(unsigned long long seed, unsigned replica, int stream, long long step, int n, int mixed,
                  double* z, cudaStream_t st);
void launch_scale(double* p, int n, double s, cudaStream_t st);
void launch_init_velocities(const DevBatch& B, int fix_cm, cudaStream_t st);
void launch_spring(const double* x, const double* x0, int n, double k, double* f, double* e,
                   double* scratch, cudaStream_t st);
void launch_export(const DevBatch& B, bool mixed, double* f_out, double* e_out, cudaStream_t st);
void launch_msd_sample(const DevBatch& B, double* acc, cudaStream_t st);
// gE, or with gw != nullptr the per-step weight gw[*ctr + j - s_off] read on
// the device (runs replayed from graphs); set_attr: set the kernel's shared-
// memory attribute (not inside a stream capture)
size_t backward_block_bytes(int nk);  // one mixed backward block's bins (device and shared memory)
size_t backward_bins_bytes(int nk, int n_blocks);  // the whole bins buffer: F's (zeroed once), then the blocks'
bool backward_fits(int nk);           // those bins fit one block's shared memory
void launch_backward(const DevBatch& B, bool mixed, double gE, double* gx, double* gtheta,
                     float* bins, int n_bin_blocks, bool accumulate, cudaStream_t st,
                     const double* gw = nullptr, const long long* ctr = nullptr, int j = 0,
                     long long s_off = 0, bool set_attr = true);
int backward_bin_blocks(const DevBatch& B);
cudaError_t prepare_backward(const DevBatch& B);  // the mixed backward kernel's shared-memory attribute
void launch_virial(const DevBatch& B, double* out, cudaStream_t st);
void launch_npt_box(const DevBatch& B, const Sched& S, const long long* step_base, int j, cudaStream_t st);
}  // namespace ne
