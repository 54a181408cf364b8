// ne_cluster.cu -- persistent batched runner for crystals (mixed precision):
// one thread-block cluster per replica runs a whole step range of the
// four-phase switching schedule in one launch.
//
// Per replica, the cluster's C CTAs each own up to 256 atoms.  Every CTA
// keeps, in shared memory, the displacements from the lattice sites
// u_j = x_j - r0_j (FP32) and F'(rho_j) of all atoms of the replica; each CTA
// broadcasts its atoms' values to the other CTAs through distributed shared
// memory.  Neighbours come from a lattice stencil: for the basis site b of
// atom i, the sites j with |r0_j - r0_i| < r_c + 2D sorted by that distance,
// so r_ij = (r0_j - r0_i) + u_j - u_i needs no minimum image and no list, and
// a pair can lie inside r_c only if |r0_j - r0_i| < r_c + |u_i| + max_j |u_j|
// -- the loop over the stencil stops there.  D (<= 2 A) is the largest
// displacement from a site the stencil covers; a replica whose atoms stray
// further is reported (NE_ERANGE) -- the crystal has melted.
//
// One MD step (same arithmetic order as the multi-kernel path):
//   [cluster barrier]  pass 1: rho, F(rho), F'(rho), short list in smem,
//                      F' broadcast
//   [cluster barrier]  pass 2: forces, pair energy, this step's normals;
//                      CTA partial sums to rank 0
//   [cluster barrier]  replica totals (fixed order); work increment (rank 0);
//                      closing and opening half kicks, drift, OU, drift;
//                      new u broadcast; partial sums for the next step
// The barriers are barrier.cluster arrive/wait (hardware; every CTA of a
// cluster is co-scheduled), so no thread spins on memory.
//
// Precision: pair distances, splines, forces, velocities and the OU update in
// FP32; positions x (registers, FP64), rho accumulation (FP32 chunks of 8 into
// FP64), the work W and all replica sums in FP64 (CTA sums as FP32
// double-float pairs, summed across the cluster in FP64).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "ne_internal.cuh"
#include "ne_cluster.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int THREADS = 512;
constexpr int TPA = 2;
constexpr int SLOTS = THREADS / TPA;  // atoms per CTA
constexpr int SLMAX = 96;             // short-list entries per atom
constexpr int NWARP = THREADS / 32;

// partial sums
enum { A_UEMB = 0, A_UPAIR, A_FX, A_FY, A_FZ, A_XX, A_XY, A_XZ, NA_ };
enum { B_UE = 0, B_UX, B_UY, B_UZ, B_U2, B_KE, B_UMAX, NB_ };

struct dfl {
    float hi, lo;
};

// Error-free sum of two double-float values (TwoSum + renormalisation).
__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    float s = a.hi + b.hi;
    float bp = s - a.hi;
    float e = (a.hi - (s - bp)) + (b.hi - bp);
    e += a.lo + b.lo;
    float h = s + e;
    return {h, e - (h - s)};
}

template <int NV>
__device__ __forceinline__ void warp_df_sum(dfl (&v)[NV])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            dfl w = {__shfl_xor_sync(0xffffffffu, v[q].hi, o), __shfl_xor_sync(0xffffffffu, v[q].lo, o)};
            v[q] = df_add(v[q], w);
        }
}

// CTA sum of NV double-float values -> doubles (thread 0 returns them in out).
template <int NV>
__device__ void cta_sum(dfl (&v)[NV], float* s_red, double* out)
{
    warp_df_sum<NV>(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int q = 0; q < NV; ++q) {
            s_red[(w * NV + q) * 2] = v[q].hi;
            s_red[(w * NV + q) * 2 + 1] = v[q].lo;
        }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < NV; ++q) {
            double acc = 0.0;
            for (int ww = 0; ww < NWARP; ++ww)
                acc += (double)s_red[(ww * NV + q) * 2] + (double)s_red[(ww * NV + q) * 2 + 1];
            out[q] = acc;
        }
    __syncthreads();
}

__device__ __forceinline__ float cta_max(float v, float* s_red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) s_red[w] = v;
    __syncthreads();
    float m = 0.f;
    for (int ww = 0; ww < NWARP; ++ww) m = fmaxf(m, s_red[ww]);
    __syncthreads();
    return m;
}

struct Site {
    int ix, iy, iz, b;
};

__device__ __forceinline__ Site site_of(const XRep& R, int a)
{
    Site s;
    s.b = a % R.nb;
    int c = a / R.nb;
    s.iz = c % R.nz;
    c /= R.nz;
    s.iy = c % R.ny;
    s.ix = c / R.ny;
    return s;
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Atom index of stencil entry `code` seen from site s.
__device__ __forceinline__ int neighbour(const XRep& R, const Site& s, int code)
{
    const int dx = (code & 255) - 128, dy = ((code >> 8) & 255) - 128, dz = ((code >> 16) & 255) - 128;
    const int b2 = (code >> 24) & 255;
    const int jx = wrapi(s.ix + dx, R.nx), jy = wrapi(s.iy + dy, R.ny), jz = wrapi(s.iz + dz, R.nz);
    return ((jx * R.ny + jy) * R.nz + jz) * R.nb + b2;
}

__device__ __forceinline__ float blendf(int path, float lam, float F0, float FE)
{
    return path == 0 ? (1.f - lam) * F0 + lam * FE : lam * F0;
}

__global__ void __launch_bounds__(THREADS, 2)
    k_cluster(const XRep* __restrict__ reps, const float4* __restrict__ st_vec, const int* __restrict__ st_code,
              double* __restrict__ xg, double* __restrict__ vg, double* __restrict__ Wg, int* status, Sched S,
              long long s_begin, long long n_steps, Tables tab, unsigned long long* work)
{
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int rep = blockIdx.x / C;
    const XRep& R = reps[rep];
    const int n = R.n;
    const int nst = R.st_cnt;
    const int A_c = (n + C - 1) / C;

    // ---- shared memory
    float4* s_u = (float4*)smem;                                  // [n] (u, F')
    float4* s_sv = s_u + n;                                       // [nb * nst]
    int* s_sc = (int*)(s_sv + R.nb * nst);                        // [nb * nst]
    unsigned short* s_sl = (unsigned short*)(s_sc + R.nb * nst);  // [SLOTS][SLMAX]
    double* s_slotA = (double*)(((size_t)(s_sl + SLOTS * SLMAX) + 15) & ~(size_t)15);  // [16][NA_]
    double* s_slotB = s_slotA + 16 * NA_;                         // [2][16][NB_]
    double* s_tot = s_slotB + 2 * 16 * NB_;                       // [NA_ + NB_]
    double* s_cta = s_tot + NA_ + NB_;                            // [8]
    float* s_red = (float*)(s_cta + 8);                           // [NWARP][8][2]
    float* s_misc = s_red + NWARP * 16;                           // [4]

    for (int q = threadIdx.x; q < R.nb * nst; q += THREADS) {
        s_sv[q] = st_vec[R.st_off + q];
        s_sc[q] = st_code[R.st_off + q];
    }

    const int slot = threadIdx.x / TPA, lane = threadIdx.x % TPA;
    const int a = rank * A_c + slot;
    const bool valid = slot < A_c && a < n;
    const bool owner = valid && lane == 0;
    const int ai = valid ? a : 0;
    const Site site = site_of(R, ai);
    const int stb = site.b * nst;
    cluster.sync();  // every CTA of the cluster has started: distributed shared memory is usable

    // ---- state of the owned atom: x FP64 (registers), v FP32
    double x[3] = {0, 0, 0}, r0[3];
    float v[3] = {0, 0, 0}, u[3] = {0, 0, 0};
    r0[0] = R.a * (site.ix + R.basis[site.b][0]);
    r0[1] = R.a * (site.iy + R.basis[site.b][1]);
    r0[2] = R.a * (site.iz + R.basis[site.b][2]);
    const size_t gi = (size_t)(R.off + ai) * 3;
    int bad = 0;
    if (owner) {
        for (int c = 0; c < 3; ++c) {
            x[c] = xg[gi + c];
            v[c] = (float)vg[gi + c];
            u[c] = (float)(x[c] - r0[c]);
        }
        const float4 uv = make_float4(u[0], u[1], u[2], 0.f);
        for (int r = 0; r < C; ++r) cluster.map_shared_rank(s_u, r)[a] = uv;
    }
    // partials for the first step
    {
        dfl pb[NB_ - 1] = {};
        float umax = 0.f;
        if (owner) {
            const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            pb[B_UE] = {0.5f * R.kf * u2, 0.f};
            pb[B_UX] = {u[0], 0.f};
            pb[B_UY] = {u[1], 0.f};
            pb[B_UZ] = {u[2], 0.f};
            pb[B_U2] = {u2, 0.f};
            pb[B_KE] = {0.5f * R.mf * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]), 0.f};
            umax = sqrtf(u2);
        }
        cta_sum<NB_ - 1>(pb, s_red, s_cta);
        umax = cta_max(umax, s_red);
        if (threadIdx.x == 0) {
            double* dst = cluster.map_shared_rank(s_slotB, 0) + ((s_begin & 1) * 16 + rank) * NB_;
            for (int q = 0; q < NB_ - 1; ++q) dst[q] = s_cta[q];
            dst[B_UMAX] = umax;
        }
    }

    unsigned long long n_cand = 0, n_pair = 0;  // work counters (stencil entries visited, pairs < r_c)
    const float rc = (float)tab.r_c, rc2 = tab.rc2f, rmin2 = tab.rmin2f, inv_h = tab.inv_h_rf;
    const int nk = tab.nk;
    const float dt = (float)S.dt;
    float F0[3] = {0, 0, 0}, xi[3] = {0, 0, 0};

    for (long long it = 0; it <= n_steps; ++it) {
        const long long s = s_begin + it;
        const bool fin = it == n_steps;
        cluster.sync();  // u of step s visible everywhere
        if (threadIdx.x == 0) {
            const double* sb = cluster.map_shared_rank(s_slotB, 0) + (s & 1) * 16 * NB_;
            double um = 0.0;
            for (int r = 0; r < C; ++r) um = fmax(um, sb[r * NB_ + B_UMAX]);
            s_misc[0] = (float)um;
            if (um > (double)R.D) ne_set_status(status, ST_ERANGE);
        }
        __syncthreads();
        const float umax = s_misc[0];

        // ---------------- pass 1: density, F(rho), F'(rho), short list
        const float4 ui = s_u[ai];
        float emb = 0.f;
        int m = 0;
        {
            const float cut = rc + sqrtf(ui.x * ui.x + ui.y * ui.y + ui.z * ui.z) + umax;
            double rho = 0.0;
            float chunk = 0.f;
            int nchunk = 0;
            if (valid) {
                for (int k = lane; k < nst; k += TPA) {
                    const float4 e = s_sv[stb + k];
                    if (e.w >= cut) break;
                    const int j = neighbour(R, site, s_sc[stb + k]);
                    const float4 uj = s_u[j];
                    const float dx = e.x + uj.x - ui.x, dy = e.y + uj.y - ui.y, dz = e.z + uj.z - ui.z;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    ++n_cand;
                    if (r2 < rc2) {
                        ++n_pair;
                        if (r2 < rmin2) bad |= ST_ERANGE;
                        const float r = sqrtf(r2);
                        const float t = r * inv_h;
                        const int kk = min(max((int)t, 0), nk - 2);
                        const float w = t - (float)kk;
                        const float4 c = __ldg(&tab.pf32[2 * kk + 1]);
                        chunk += c.x + w * (c.y + w * (c.z + w * c.w));
                        if (++nchunk == 8) {
                            rho += (double)chunk;
                            chunk = 0.f;
                            nchunk = 0;
                        }
                        if (m < SLMAX / TPA)
                            s_sl[slot * SLMAX + m * TPA + lane] = (unsigned short)k;
                        else
                            bad |= ST_ENEIGH;
                        ++m;
                    }
                }
                m = min(m, SLMAX / TPA);
            }
            rho += (double)chunk;
            for (int o = TPA >> 1; o > 0; o >>= 1) rho += __shfl_xor_sync(0xffffffffu, rho, o);
            if (owner) {
                if (!(rho < tab.rho_max)) bad |= ST_ERANGE;
                const double t = rho * tab.inv_h_rho;
                const int kk = min(max((int)t, 0), nk - 2);
                const float w = (float)(t - kk);
                const float4 c = __ldg(&tab.F32[kk]);
                emb = c.x + w * (c.y + w * (c.z + w * c.w));
                const float dF = (c.y + w * (2.f * c.z + 3.f * w * c.w)) * tab.inv_h_rhof;
                for (int r = 0; r < C; ++r) cluster.map_shared_rank(s_u, r)[a].w = dF;
                if (!isfinite(emb)) bad |= ST_ENAN;
            }
        }
        cluster.sync();  // F' visible everywhere

        // ---------------- pass 2: forces, pair energy, noise
        {
            float fx = 0.f, fy = 0.f, fz = 0.f, ep = 0.f;
            if (valid) {
                const float dFi = s_u[ai].w;
                for (int q = 0; q < m; ++q) {
                    const int k = s_sl[slot * SLMAX + q * TPA + lane];
                    const float4 e = s_sv[stb + k];
                    const int j = neighbour(R, site, s_sc[stb + k]);
                    const float4 uj = s_u[j];
                    const float dx = e.x + uj.x - ui.x, dy = e.y + uj.y - ui.y, dz = e.z + uj.z - ui.z;
                    const float r = sqrtf(dx * dx + dy * dy + dz * dz);
                    const float ir = 1.f / r;
                    const float t = r * inv_h;
                    const int kk = min(max((int)t, 0), nk - 2);
                    const float w = t - (float)kk;
                    const float4 c = __ldg(&tab.pf32[2 * kk]);
                    const float4 g = __ldg(&tab.pf32[2 * kk + 1]);
                    const float phi = c.x + w * (c.y + w * (c.z + w * c.w));
                    const float dphi = (c.y + w * (2.f * c.z + 3.f * w * c.w)) * inv_h;
                    const float df = (g.y + w * (2.f * g.z + 3.f * w * g.w)) * inv_h;
                    const float sc = (dphi + (dFi + uj.w) * df) * ir;
                    fx += sc * dx;
                    fy += sc * dy;
                    fz += sc * dz;
                    ep += 0.5f * phi;
                }
            }
            for (int o = TPA >> 1; o > 0; o >>= 1) {
                fx += __shfl_xor_sync(0xffffffffu, fx, o);
                fy += __shfl_xor_sync(0xffffffffu, fy, o);
                fz += __shfl_xor_sync(0xffffffffu, fz, o);
                ep += __shfl_xor_sync(0xffffffffu, ep, o);
            }
            dfl pa[NA_] = {};
            if (owner) {
                F0[0] = fx;
                F0[1] = fy;
                F0[2] = fz;
                if (!fin) {
                    ne_normals32(ne_philox_block(R.seed, R.replica, (unsigned)S.stream, (unsigned)a,
                                                 (unsigned long long)s),
                                 xi);
                }
                pa[A_UEMB] = {emb, 0.f};
                pa[A_UPAIR] = {ep, 0.f};
                pa[A_FX] = {fx, 0.f};
                pa[A_FY] = {fy, 0.f};
                pa[A_FZ] = {fz, 0.f};
                pa[A_XX] = {xi[0], 0.f};
                pa[A_XY] = {xi[1], 0.f};
                pa[A_XZ] = {xi[2], 0.f};
            }
            cta_sum<NA_>(pa, s_red, s_cta);
            if (threadIdx.x == 0) {
                double* dst = cluster.map_shared_rank(s_slotA, 0) + rank * NA_;
                for (int q = 0; q < NA_; ++q) dst[q] = s_cta[q];
            }
        }
        cluster.sync();  // partial sums of step s complete

        // ---------------- replica totals (fixed order over the cluster's CTAs)
        if (threadIdx.x < NA_ + NB_ - 1) {
            const int q = threadIdx.x;
            double acc = 0.0;
            if (q < NA_) {
                const double* sa = cluster.map_shared_rank(s_slotA, 0);
                for (int r = 0; r < C; ++r) acc += sa[r * NA_ + q];
            } else {
                const double* sb = cluster.map_shared_rank(s_slotB, 0) + (s & 1) * 16 * NB_;
                for (int r = 0; r < C; ++r) acc += sb[r * NB_ + (q - NA_)];
            }
            s_tot[q] = acc;
        }
        __syncthreads();
        const double lam_s = ne_sched_lambda(S, s), lam_n = ne_sched_lambda(S, s + 1);
        if (!fin && rank == 0 && threadIdx.x == 0) {
            const double U0 = s_tot[A_UEMB] + s_tot[A_UPAIR];
            const double g = S.path == 0 ? U0 - s_tot[NA_ + B_UE] : U0;
            int wslot = -1;
            if (s >= S.t_eq && s < S.t_eq + S.t_s) wslot = 0;
            else if (s >= 2 * S.t_eq + S.t_s && s < 2 * S.t_eq + 2 * S.t_s) wslot = 1;
            if (wslot >= 0) Wg[2 * rep + wslot] += (lam_n - lam_s) * g;
        }

        // ---------------- fused step of the owned atom
        {
            dfl pb[NB_ - 1] = {};
            float un = 0.f;
            if (owner) {
                const float invN = 1.f / (float)n;
                float mF0[3], mFE[3], mxi[3];
                for (int c = 0; c < 3; ++c) {
                    mF0[c] = S.fix_cm ? (float)(s_tot[A_FX + c] * invN) : 0.f;
                    mFE[c] = S.fix_cm ? (float)(-R.k * s_tot[NA_ + B_UX + c] * invN) : 0.f;
                    mxi[c] = S.fix_cm ? (float)(s_tot[A_XX + c] * invN) : 0.f;
                }
                const float ls = (float)lam_s, ln = (float)lam_n;
                if (it > 0)
                    for (int c = 0; c < 3; ++c)
                        v[c] += R.hdt_mf * blendf(S.path, ls, F0[c] - mF0[c], -R.kf * u[c] - mFE[c]);
                if (!fin) {
                    for (int c = 0; c < 3; ++c) {
                        v[c] += R.hdt_mf * blendf(S.path, ln, F0[c] - mF0[c], -R.kf * u[c] - mFE[c]);
                        const float v1 = v[c];
                        v[c] = R.c1f * v[c] + R.c2f * (xi[c] - mxi[c]);
                        x[c] += (double)(0.5f * dt * (v1 + v[c]));
                        u[c] = (float)(x[c] - r0[c]);
                    }
                    const float4 uv = make_float4(u[0], u[1], u[2], 0.f);
                    for (int r = 0; r < C; ++r) cluster.map_shared_rank(s_u, r)[a] = uv;
                }
                const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                pb[B_UE] = {0.5f * R.kf * u2, 0.f};
                pb[B_UX] = {u[0], 0.f};
                pb[B_UY] = {u[1], 0.f};
                pb[B_UZ] = {u[2], 0.f};
                pb[B_U2] = {u2, 0.f};
                pb[B_KE] = {0.5f * R.mf * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]), 0.f};
                un = sqrtf(u2);
                for (int c = 0; c < 3; ++c)
                    if (!isfinite(x[c]) || !isfinite(v[c])) bad |= ST_ENAN;
            }
            if (!fin) {
                cta_sum<NB_ - 1>(pb, s_red, s_cta);
                un = cta_max(un, s_red);
                if (threadIdx.x == 0) {
                    double* dst = cluster.map_shared_rank(s_slotB, 0) + (((s + 1) & 1) * 16 + rank) * NB_;
                    for (int q = 0; q < NB_ - 1; ++q) dst[q] = s_cta[q];
                    dst[B_UMAX] = un;
                }
            }
        }
    }
    if (owner)
        for (int c = 0; c < 3; ++c) {
            xg[gi + c] = x[c];
            vg[gi + c] = (double)v[c];
        }
    if (bad) ne_set_status(status, bad);
    if (work) {
        for (int o = 16; o > 0; o >>= 1) {
            n_cand += __shfl_xor_sync(0xffffffffu, n_cand, o);
            n_pair += __shfl_xor_sync(0xffffffffu, n_pair, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&work[0], n_cand);
            atomicAdd(&work[1], n_pair);
        }
    }
    cluster.sync();  // no CTA leaves while others may still touch its shared memory
}

}  // namespace

namespace ne {

size_t cluster_smem_bytes(int n_max, int nb_nst_max)
{
    size_t b = sizeof(float4) * (size_t)n_max + (sizeof(float4) + sizeof(int)) * (size_t)nb_nst_max +
               sizeof(unsigned short) * SLOTS * SLMAX;
    b = (b + 15) & ~(size_t)15;
    b += sizeof(double) * (16 * NA_ + 2 * 16 * NB_ + NA_ + NB_ + 8) + sizeof(float) * (NWARP * 16 + 4);
    return b;
}

int cluster_atoms_per_cta() { return SLOTS; }

cudaError_t launch_cluster(const XRep* reps, int n_rep, int C, size_t smem, const float4* st_vec,
                           const int* st_code, double* x, double* v, double* W, int* status, const Sched& S,
                           long long s_begin, long long n_steps, const Tables& tab, unsigned long long* work,
                           cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(k_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (C > 8) {
        e = cudaFuncSetAttribute(k_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_rep * C, 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_cluster, reps, st_vec, st_code, x, v, W, status, S, s_begin, n_steps, tab,
                              work);
}

}  // namespace ne
