// ne_brick.cu -- persistent batched runner for crystals too large for one
// thread-block cluster (mixed precision): one cooperative launch in which
// every CTA owns a block of consecutive cells of one replica and the CTAs of
// a replica exchange what the cluster runner keeps in distributed shared
// memory -- the displacements u_j = x_j - r0_j and F'(rho_j) -- through global
// memory (L2) between grid barriers.
//
// The arithmetic of a step is that of the cluster runner (ne_cluster.cu):
// the same lattice stencil and scan bound, rho as a double-float, positions
// in fixed point, FP32 pair arithmetic, the work W in FP64, and the same
// Philox noise, so a replica gives the cluster runner's trajectory to the
// rounding of its replica sums (which depend on how the atoms are split over
// CTAs).  Per step:
//   replica sums of step s from the CTA partials written at the end of s-1
//   pass 1: rho, pair forces and energy, f'(r)/r of every visit to tensor memory (u_j from L2);
//           F'(rho) of the owned atoms to global memory
//   [grid barrier]
//   pass 2: embedding forces over the visits inside r_c (u_j, F'_j from L2)
//   fused step of the owned atoms; u of step s+1 to the other parity buffer;
//           CTA partials for step s+1
//   [grid barrier]
// Two grid barriers a step; u is double-buffered by step parity, so no CTA
// overwrites a u another still reads.  With the barostat (reading A23, the
// cluster runner's arithmetic) pass 2 also sums the diagonal virial; the
// CTA sums go to global memory behind a third grid barrier, after which
// every CTA of the replica forms the same scale factors (the same sums in
// the same order, the same Philox normal) before its integration.  The barrier is an arrival counter and
// a generation word in global memory; every CTA of the launch is resident at
// once (cooperative launch), and every wait is bounded: after BAR_SPIN_LIMIT
// polls a CTA records NE_ETIMEOUT, raises the abort word and leaves, and the
// others leave at their next barrier.  Loads of data other CTAs wrote use
// ld.global.cg (L2, never a stale L1 line).
//
// Threads: TPA threads per atom (8, 4, 3, 2 or 1, the largest at which the
// batch's CTAs fit the device at one CTA per SM); thread t works on slot
// t % SLOTS and takes the stencil entries k = lane + TPA q, lane = t / SLOTS,
// so the 32 threads of a warp read one stencil entry.  One thread per atom
// for the embedding and the integration.
#include <algorithm>
#include <cuda_runtime.h>

#include "ne_internal.cuh"
#include "ne_cluster.cuh"

namespace {

constexpr int BTHREADS = 768;
// TMEM scratch (as in the cluster runner): warp w owns lanes 32 (w mod 4)
// .. +31 and the QMAX columns from QMAX (w div 4): f'(r)/r of a thread's
// first QF visits (written by pass 1, read by pass 2; later visits are
// recomputed in pass 2), then the neighbour index of its first QJ visits
// (32 bits a column, written once per launch and read by pass 1: a lattice
// stencil sends atom i's k-th entry to the same atom for the whole launch).  QF and QJ depend
// on the threads per atom: at 1 a thread visits up to ~112 entries and all
// columns hold f'(r)/r
constexpr int FRB = NE_TM_BATCH;
constexpr int QMAX = NE_TM_COLS / (BTHREADS / 32 / 4) / FRB * FRB;
constexpr int NKT = 256;    // scan-bound bins of the stencil distance
constexpr int NWARP = BTHREADS / 32;
enum { P_U0 = 0, P_UE, P_UX, P_UY, P_UZ, P_XX, P_XY, P_XZ, NP_ };
constexpr int ND_ = 2, NF_ = NP_ - ND_;
constexpr int NSV = 2 * ND_ + NF_;  // floats of the sums: (hi, lo) per energy, then the FP32 sums
constexpr int NPART = NSV + 1;      // and max |u|
constexpr int T_UX = 2 * ND_ + (P_UX - ND_), T_XX = 2 * ND_ + (P_XX - ND_);
constexpr int NRED = (int)NP_ + 1;
constexpr unsigned BAR_SPIN_LIMIT = 1u << 22;  // polls, each >= 64 ns: a few seconds at most
constexpr double XSCALE = 4294967296.0;        // fixed point: 2^32 per Angstrom

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    float s = a.hi + b.hi;
    float bp = s - a.hi;
    float e = (a.hi - (s - bp)) + (b.hi - bp);
    e += a.lo + b.lo;
    float h = s + e;
    return {h, e - (h - s)};
}

__device__ __forceinline__ float fix_to_float(long long d)
{
    const int hi = (int)(d >> 16), lo = (int)(d & 0xffff);
    return fmaf((float)hi, 1.52587890625e-05f, (float)lo * 2.3283064365386963e-10f);
}

__device__ __forceinline__ float blendf(int path, float lam, float F0, float FE)
{
    return path == 0 ? (1.f - lam) * F0 + lam * FE : lam * F0;
}

__host__ __device__ inline int brick_cta_atoms(int n, int C, int nb)
{
    return (((n + C - 1) / C) + nb - 1) / nb * nb;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier over every CTA of the launch.  Returns false when a wait gave up
// (here or, through the abort word, in another CTA): the caller leaves.
__device__ bool grid_barrier(unsigned* bar, unsigned n_cta, unsigned& gen, int* status, int* abortf, int* s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();  // this CTA's global writes before its arrival
        const unsigned g = gen;
        if (atomicAdd(&bar[0], 1u) == n_cta - 1) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicExch(&bar[1], g + 1u);
        } else {
            unsigned spins = 0;
            while (ld_acquire(&bar[1]) == g) {
                if (++spins > BAR_SPIN_LIMIT || ld_acquire((const unsigned*)abortf) != 0u) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (!ok || ld_acquire((const unsigned*)abortf) != 0u) {
            ok = 0;
            ne_set_status(status, ST_ETIMEOUT);
            atomicExch(abortf, 1);
        }
        gen = g + 1u;
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// Sum of three double-float values over the 32 lanes of a warp (fixed tree).
__device__ __forceinline__ void warp_df3(dfl (&v)[3])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 3; ++q)
            v[q] = df_add(v[q], {__shfl_xor_sync(0xffffffffu, v[q].hi, o), __shfl_xor_sync(0xffffffffu, v[q].lo, o)});
}

template <int TPA, bool NPT>
__global__ void __launch_bounds__(BTHREADS, 1)
    k_brick(const XRep* __restrict__ reps, const int* __restrict__ cta_rep, const float4* __restrict__ st_vec,
            const float* __restrict__ st_dist, double* __restrict__ xg, double* __restrict__ vg,
            double* __restrict__ Wg, int* status, Sched S, long long s_begin, long long n_steps, Tables tab,
            unsigned long long* work, int k_lo, const double* __restrict__ lam_tab, double* __restrict__ wcum,
            ne::BrickBufs bb, long long n_tot, double* __restrict__ boxes_out)
{
    constexpr int SLOTS = BTHREADS / TPA;
    static_assert(BTHREADS % TPA == 0 && SLOTS % 32 == 0, "whole warps of one pair lane");
    constexpr int QF = TPA == 1 ? QMAX : (TPA == 2 ? 56 : 48);
    constexpr int QJ = TPA == 1 ? 0 : QMAX - QF;
    static_assert(QF % FRB == 0 && QJ % FRB == 0 && QF + QJ <= QMAX && QJ <= QF, "TMEM columns per warp");
    extern __shared__ __align__(16) unsigned char smem[];
    const int rep = cta_rep[blockIdx.x];
    const XRep& R_ = reps[rep];
    const int C = R_.ncta, rank = (int)blockIdx.x - R_.cta0;
    const unsigned n_cta = gridDim.x;
    const int n = R_.n, nb = R_.nb, nx = R_.nx, ny = R_.ny, nz = R_.nz;
    const int nst = R_.st_cnt, M = R_.st_margin;
    const int A_c = brick_cta_atoms(n, C, nb);
    const int cells_c = A_c / nb;
    const int ncell = n / nb;

    // ---- shared memory (brick_smem_bytes gives the same sizes)
    float4* s_sv = (float4*)smem;                                 // [nb * nst]
    float* s_sd = (float*)(s_sv + nb * nst);                      // [nb * nst]
    const int LY = ny + 2 * M;
    int* s_lxy = (int*)(s_sd + nb * nst);                         // [(nx + 2M) * LY]
    int* s_lz = s_lxy + (nx + 2 * M) * LY;                        // [nb][nz + 2M]
    unsigned short* s_K = (unsigned short*)(s_lz + nb * (nz + 2 * M));  // [4][NKT]
    float* s_tot = (float*)(((size_t)(s_K + 4 * NKT) + 15) & ~(size_t)15);  // [NSV]
    float4* s_f = (float4*)(((size_t)(s_tot + NSV) + 15) & ~(size_t)15);  // [TPA - 1][SLOTS]
    float2* s_rho = (float2*)(s_f + (TPA - 1) * SLOTS);           // [TPA - 1][SLOTS]
    float* s_red = (float*)(s_rho + (TPA - 1) * SLOTS);           // [NWARP][NRED][2]
    int* s_flag = (int*)(s_red + NWARP * NRED * 2);               // [4]
    unsigned* s_tm = (unsigned*)(s_flag + 4);                     // [4] TMEM base address
    unsigned char* s_end = (unsigned char*)(s_tm + 4);
    float4* s_vir = nullptr;  // barostat: [TPA - 1][SLOTS] pair-lane virials
    float* s_vred = nullptr;  // [NWARP][6] warp sums of the virial
    double* s_mu = nullptr;   // [3] the step's scale factors
    if constexpr (NPT) {
        s_vir = (float4*)(((size_t)s_end + 15) & ~(size_t)15);
        s_vred = (float*)(s_vir + (TPA - 1) * SLOTS);
        s_mu = (double*)(((size_t)(s_vred + NWARP * 6) + 15) & ~(size_t)15);
        s_end = (unsigned char*)(s_mu + 4);
    }
    float4* s_tabP = (float4*)(((size_t)s_end + 15) & ~(size_t)15);  // [nk - 1 - k_lo]
    const int n_int = tab.nk - 1 - k_lo;
    float4* s_tabF = s_tabP + n_int;
    {
        unsigned dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        // every CTA takes this decision alike (the same counts for all), so
        // either all run or none does
        if ((size_t)((unsigned char*)(s_tabF + n_int) - smem) > (size_t)dyn) {
            if (threadIdx.x == 0) {
                ne_set_status(status, ST_EINVAL);
                ne_set_status(status + 1 + R_.widx, ST_EINVAL);
            }
            return;
        }
    }
    for (int q = threadIdx.x; q < nb * nst; q += BTHREADS) {
        s_sv[q] = st_vec[R_.st_off + q];
        s_sd[q] = st_dist[R_.st_off + q];
    }
    for (int q = threadIdx.x; q < 2 * n_int; q += BTHREADS)
        ((q & 1) ? s_tabF : s_tabP)[q >> 1] = tab.pf32[2 * k_lo + q];
    for (int q = threadIdx.x; q < (nx + 2 * M) * LY; q += BTHREADS)
        s_lxy[q] = ((((q / LY - M) % nx + nx) % nx) * ny + ((q % LY - M) % ny + ny) % ny) * nz;
    for (int q = threadIdx.x; q < nb * (nz + 2 * M); q += BTHREADS) {
        const int Z = q % (nz + 2 * M);
        s_lz[q] = ((Z - M) % nz + nz) % nz + (q / (nz + 2 * M)) * ncell;
    }
    // TMEM: all columns for this CTA (one per SM), returned after the step
    // loop, which every thread of the CTA leaves at the same step
    ne_tm_alloc(s_tm);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tm_base = *s_tm;
    const unsigned tm_w = tm_base + ((unsigned)(32 * ((threadIdx.x >> 5) & 3)) << 16) +
                          (unsigned)(QMAX * (threadIdx.x >> 7));  // this warp's lanes and columns
    const float Dr = R_.D;
    for (int q = threadIdx.x; q < nb * NKT; q += BTHREADS) {
        const int b = q / NKT, iq = q % NKT;
        // the last bin holds every real entry (padding entries have distance 1e30)
        const float cq = iq < NKT - 1 ? (float)tab.r_c + (float)iq * (2.f * Dr / (float)(NKT - 1)) : 1e29f;
        int lo = 0, hi = nst;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_sd[b * nst + mid] < cq) lo = mid + 1;
            else hi = mid;
        }
        s_K[q] = (unsigned short)lo;
    }
    const float inv_dK = (float)(NKT - 1) / (2.f * Dr);

    // the replica's atoms in global memory, basis-major: entry b * ncell + cell
    const size_t gofs = (size_t)R_.off;
    float4* u_cur = bb.u4;  // set per step from the parity
    auto slot_atom = [&](int sl) { return rank * A_c + (sl % cells_c) * nb + sl / cells_c; };
    const int slot = threadIdx.x % SLOTS, lane = threadIdx.x / SLOTS;
    const int a = slot_atom(slot);
    const bool valid = slot < A_c && a < n;
    const int ai = valid ? a : 0;
    int sxy, sz, stb, skb, sui;
    {
        const int b = ai % nb;
        sui = b * ncell + ai / nb;
        int c = ai / nb;
        sz = c % nz;
        c /= nz;
        sxy = (c / ny) * LY + c % ny;
        stb = b * nst;
        skb = b * NKT;
    }
    if constexpr (QJ > 0) {
        // the neighbour indices of this thread's first QJ visits (visits past
        // the stencil read its last entry, as in the passes)
#pragma unroll 1
        for (int q0 = 0; q0 < QJ; q0 += FRB) {
            float jf[FRB];
#pragma unroll
            for (int uq = 0; uq < FRB; ++uq) {
                const int k = min(lane + TPA * (q0 + uq), nst - 1);
                const int code = __float_as_int(s_sv[stb + k].w);
                jf[uq] = __int_as_float(s_lxy[sxy + (code & 0xffff)] + s_lz[sz + ((unsigned)code >> 16)]);
            }
            __syncwarp();
            ne_tm_st(tm_w + (unsigned)(QF + q0), jf);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    const int ta = slot_atom(threadIdx.x);
    const bool own = threadIdx.x < A_c && ta < n;
    const int tsu = own ? (ta % nb) * ncell + ta / nb : 0;
    const int own_warps = (A_c + 31) / 32;
    auto site_fix = [&](int q) -> long long {
        const int b = ta % nb;
        int c = ta / nb;
        const int iz = c % nz;
        c /= nz;
        const int ic = q == 0 ? c / ny : (q == 1 ? c % ny : iz);
        return __double2ll_rn(R_.cell[q] * (ic + R_.basis[b][q]) * XSCALE);
    };
    const size_t gi = (size_t)(R_.off + (own ? ta : 0)) * 3;
    const bool spc = R_.nsp >= 2;
    auto spq = [&]() { return spc && own ? (int)R_.sp[ta] : 0; };
    auto k_of = [&](int q) { return spc ? R_.kfs[q] : R_.kf; };

    // CTA sums of ND double-float and NF FP32 values and the maximum of mx,
    // to this CTA's slot of the partials of parity p: each warp reduces its
    // lanes, then warp q combines quantity q over the warps in a fixed order
    auto cta_partials = [&](dfl(&vd)[ND_], float(&vf)[NF_], float mx, int p) {
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (w < own_warps) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int q = 0; q < ND_; ++q)
                    vd[q] = df_add(vd[q], {__shfl_xor_sync(0xffffffffu, vd[q].hi, o),
                                           __shfl_xor_sync(0xffffffffu, vd[q].lo, o)});
#pragma unroll
                for (int q = 0; q < NF_; ++q) vf[q] += __shfl_xor_sync(0xffffffffu, vf[q], o);
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if (l == 0) {
                for (int q = 0; q < ND_; ++q) {
                    s_red[(w * NRED + q) * 2] = vd[q].hi;
                    s_red[(w * NRED + q) * 2 + 1] = vd[q].lo;
                }
                for (int q = 0; q < NF_; ++q) s_red[(w * NRED + ND_ + q) * 2] = vf[q];
                s_red[(w * NRED + NP_) * 2] = mx;
            }
        }
        __syncthreads();
        if (w <= NP_) {
            const int q = w;
            const bool has = l < own_warps;
            float* dst = bb.part + ((size_t)p * n_cta + blockIdx.x) * NPART;
            if (q < ND_) {
                dfl v = has ? dfl{s_red[(l * NRED + q) * 2], s_red[(l * NRED + q) * 2 + 1]} : dfl{0.f, 0.f};
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    v = df_add(v, {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
                if (l == 0) {
                    dst[2 * q] = v.hi;
                    dst[2 * q + 1] = v.lo;
                }
            } else if (q < NP_) {
                float v = has ? s_red[(l * NRED + q) * 2] : 0.f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (l == 0) dst[ND_ + q] = v;
            } else {
                float m = has ? s_red[(l * NRED + NP_) * 2] : 0.f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (l == 0) dst[NSV] = m;
            }
        }
    };

    // ---- state of the owned atom
    long long xr[3] = {0, 0, 0};
    float v[3] = {0, 0, 0}, u[3] = {0, 0, 0}, xi[3] = {0, 0, 0};
    int bad = 0;
    {
        const float kf = k_of(spq());
        dfl pd[ND_] = {};
        float pf[NF_] = {};
        float um = 0.f;
        if (own) {
            for (int q = 0; q < 3; ++q) {
                xr[q] = __double2ll_rn(xg[gi + q] * XSCALE) - site_fix(q);
                v[q] = (float)vg[gi + q];
                u[q] = fix_to_float(xr[q]);
            }
            bb.u4[(size_t)(s_begin & 1) * n_tot + gofs + tsu] = make_float4(u[0], u[1], u[2], 0.f);
            ne_normals32(ne_philox_block(R_.seed, R_.replica, (unsigned)S.stream, (unsigned)ta,
                                         (unsigned long long)s_begin),
                         xi);
            const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            pd[P_UE] = {0.5f * kf * u2, 0.f};
            const float wxi = spc ? R_.mfs[spq()] * R_.c2fs[spq()] : 1.f;
            for (int c = 0; c < 3; ++c) {
                pf[P_UX - ND_ + c] = spc ? kf * u[c] : u[c];
                pf[P_XX - ND_ + c] = spc ? wxi * xi[c] : xi[c];
            }
            um = sqrtf(u2);
        }
        cta_partials(pd, pf, um, (int)(s_begin & 1));
    }
    unsigned gen = 0;
    bool alive = grid_barrier(bb.bar, n_cta, gen, status, bb.abortf, s_flag);

    unsigned n_cand = 0, n_pair = 0;
    const float rc2 = tab.rc2f, rmin2 = tab.rmin2f, inv_h = tab.inv_h_rf;
    const int nk = tab.nk;
    const int kchk = max(k_lo, (int)(sqrtf(rmin2) * inv_h) + 2);
    const float dt = (float)S.dt;
    const float rho_maxf = (float)tab.rho_max;
    const float ihr_hi = (float)tab.inv_h_rho, ihr_lo = (float)(tab.inv_h_rho - (double)ihr_hi);
    const bool wthread = rank == 0 && threadIdx.x == BTHREADS - 1;
    double Wacc[2] = {0.0, 0.0};
    if (wthread) {
        Wacc[0] = Wg[2 * R_.widx];
        Wacc[1] = Wg[2 * R_.widx + 1];
    }
    double UE_prev = 0.0;
    bool dead = false;  // the replica left the stencil range: its CTAs keep to the barriers only
    // barostat: the box and the sites scale by mu_tot per axis from the
    // call's start (the same values in every CTA of the replica); stencil
    // vectors are multiplied by it
    double mu_tot[3] = {1.0, 1.0, 1.0};
    float muf[3] = {1.f, 1.f, 1.f}, mu_min = 1.f;

#pragma unroll 1
    for (long long it = 0; it <= n_steps && alive; ++it) {
        const long long s = s_begin + it;
        const bool fin = it == n_steps;
        const int p = (int)(s & 1);
        u_cur = bb.u4 + (size_t)p * n_tot + gofs;

        // ---- replica sums of step s from the CTA partials (fixed order)
        float umax;
        {
            const int q = threadIdx.x >> 5, l = threadIdx.x & 31;
            const float* sp = bb.part + ((size_t)p * n_cta + R_.cta0) * NPART;
            if (q < ND_) {
                dfl acc = {0.f, 0.f};
                for (int r = l; r < C; r += 32)
                    acc = df_add(acc, {__ldcg(&sp[r * NPART + 2 * q]), __ldcg(&sp[r * NPART + 2 * q + 1])});
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    acc = df_add(acc, {__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)});
                if (l == 0) {
                    s_tot[2 * q] = acc.hi;
                    s_tot[2 * q + 1] = acc.lo;
                }
            } else if (q < NP_) {
                float acc = 0.f;
                for (int r = l; r < C; r += 32) acc += __ldcg(&sp[r * NPART + ND_ + q]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (l == 0) s_tot[ND_ + q] = acc;
            }
            float um = 0.f;
            for (int r = l; r < C; r += 32) um = fmaxf(um, __ldcg(&sp[r * NPART + NSV]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, o));
            umax = um;
        }
        bool out_ = !(umax <= R_.D);
        if constexpr (NPT) {
            // the scaled stencil must still cover r_c + 2 max|u|, and the box
            // must keep two periodic images more than 2 r_c apart
            const float need = ((float)tab.r_c + 2.f * umax) / mu_min - (float)tab.r_c;
            out_ = out_ || !(need <= 2.f * R_.D);
            for (int c = 0; c < 3; ++c) out_ = out_ || !(mu_tot[c] * R_.box0[c] > 2.0 * tab.r_c + 1.2);
        }
        if (!dead && out_) {
            // an atom beyond the stencil range: the replica's result is void;
            // every CTA of the replica sees the same sums and stops working
            if (threadIdx.x == 0) {
                const int e = isnan(umax) ? ST_ENAN : ST_ERANGE;
                ne_set_status(status, e);
                ne_set_status(status + 1 + R_.widx, e);
            }
            dead = true;
        }

        // ---- pass 1: density, pair forces and energy, f'(r)/r of every visit to TMEM
        const float4 ui = dead ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldcg(&u_cur[sui]);
        int m = 0, nq = 0;  // pairs inside r_c; the warp's visits
        float fx = 0.f, fy = 0.f, fz = 0.f, ep = 0.f;
        float vxx = 0.f, vyy = 0.f, vzz = 0.f;  // diagonal virial (barostat only)
        dfl rho = {0.f, 0.f};
        if (!dead) {
            float c = sqrtf(ui.x * ui.x + ui.y * ui.y + ui.z * ui.z) + umax;
            if constexpr (NPT) c = ((float)tab.r_c + c) / mu_min - (float)tab.r_c;  // in lattice units
            const int K = valid ? (int)s_K[skb + min(NKT - 1, (int)(c * inv_dK) + 2)] : 0;
            // every thread of the warp visits up to the warp's largest bound in
            // whole batches of FRB (TMEM stores are warp-wide); entries past a
            // thread's own bound lie outside r_c for it, and visits past the
            // stencil read its last entry, a far padding site
            const int Kw = __reduce_max_sync(0xffffffffu, K);
            nq = Kw > lane ? ((Kw - lane + TPA - 1) / TPA + FRB - 1) / FRB * FRB : 0;
            int ql = -1;  // this thread's last visit inside r_c
            float rh = 0.f, rl = 0.f;
            // one stencil visit (entry e, neighbour index j, visit index qv):
            // the pair's terms of rho, the forces and the energy; returns
            // f'(r)/r inside r_c, else 0
            auto visit = [&](float4 e, int j, int qv) -> float {
                float fr = 0.f;
                const float4 uj = __ldcg(&u_cur[j]);
                if constexpr (NPT) {
                    e.x *= muf[0];
                    e.y *= muf[1];
                    e.z *= muf[2];
                }
                const float dx = e.x + uj.x - ui.x, dy = e.y + uj.y - ui.y, dz = e.z + uj.z - ui.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < rc2) {
                    const float irh = rsqrtf(r2) * inv_h;
                    const float t = r2 * irh;
                    const int kk = min((int)t, nk - 2);
                    const float w = t - (float)kk;
                    float4 cf, g;
                    if (kk < kchk) {
                        if (r2 < rmin2) bad |= ST_ERANGE;
                        if (kk >= k_lo) {
                            cf = s_tabP[kk - k_lo];
                            g = s_tabF[kk - k_lo];
                        } else {
                            cf = __ldg(&tab.pf32[2 * kk]);
                            g = __ldg(&tab.pf32[2 * kk + 1]);
                        }
                    } else {
                        cf = s_tabP[kk - k_lo];
                        g = s_tabF[kk - k_lo];
                    }
                    {
                        // f and df/dw together (Horner with derivative)
                        float fv = fmaf(g.w, w, g.z), fd = g.w;
                        fd = fmaf(fd, w, fv);
                        fv = fmaf(fv, w, g.y);
                        fd = fmaf(fd, w, fv);
                        fv = fmaf(fv, w, g.x);
                        const float s_ = rh + fv, bp = s_ - rh;
                        rl += (rh - (s_ - bp)) + (fv - bp);
                        rh = s_;
                        fr = fd * irh;  // f'(r) / r
                        ql = qv;
                    }
                    float pv = fmaf(cf.w, w, cf.z), pd = cf.w;
                    pd = fmaf(pd, w, pv);
                    pv = fmaf(pv, w, cf.y);
                    pd = fmaf(pd, w, pv);
                    pv = fmaf(pv, w, cf.x);
                    const float sc = pd * irh;
                    fx += sc * dx;
                    fy += sc * dy;
                    fz += sc * dz;
                    ep += pv;
                    if constexpr (NPT) {  // -(1/2) r_a^2 / r dU/dr of the pair's half
                        vxx -= 0.5f * sc * dx * dx;
                        vyy -= 0.5f * sc * dy * dy;
                        vzz -= 0.5f * sc * dz * dz;
                    }
                    ++m;
                }
                return fr;
            };
            // the first QJ visits: neighbour indices from TMEM
            const int nqa = QJ > 0 ? min(nq, QJ) : 0;
#pragma unroll 1
            for (int q0 = 0; q0 < nqa; q0 += FRB) {
                float jf[FRB], frv[FRB];
                __syncwarp();
                ne_tm_ld(tm_w + (unsigned)(QF + q0), jf);
#pragma unroll
                for (int uq = 0; uq < FRB; ++uq) {
                    const int k = min(lane + TPA * (q0 + uq), nst - 1);
                    frv[uq] = visit(s_sv[stb + k], __float_as_int(jf[uq]), q0 + uq);
                }
                __syncwarp();
                ne_tm_st(tm_w + (unsigned)q0, frv);
            }
            // the rest: indices from the wrapped-cell tables
#pragma unroll 1
            for (int q0 = nqa; q0 < nq; q0 += FRB) {
                float frv[FRB];
#pragma unroll
                for (int uq = 0; uq < FRB; ++uq) {
                    const int k = min(lane + TPA * (q0 + uq), nst - 1);
                    const float4 e = s_sv[stb + k];
                    const int code = __float_as_int(e.w);
                    frv[uq] = visit(e, s_lxy[sxy + (code & 0xffff)] + s_lz[sz + ((unsigned)code >> 16)], q0 + uq);
                }
                if (q0 < QF) {
                    __syncwarp();
                    ne_tm_st(tm_w + (unsigned)q0, frv);
                }
            }
            __syncwarp();
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");  // the stores land before pass 2 loads
            rho = {rh, rl};
            n_cand += valid ? (unsigned)nq : 0u;
            n_pair += valid ? (unsigned)m : 0u;
            nq = __reduce_max_sync(0xffffffffu, ql) + 1;  // pass 2 stops after the warp's last pair
            ep *= 0.5f;
            if (valid && lane > 0) s_rho[(lane - 1) * SLOTS + slot] = make_float2(rho.hi, rho.lo);
        }
        __syncthreads();
        float emb = 0.f;
        if (own && !dead) {
            dfl rr = rho;
            for (int l2 = 1; l2 < TPA; ++l2) {
                const float2 r1_ = s_rho[(l2 - 1) * SLOTS + threadIdx.x];
                rr = df_add(rr, {r1_.x, r1_.y});
            }
            if (!(rr.hi < rho_maxf)) bad |= ST_ERANGE;
            const int kk = min(max((int)(rr.hi * ihr_hi), 0), nk - 2);
            const float w = fmaf(rr.hi, ihr_hi, -(float)kk) + (rr.hi * ihr_lo + rr.lo * ihr_hi);
            const float4 c = __ldg(&tab.F32[kk]);
            emb = c.x + w * (c.y + w * (c.z + w * c.w));
            const float dF = (c.y + w * (2.f * c.z + 3.f * w * c.w)) * tab.inv_h_rhof;
            bb.fp[gofs + tsu] = dF;
            if (!isfinite(emb)) bad |= ST_ENAN;
        }
        alive = grid_barrier(bb.bar, n_cta, gen, status, bb.abortf, s_flag);  // F' visible everywhere
        if (!alive) break;

        // ---- pass 2: embedding forces over the visits of pass 1, f'(r)/r from TMEM
        if (!dead) {
            const float dFi = __ldcg(&bb.fp[gofs + sui]);
            const float* fp_r = bb.fp + gofs;
            const int nqt = min(nq, QF);
#pragma unroll 1
            for (int q0 = 0; q0 < nqt; q0 += FRB) {
                // (the neighbour indices from the tables: also reading them
                // from TMEM here, 16 live words a batch, spilled at the
                // 80-register cap)
                float frv[FRB];
                __syncwarp();
                ne_tm_ld(tm_w + (unsigned)q0, frv);
#pragma unroll
                for (int uq = 0; uq < FRB; ++uq) {
                    if (frv[uq] != 0.f) {  // inside r_c (f' vanishes only at r_c)
                        const int k = min(lane + TPA * (q0 + uq), nst - 1);
                        float4 e = s_sv[stb + k];
                        const int code = __float_as_int(e.w);
                        const int j = s_lxy[sxy + (code & 0xffff)] + s_lz[sz + ((unsigned)code >> 16)];
                        const float4 uj = __ldcg(&u_cur[j]);
                        const float dFj = __ldcg(&fp_r[j]);
                        if constexpr (NPT) {
                            e.x *= muf[0];
                            e.y *= muf[1];
                            e.z *= muf[2];
                        }
                        const float dx = e.x + uj.x - ui.x, dy = e.y + uj.y - ui.y, dz = e.z + uj.z - ui.z;
                        const float sc = (dFi + dFj) * frv[uq];
                        fx += sc * dx;
                        fy += sc * dy;
                        fz += sc * dz;
                        if constexpr (NPT) {
                            vxx -= 0.5f * sc * dx * dx;
                            vyy -= 0.5f * sc * dy * dy;
                            vzz -= 0.5f * sc * dz * dz;
                        }
                    }
                }
            }
            // visits past the TMEM columns: the pair recomputed
            for (int q = QF; q < nq; ++q) {
                const int k = min(lane + TPA * q, nst - 1);
                float4 e = s_sv[stb + k];
                const int code = __float_as_int(e.w);
                const int j = s_lxy[sxy + (code & 0xffff)] + s_lz[sz + ((unsigned)code >> 16)];
                const float4 uj = __ldcg(&u_cur[j]);
                if constexpr (NPT) {
                    e.x *= muf[0];
                    e.y *= muf[1];
                    e.z *= muf[2];
                }
                const float dx = e.x + uj.x - ui.x, dy = e.y + uj.y - ui.y, dz = e.z + uj.z - ui.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < rc2)) continue;
                const float dFj = __ldcg(&fp_r[j]);
                const float irh = rsqrtf(r2) * inv_h;
                const float t = r2 * irh;
                const int kk = min((int)t, nk - 2);
                const float w = t - (float)kk;
                const float4 g = kk >= k_lo ? s_tabF[kk - k_lo] : __ldg(&tab.pf32[2 * kk + 1]);
                const float sc = (dFi + dFj) * ((g.y + w * (2.f * g.z + 3.f * w * g.w)) * irh);
                fx += sc * dx;
                fy += sc * dy;
                fz += sc * dz;
                if constexpr (NPT) {
                    vxx -= 0.5f * sc * dx * dx;
                    vyy -= 0.5f * sc * dy * dy;
                    vzz -= 0.5f * sc * dz * dz;
                }
            }
            if (valid && lane > 0) s_f[(lane - 1) * SLOTS + slot] = make_float4(fx, fy, fz, ep);
            if constexpr (NPT)
                if (valid && lane > 0) s_vir[(lane - 1) * SLOTS + slot] = make_float4(vxx, vyy, vzz, 0.f);
        }
        __syncthreads();
        double mus[3] = {1.0, 1.0, 1.0};  // this step's scale factors (barostat)
        if constexpr (NPT) {
            if (!fin) {
                // the diagonal virial of this CTA's atoms at x_s (double-float
                // per axis: a fixed warp tree, then warp 0 over the warps) to
                // global memory; after the barrier warp 0 of every CTA sums the
                // replica's CTAs in a fixed order and thread 0 takes the
                // barostat step of the cluster runner
                const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
                dfl vd[3] = {};
                if (own && !dead) {
                    vd[0] = {vxx, 0.f};
                    vd[1] = {vyy, 0.f};
                    vd[2] = {vzz, 0.f};
                    for (int l2 = 1; l2 < TPA; ++l2) {
                        const float4 v1 = s_vir[(l2 - 1) * SLOTS + threadIdx.x];
                        vd[0] = df_add(vd[0], {v1.x, 0.f});
                        vd[1] = df_add(vd[1], {v1.y, 0.f});
                        vd[2] = df_add(vd[2], {v1.z, 0.f});
                    }
                }
                if (w < own_warps) {
                    warp_df3(vd);
                    if (l == 0)
                        for (int a3 = 0; a3 < 3; ++a3) {
                            s_vred[w * 6 + 2 * a3] = vd[a3].hi;
                            s_vred[w * 6 + 2 * a3 + 1] = vd[a3].lo;
                        }
                }
                __syncthreads();
                if (w == 0) {
                    dfl t[3];
                    for (int a3 = 0; a3 < 3; ++a3)
                        t[a3] = l < own_warps ? dfl{s_vred[l * 6 + 2 * a3], s_vred[l * 6 + 2 * a3 + 1]} : dfl{0.f, 0.f};
                    warp_df3(t);
                    if (l == 0)
                        for (int a3 = 0; a3 < 3; ++a3) {
                            bb.vir[(size_t)blockIdx.x * 6 + 2 * a3] = t[a3].hi;
                            bb.vir[(size_t)blockIdx.x * 6 + 2 * a3 + 1] = t[a3].lo;
                        }
                }
                alive = grid_barrier(bb.bar, n_cta, gen, status, bb.abortf, s_flag);  // virials visible
                if (!alive) break;
                if (w == 0) {
                    dfl t[3] = {};
                    const float* vp = bb.vir + (size_t)R_.cta0 * 6;
                    for (int r = l; r < C; r += 32)
                        for (int a3 = 0; a3 < 3; ++a3)
                            t[a3] = df_add(t[a3], {__ldcg(&vp[r * 6 + 2 * a3]), __ldcg(&vp[r * 6 + 2 * a3 + 1])});
                    warp_df3(t);
                    if (l == 0) {
                        double Wa[3];
                        for (int a3 = 0; a3 < 3; ++a3) Wa[a3] = (double)t[a3].hi + (double)t[a3].lo;
                        const double V = mu_tot[0] * R_.box0[0] * mu_tot[1] * R_.box0[1] * mu_tot[2] * R_.box0[2];
                        const double lam = lam_tab[it + 1], dtd = S.dt;
                        double z[3];
                        ne_normals64(ne_philox_block(R_.seed, R_.replica, (unsigned)STREAM_BARO, 0u,
                                                     (unsigned long long)s),
                                     z);
                        const double noise = sqrt(2.0 * R_.kT * R_.mp * dtd / V);
                        if (R_.npt == 2) {
                            for (int a3 = 0; a3 < 3; ++a3) {
                                const double drive = (R_.dof / 3.0 * R_.kT + lam * Wa[a3]) / V - R_.P0;
                                s_mu[a3] = exp(R_.mp * drive * dtd + noise * z[a3]);
                            }
                        } else {  // isotropic; a replica without the barostat has mp = 0: mu = 1
                            const double drive = (R_.dof * R_.kT + lam * (Wa[0] + Wa[1] + Wa[2])) / (3.0 * V) - R_.P0;
                            s_mu[0] = s_mu[1] = s_mu[2] = exp((R_.mp * drive * dtd + noise * z[0]) / 3.0);
                        }
                    }
                }
                __syncthreads();
                for (int a3 = 0; a3 < 3; ++a3) {
                    mus[a3] = s_mu[a3];
                    mu_tot[a3] *= mus[a3];
                    muf[a3] = (float)mu_tot[a3];
                }
                mu_min = fminf(muf[0], fminf(muf[1], muf[2]));
            }
        }

        // ---- fused step of the owned atom
        if (wthread && !dead) {
            // work increment of step s - 1 from the sums of step s
            const double U0 = (double)s_tot[2 * P_U0] + (double)s_tot[2 * P_U0 + 1];
            if (it > 0) {
                const long long sp = s - 1;
                const double gw = S.path == 0 ? U0 - UE_prev : U0;
                int wslot = -1;
                if (sp >= S.t_eq && sp < S.t_eq + S.t_s) wslot = 0;
                else if (sp >= 2 * S.t_eq + S.t_s && sp < 2 * S.t_eq + 2 * S.t_s) wslot = 1;
                if (wslot >= 0) {
                    Wacc[wslot] += (lam_tab[it] - lam_tab[it - 1]) * gw;
                    if (wcum) {
                        const long long k = wslot == 0 ? sp - S.t_eq : sp - (2 * S.t_eq + S.t_s);
                        double* wc = wcum + (size_t)(2 * R_.widx + wslot) * (size_t)(S.t_s + 1);
                        if (k == 0) wc[0] = 0.0;
                        wc[k + 1] = Wacc[wslot];
                    }
                }
            }
            UE_prev = (double)s_tot[2 * P_UE] + (double)s_tot[2 * P_UE + 1];
        }
        {
            dfl pd[ND_] = {};
            float pf[NF_] = {};
            float un = 0.f;
            if (own && !dead) {
                float4 f = make_float4(fx, fy, fz, ep);
                for (int l2 = 1; l2 < TPA; ++l2) {
                    const float4 f1_ = s_f[(l2 - 1) * SLOTS + threadIdx.x];
                    f.x += f1_.x;
                    f.y += f1_.y;
                    f.z += f1_.z;
                    f.w += f1_.w;
                }
                const float F0[3] = {f.x, f.y, f.z};
                const int q = spq();
                const float c1 = R_.c1f, kf = k_of(q);
                const float hdt = spc ? R_.hdts[q] : R_.hdt_mf, c2 = spc ? R_.c2fs[q] : R_.c2f;
                const float wcm = spc ? R_.mfs[q] * R_.invM : 0.f;
                const float invN = 1.f / (float)n;
                float mFE[3], mxi[3];
                for (int c = 0; c < 3; ++c) {
                    if (spc) {
                        mFE[c] = S.fix_cm ? -wcm * s_tot[T_UX + c] : 0.f;
                        mxi[c] = S.fix_cm ? s_tot[T_XX + c] * R_.invM : 0.f;
                    } else {
                        mFE[c] = S.fix_cm ? -kf * s_tot[T_UX + c] * invN : 0.f;
                        mxi[c] = S.fix_cm ? s_tot[T_XX + c] * invN : 0.f;
                    }
                }
                const float ls = (float)lam_tab[it], ln = (float)lam_tab[it + 1];
                if (it > 0)
                    for (int c = 0; c < 3; ++c) v[c] += hdt * blendf(S.path, ls, F0[c], -kf * u[c] - mFE[c]);
                pd[P_U0] = {emb + f.w, 0.f};
                if (!fin) {
                    for (int c = 0; c < 3; ++c) {
                        v[c] += hdt * blendf(S.path, ln, F0[c], -kf * u[c] - mFE[c]);
                        const float v1 = v[c];
                        v[c] = spc ? c1 * v[c] + (c2 * xi[c] - mxi[c]) : c1 * v[c] + c2 * (xi[c] - mxi[c]);
                        const float dlt = 0.5f * dt * (v1 + v[c]);
                        if (!(fabsf(dlt) < 0.25f)) bad |= ST_ERANGE;
                        xr[c] += (long long)__float2int_rn(dlt * 4294967296.f);
                        // barostat: positions scale about the origin, so the
                        // displacement from the scaled site scales by mu
                        if constexpr (NPT) xr[c] = __double2ll_rn(mus[c] * (double)xr[c]);
                        u[c] = fix_to_float(xr[c]);
                    }
                    ne_normals32(ne_philox_block(R_.seed, R_.replica, (unsigned)S.stream, (unsigned)ta,
                                                 (unsigned long long)(s + 1)),
                                 xi);
                    bb.u4[(size_t)(p ^ 1) * n_tot + gofs + tsu] = make_float4(u[0], u[1], u[2], 0.f);
                }
                const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                const float wxi = spc ? R_.mfs[q] * R_.c2fs[q] : 1.f;
                pd[P_UE] = {0.5f * kf * u2, 0.f};
                for (int c = 0; c < 3; ++c) {
                    pf[P_UX - ND_ + c] = spc ? kf * u[c] : u[c];
                    pf[P_XX - ND_ + c] = spc ? wxi * xi[c] : xi[c];
                }
                un = sqrtf(u2);
                for (int c = 0; c < 3; ++c)
                    if (!isfinite(v[c])) bad |= ST_ENAN;
            }
            if (!fin) {
                cta_partials(pd, pf, dead ? 1e30f : un, p ^ 1);
                alive = grid_barrier(bb.bar, n_cta, gen, status, bb.abortf, s_flag);  // u of s + 1 visible
            }
        }
    }
    ne_tm_free(tm_base);  // every warp is past its last TMEM access
    if (bad) {
        ne_set_status(status, bad);
        ne_set_status(status + 1 + R_.widx, bad);
    }
    if (work) {
        for (int o = 16; o > 0; o >>= 1) {
            n_cand += __shfl_xor_sync(0xffffffffu, n_cand, o);
            n_pair += __shfl_xor_sync(0xffffffffu, n_pair, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&work[0], (unsigned long long)n_cand);
            atomicAdd(&work[1], (unsigned long long)n_pair);
        }
    }
    if (!alive) return;  // a wait gave up: the call reports NE_ETIMEOUT and writes nothing back
    // every CTA's error bits for its replica are in the status word after
    // this barrier; a replica that raised none writes its state back
    alive = grid_barrier(bb.bar, n_cta, gen, status, bb.abortf, s_flag);
    if (!alive) return;
    if (threadIdx.x == 0) s_flag[1] = atomicOr(status + 1 + R_.widx, 0);
    __syncthreads();
    if (s_flag[1] == 0) {
        if (own)
            for (int c = 0; c < 3; ++c) {
                // the site of the atom in the (scaled) box
                const long long site = NPT ? __double2ll_rn(mu_tot[c] * (double)site_fix(c)) : site_fix(c);
                xg[gi + c] = (double)(xr[c] + site) / XSCALE;
                vg[gi + c] = (double)v[c];
            }
        if (wthread) {
            Wg[2 * R_.widx] = Wacc[0];
            Wg[2 * R_.widx + 1] = Wacc[1];
            if (NPT && boxes_out)
                for (int c = 0; c < 3; ++c) boxes_out[3 * R_.widx + c] = mu_tot[c] * R_.box0[c];
        }
    }
}

template <int TPA, bool NPT>
cudaError_t brick_attributes(size_t smem)
{
    return cudaFuncSetAttribute(k_brick<TPA, NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int TPA, bool NPT>
cudaError_t brick_occupancy(size_t smem, int* per)
{
    cudaError_t e = brick_attributes<TPA, NPT>(smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_brick<TPA, NPT>, BTHREADS, smem);
    return e;
}

template <int TPA, bool NPT>
cudaError_t brick_launch(cudaLaunchConfig_t& cfg, const XRep* reps, const int* cta_rep, const float4* st_vec,
                         const float* st_dist, double* x, double* v, double* W, int* status, const Sched& S,
                         long long s_begin, long long n_steps, const Tables& tab, unsigned long long* work, int k_lo,
                         const double* lam_tab, double* wcum, const ne::BrickBufs& bb, long long n_tot,
                         double* boxes_out)
{
    cudaError_t e = brick_attributes<TPA, NPT>(cfg.dynamicSmemBytes);
    if (e == cudaSuccess)
        e = cudaLaunchKernelEx(&cfg, k_brick<TPA, NPT>, reps, cta_rep, st_vec, st_dist, x, v, W, status, S, s_begin,
                               n_steps, tab, work, k_lo, lam_tab, wcum, bb, n_tot, boxes_out);
    return e;
}

}  // namespace

namespace ne {

size_t brick_smem_bytes(int tpa, int nb_nst_max, int lut_max, bool npt)
{
    const size_t slots = (size_t)(BTHREADS / tpa);
    size_t b = (sizeof(float4) + sizeof(float)) * (size_t)nb_nst_max + sizeof(int) * (size_t)lut_max +
               sizeof(unsigned short) * 4 * NKT;
    b = (b + 15) & ~(size_t)15;
    b += sizeof(float) * NSV;
    b = (b + 15) & ~(size_t)15;
    b += (sizeof(float4) + sizeof(float2)) * (size_t)(tpa - 1) * slots + sizeof(float) * NWARP * NRED * 2 +
         sizeof(int) * 4 + sizeof(unsigned) * 4;
    if (npt) {  // pair-lane virials, warp sums, scale factors
        b = (b + 15) & ~(size_t)15;
        b += sizeof(float4) * (size_t)(tpa - 1) * slots + sizeof(float) * NWARP * 6;
        b = (b + 15) & ~(size_t)15;
        b += sizeof(double) * 4;
    }
    return ((b + 15) & ~(size_t)15) + 16;  // + alignment of the tables
}

int brick_atoms_per_cta(int tpa) { return BTHREADS / tpa; }

int brick_max_ctas(int tpa, size_t smem, bool npt)
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    cudaError_t e;
    switch (tpa) {
    case 1: e = npt ? brick_occupancy<1, true>(smem, &per) : brick_occupancy<1, false>(smem, &per); break;
    case 2: e = npt ? brick_occupancy<2, true>(smem, &per) : brick_occupancy<2, false>(smem, &per); break;
    case 3: e = npt ? brick_occupancy<3, true>(smem, &per) : brick_occupancy<3, false>(smem, &per); break;
    case 4: e = npt ? brick_occupancy<4, true>(smem, &per) : brick_occupancy<4, false>(smem, &per); break;
    default: e = npt ? brick_occupancy<8, true>(smem, &per) : brick_occupancy<8, false>(smem, &per); break;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return per * sms;
}

cudaError_t launch_brick(int tpa, const XRep* reps, const int* cta_rep, int n_cta, size_t smem, const float4* st_vec,
                         const float* st_dist, double* x, double* v, double* W, int* status, const Sched& S,
                         long long s_begin, long long n_steps, const Tables& tab, unsigned long long* work,
                         int k_lo, const double* lam_tab, double* wcum, const BrickBufs& bb, long long n_tot,
                         cudaStream_t st, bool npt, double* boxes_out)
{
    if (npt && !bb.vir) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(bb.bar, 0, 2 * sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bb.abortf, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_cta, 1, 1);
    cfg.blockDim = dim3(BTHREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident at once: the grid barrier needs it
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#define NE_BRICK_ARGS cfg, reps, cta_rep, st_vec, st_dist, x, v, W, status, S, s_begin, n_steps, tab, work, k_lo, \
                      lam_tab, wcum, bb, n_tot, boxes_out
    switch (tpa) {
    case 1: return npt ? brick_launch<1, true>(NE_BRICK_ARGS) : brick_launch<1, false>(NE_BRICK_ARGS);
    case 2: return npt ? brick_launch<2, true>(NE_BRICK_ARGS) : brick_launch<2, false>(NE_BRICK_ARGS);
    case 3: return npt ? brick_launch<3, true>(NE_BRICK_ARGS) : brick_launch<3, false>(NE_BRICK_ARGS);
    case 4: return npt ? brick_launch<4, true>(NE_BRICK_ARGS) : brick_launch<4, false>(NE_BRICK_ARGS);
    case 8: return npt ? brick_launch<8, true>(NE_BRICK_ARGS) : brick_launch<8, false>(NE_BRICK_ARGS);
    default: return cudaErrorInvalidValue;
    }
#undef NE_BRICK_ARGS
}

}  // namespace ne
