// ne_cluster.cu -- persistent batched runner for crystals (mixed precision):
// one thread-block cluster per replica runs a whole step range of the
// four-phase switching schedule in one launch.
//
// Per replica, the cluster's C CTAs each own up to 384 atoms.  Every CTA
// keeps, in shared memory, the displacements from the lattice sites
// u_j = x_j - r0_j (FP32) and F'(rho_j) of all atoms of the replica; each CTA
// broadcasts its atoms' values to the other CTAs through distributed shared
// memory.  Neighbours come from a lattice stencil: for the basis site b of
// atom i, the sites j with |r0_j - r0_i| < r_c + 2D sorted by that distance,
// so r_ij = (r0_j - r0_i) + u_j - u_i needs no minimum image and no list, and
// a pair can lie inside r_c only if |r0_j - r0_i| < r_c + |u_i| + max_j |u_j|
// -- the loop over the stencil stops there.  D (2 A) is the largest
// displacement from a site the stencil covers; a replica whose atoms stray
// further is reported (NE_ERANGE) -- the crystal has melted.
//
// One MD step s:
//   [cluster barrier]  replica sums of step s (from the partial sums every
//                      CTA broadcast at the end of step s-1): noise mean,
//                      spring mean, max |u|; the work increment of step s-1;
//                      pass 1: rho, the pair forces phi'(r) and energy phi(r),
//                      f'(r)/r of every visit into tensor memory; F(rho),
//                      F'(rho), F' broadcast
//   [cluster barrier]  pass 2: the embedding forces (F'_i + F'_j) f'(r) r_ij/r
//                      over the visits inside r_c, f'(r)/r from tensor memory
//   [arrive]           closing and opening half kicks, drift,
//                      Ornstein-Uhlenbeck, drift; the normals of step s+1
//                      (counter-based, so drawn one step ahead)
//   [wait]             new u broadcast (no CTA still reads u of step s);
//                      CTA partial sums for step s+1.
// The work increment of step s is applied at step s+1 from those sums, in
// the same order, so a segment boundary changes no bit of the result.  The
// barriers are barrier.cluster arrive/wait (hardware; every CTA of a cluster
// is co-scheduled), so no thread spins on memory.  The EAM forces sum to zero
// in exact arithmetic; their FP32 round-off mean is not subtracted (the spring
// and noise means are), which lets the centre of mass move by ~1e-4 A per
// 100 ps.
//
// Precision: pair distances, splines, forces, velocities and the OU update
// in FP32; rho as a double-float; positions in fixed point (2^-32 A,
// registers); the work W in FP64; the replica energies as double-float pairs
// (within a CTA and across the cluster), the sums for the mean removal in
// FP32.
#include <algorithm>
#include <atomic>
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "ne_internal.cuh"
#include "ne_cluster.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int THREADS = 768;  // 24 warps: six per SMSP, 80 registers a thread
constexpr int TPA = 2;
constexpr int SLOTS = THREADS / TPA;  // atoms per CTA (one CTA per SM)
// Tensor memory as per-thread scratch: the shared-memory slot j of the
// neighbour at each of a thread's first QMAX stencil visits (fixed for the
// whole launch: the stencil is a lattice one, so atom i's k-th entry is
// always the same atom), written once before the step loop, and f'(r)/r of
// each of those visits (0 outside r_c), written by pass 1 and read by pass
// 2 instead of gathering the f table again.  The CTA holds all TM_COLS
// columns (one CTA per SM); warp w uses TMEM lanes 32 (w mod 4) .. +31 (its
// sub-partition's) and the CW columns from CW (w div 4): visit q of a thread
// is column q of its lane for f'(r)/r and half of column QMAX + q / 2 for j
// (two 16-bit slots a column), loaded FRB visits at a time.  Visits past
// QMAX (a hot or disordered replica) take j from the wrapped-cell tables
// and are recomputed in pass 2.
constexpr int TM_COLS = NE_TM_COLS;
constexpr int FRB = NE_TM_BATCH;
// stencil scan bounds: entries of basis b with |r0_j - r0_i| < r_c + c for
// c = q * 2D / (NKT - 1), q = 0 .. NKT - 1 (the last: the whole stencil)
constexpr int NKT = 256;
constexpr int NWARP = THREADS / 32;
constexpr int WQ = NWARP / 4;  // warps per TMEM lane quarter
constexpr int QMAX = TM_COLS / WQ * 2 / 3 / FRB * FRB;
constexpr int CW = QMAX + QMAX / 2;  // TMEM columns per warp
static_assert(NWARP % 4 == 0 && QMAX >= FRB && QMAX % FRB == 0 && WQ * CW <= TM_COLS, "TMEM columns per warp");

// partial sums broadcast at the end of step s for step s+1: the energies
// (double-float), then sum u and sum xi for the mean removal (FP32)
enum { P_U0 = 0, P_UE, P_UX, P_UY, P_UZ, P_XX, P_XY, P_XZ, NP_ };
constexpr int ND_ = 2, NF_ = NP_ - ND_;
// floats per CTA partial (and in the replica totals): (hi, lo) of each energy,
// then the FP32 sums; T_UX, T_XX: where sum u and sum xi start
constexpr int NSV = 2 * ND_ + NF_;
constexpr int T_UX = 2 * ND_ + (P_UX - ND_), T_XX = 2 * ND_ + (P_XX - ND_);
// values per warp in the reduction scratch: the larger of the two reductions
constexpr int NRED = (int)NP_ + 1;  // sums and one maximum

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

// CTA sums of ND double-float and NF FP32 values and the maximum of mx,
// written into slot `rank` of the slot arrays of every CTA of the cluster:
// dst[rank * NSV + ...] gets (hi, lo) of each double-float sum, then the FP32
// sums; mslot[rank] the maximum.  Each warp reduces its lanes; then warp q
// combines quantity q over the warps with a shuffle tree (a fixed order) and
// its lanes r < C store it into CTA r.  One __syncthreads; the caller
// separates two uses of s_red by a cluster barrier.
template <int ND, int NF>
__device__ __forceinline__ void cta_sum_bcast(cg::cluster_group& cluster, dfl (&vd)[ND], float (&vf)[NF], float mx,
                                              float* s_red, float* dst, float* mslot, int rank, int C, int nwarp)
{
    constexpr int NV = ND + NF;
    static_assert(NV + 1 <= NRED && NV + 1 <= NWARP, "reduction scratch too small");
    static_assert(2 * ND + NF == NSV, "slot layout");
    // only the first nwarp warps hold values (the threads that own atoms)
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (w < nwarp) {
        warp_df_sum<ND>(vd);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int q = 0; q < NF; ++q) vf[q] += __shfl_xor_sync(0xffffffffu, vf[q], o);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (l == 0) {
            for (int q = 0; q < ND; ++q) {
                s_red[(w * NRED + q) * 2] = vd[q].hi;
                s_red[(w * NRED + q) * 2 + 1] = vd[q].lo;
            }
            for (int q = 0; q < NF; ++q) s_red[(w * NRED + ND + q) * 2] = vf[q];
            s_red[(w * NRED + NV) * 2] = mx;
        }
    }
    __syncthreads();
    if (w <= NV) {  // warp-uniform: warp q handles quantity q, lane l holds warp l's partial
        const int q = w;
        const bool has = l < nwarp;
        if (q < ND) {
            dfl v = has ? dfl{s_red[(l * NRED + q) * 2], s_red[(l * NRED + q) * 2 + 1]} : dfl{0.f, 0.f};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                v = df_add(v, {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
            if (l < C) {
                float* d = cluster.map_shared_rank(dst, l) + rank * NSV + 2 * q;
                d[0] = v.hi;
                d[1] = v.lo;
            }
        } else if (q < NV) {
            float v = has ? s_red[(l * NRED + q) * 2] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (l < C) cluster.map_shared_rank(dst, l)[rank * NSV + ND + q] = v;
        } else {
            float m = has ? s_red[(l * NRED + NV) * 2] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (l < C) cluster.map_shared_rank(mslot, l)[rank] = m;
        }
    }
}

// Positions of owned atoms in fixed point, X = x * 2^32 (int64): the drift
// of a step (FP32) is added as an exact integer, the displacement from the
// site is converted to FP32 with integer and FP32 instructions only (no FP64,
// which runs at 1/64 of the FP32 rate here), and a position written out as
// X * 2^-32 in FP64 reads back to the same X, so segments resume bit for bit.
constexpr double XSCALE = 4294967296.0;  // 2^32 per Angstrom

// d * 2^-32 rounded once to FP32 (exact split into 2^16 parts; |d| < 2^40)
__device__ __forceinline__ float fix_to_float(long long d)
{
    const int hi = (int)(d >> 16), lo = (int)(d & 0xffff);
    return fmaf((float)hi, 1.52587890625e-05f, (float)lo * 2.3283064365386963e-10f);
}

__device__ __forceinline__ float blendf(int path, float lam, float F0, float FE)
{
    return path == 0 ? (1.f - lam) * F0 + lam * FE : lam * F0;
}

// Lambda(s) of the schedule for s = s_begin .. s_begin + count - 1, once per
// run segment (FP64; read by the persistent kernel instead of evaluated).
__global__ void k_lambda_table(Sched S, long long s_begin, long long count, double* out)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x)
        out[q] = ne_sched_lambda(S, s_begin + q);
}

// Atoms per CTA: the replica split in C equal parts, rounded up to whole
// cells so a CTA holds every basis site of its cells.
__host__ __device__ inline int atoms_per_cta(int n, int C, int nb)
{
    return (((n + C - 1) / C) + nb - 1) / nb * nb;
}

// NPT: the replicas have the barostat of the reversible-scaling path (a
// separate instantiation, so the fixed-box kernel carries none of it)
template <bool NPT>
__global__ void __launch_bounds__(THREADS, 1)
    k_cluster(const XRep* __restrict__ reps, const float4* __restrict__ st_vec, const float* __restrict__ st_dist,
              double* __restrict__ xg, double* __restrict__ vg, double* __restrict__ Wg, int* status, Sched S,
              long long s_begin, long long n_steps, Tables tab, unsigned long long* work, int k_lo,
              const double* __restrict__ lam_tab, double* __restrict__ wcum, double* __restrict__ boxes_out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int rep = blockIdx.x / C;
    auto peer = [&](int r) { return rank + r < C ? rank + r : rank + r - C; };  // (rank + r) mod C, 0 < r < C
    const int n = reps[rep].n, nb = reps[rep].nb, nx = reps[rep].nx, ny = reps[rep].ny, nz = reps[rep].nz;
    const int nst = reps[rep].st_cnt, M = reps[rep].st_margin;
    const int A_c = atoms_per_cta(n, C, nb);
    const int cells_c = A_c / nb;

    // ---- shared memory
    float4* s_u = (float4*)smem;                                  // [n] (u, F')
    float4* s_sv = s_u + n;                                       // [nb * nst] (r0_j - r0_i, code bits)
    float* s_sd = (float*)(s_sv + nb * nst);                      // [nb * nst] |r0_j - r0_i|
    // wrapped cell offsets: s_lxy[X * LY + Y] = ((X - M) mod nx * ny + (Y - M) mod ny) * nz,
    // s_lz[b2 * (nz + 2M) + Z] = (Z - M) mod nz + b2 * ncell, for X, Y, Z =
    // cell index + stencil offset + M and basis site b2 of the neighbour
    const int LY = ny + 2 * M;
    int* s_lxy = (int*)(s_sd + nb * nst);                         // [(nx + 2M) * LY]
    int* s_lz = s_lxy + (nx + 2 * M) * LY;                        // [nb][nz + 2M]
    unsigned short* s_K = (unsigned short*)(s_lz + nb * (nz + 2 * M));  // [4][NKT] scan bounds
    float* s_slotP = (float*)(((size_t)(s_K + 4 * NKT) + 15) & ~(size_t)15);  // [2][16][NSV]
    float* s_tot = s_slotP + 2 * 16 * NSV;                        // [NSV] replica totals
    // partial force, pair energy and rho of the second pair lane of each slot
    // (the first lane is the owning thread and keeps its part in registers)
    float4* s_f = (float4*)(((size_t)(s_tot + NSV) + 15) & ~(size_t)15);  // [SLOTS]
    float2* s_rho = (float2*)(s_f + SLOTS);                       // [SLOTS] double-float
    float* s_slotM = (float*)(s_rho + SLOTS);                     // [2][16] max |u| per CTA
    float* s_red = s_slotM + 32;                                  // [NWARP][NRED][2]
    unsigned* s_tm = (unsigned*)(s_red + NWARP * NRED * 2);       // [4] TMEM base address
    // barostat: the diagonal virial of the second pair lane of each slot, the
    // warps' double-float partials, every CTA's partial (written by the CTA
    // into all CTAs of the cluster) and the step's scale factors
    float4* s_vir = (float4*)(((size_t)(s_tm + 4) + 15) & ~(size_t)15);  // [SLOTS] (NPT)
    float* s_vred = (float*)(s_vir + (NPT ? SLOTS : 0));          // [NWARP][6] (NPT)
    float* s_vcta = s_vred + (NPT ? NWARP * 6 : 0);               // [16][6] (NPT)
    double* s_mu = (double*)(((size_t)(s_vcta + (NPT ? 16 * 6 : 0)) + 7) & ~(size_t)7);  // [4] (NPT)
    // spline intervals [k_lo, nk - 1) of phi, then of f: separate arrays, so
    // consecutive intervals fall in consecutive 16-byte bank groups
    float4* s_tabP = (float4*)(((size_t)(s_mu + (NPT ? 4 : 0)) + 15) & ~(size_t)15);  // [nk-1-k_lo]
    const int n_int = tab.nk - 1 - k_lo;  // intervals of the r grid held in shared memory
    float4* s_tabF = s_tabP + n_int;                                           // [nk-1-k_lo]
    {
        // the layout must fit the launch's dynamic shared memory (sized on the
        // host from the same counts); every CTA of a cluster takes the same
        // decision before touching shared memory
        unsigned dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        if ((size_t)((unsigned char*)(s_tabF + n_int) - smem) > (size_t)dyn) {
            if (threadIdx.x == 0) {
                ne_set_status(status, ST_EINVAL);
                ne_set_status(status + 1 + reps[rep].widx, ST_EINVAL);
            }
            return;
        }
    }

    for (int q = threadIdx.x; q < nb * nst; q += THREADS) {
        s_sv[q] = st_vec[reps[rep].st_off + q];
        s_sd[q] = st_dist[reps[rep].st_off + q];
    }
    for (int q = threadIdx.x; q < 2 * n_int; q += THREADS)
        ((q & 1) ? s_tabF : s_tabP)[q >> 1] = tab.pf32[2 * k_lo + q];
    // shared-memory copy of the replica is basis-major: entry b * ncell + cell
    const int ncell = n / nb;
    for (int q = threadIdx.x; q < (nx + 2 * M) * LY; q += THREADS)
        s_lxy[q] = ((((q / LY - M) % nx + nx) % nx) * ny + ((q % LY - M) % ny + ny) % ny) * nz;
    for (int q = threadIdx.x; q < nb * (nz + 2 * M); q += THREADS) {
        const int Z = q % (nz + 2 * M);
        s_lz[q] = ((Z - M) % nz + nz) % nz + (q / (nz + 2 * M)) * ncell;
    }

    // slots are basis-major inside a CTA: the atoms of a warp share a stencil
    // and their neighbours for one stencil entry lie close together
    auto slot_atom = [&](int sl) { return rank * A_c + (sl % cells_c) * nb + sl / cells_c; };
    // pair phases: two threads per slot, in different warps (warp w and
    // w + SLOTS/32 hold the same 32 slots, one for the even and one for the
    // odd stencil entries), so the 32 lanes of a warp read one stencil entry
    // and consecutive neighbours at each iteration
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
    // atom phases (density epilogue, BAOAB, noise): one thread per slot
    const int ta = slot_atom(threadIdx.x);
    const bool own = threadIdx.x < A_c && ta < n;
    const int tsu = own ? (ta % nb) * ncell + ta / nb : 0;  // its shared-memory entry
    const int own_warps = (A_c + 31) / 32;                   // warps holding owned atoms
    // site of the owned atom, component q, in fixed point
    auto site_fix = [&](int q) -> long long {
        const int b = ta % nb;
        int c = ta / nb;
        const int iz = c % nz;
        c /= nz;
        const int ic = q == 0 ? c / ny : (q == 1 ? c % ny : iz);
        return __double2ll_rn(reps[rep].cell[q] * (ic + reps[rep].basis[b][q]) * XSCALE);
    };
    const size_t gi = (size_t)(reps[rep].off + (own ? ta : 0)) * 3;
    // TMEM: warp 0 takes all columns for the CTA (returned after the step
    // loop, which every thread leaves at the same step)
    ne_tm_alloc(s_tm);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    cluster.sync();  // every CTA of the cluster has started: distributed shared memory is usable
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tm_base = *s_tm;
    const unsigned tm_w = tm_base + ((unsigned)(32 * ((threadIdx.x >> 5) & 3)) << 16) +
                          (unsigned)(CW * (threadIdx.x >> 7));  // this warp's lanes and columns
    const unsigned tm_j = tm_w + (unsigned)QMAX;                    // its neighbour-slot columns
    // the neighbour slots of this thread's first QMAX visits (entries past
    // the stencil, which no visit reaches, get slot 0); every atom of the
    // replica has a 16-byte entry in shared memory, so slots are < 2^16
#pragma unroll 1
    for (int q0 = 0; q0 < QMAX; q0 += FRB) {
        unsigned jw[FRB / 2];
#pragma unroll
        for (int h = 0; h < FRB / 2; ++h) {
            unsigned w2 = 0u;
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const int k = lane + TPA * (q0 + 2 * h + o);
                if (k < nst) {
                    const int code = __float_as_int(s_sv[stb + k].w);
                    w2 |= (unsigned)(s_lxy[sxy + (code & 0xffff)] + s_lz[sz + ((unsigned)code >> 16)]) << (16 * o);
                }
            }
            jw[h] = w2;
        }
        __syncwarp();
        ne_tm_st_u4(tm_j + (unsigned)(q0 / 2), jw);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    const float Dr = reps[rep].D;
    for (int q = threadIdx.x; q < nb * NKT; q += THREADS) {
        const int b = q / NKT, iq = q % NKT;
        // the last bin holds every real entry (the padding entries at the
        // end of each basis site's stencil have distance 1e30)
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

    // ---- state of the owned atom: displacement from its site in fixed point
    // (x * 2^32 - site * 2^32, registers), velocity and this step's normals
    // in FP32
    long long xr[3] = {0, 0, 0};
    float v[3] = {0, 0, 0}, u[3] = {0, 0, 0}, xi[3] = {0, 0, 0};
    int bad = 0;
    // the owned atom's spring, half-step factor and noise amplitude, and its
    // weights in the centre-of-mass sums: with species tables the spring sum
    // is sum_j k_j u_j and the noise sum sum_j m_j c2_j xi_j, and atom i takes
    // m_i / M of the first and 1 / M of the second (the mass-weighted
    // constraint); with one species the plain sums and means
    // (read from the replica table where they are used, so that they hold
    // no registers through the pair passes)
    const bool spc = reps[rep].nsp >= 2;
    const XRep& R_ = reps[rep];
    auto spq = [&]() { return spc && own ? (int)R_.sp[ta] : 0; };
    auto k_of = [&](int q) { return spc ? R_.kfs[q] : R_.kf; };
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
            const float4 uv = make_float4(u[0], u[1], u[2], 0.f);
            s_u[tsu] = uv;
            for (int r = 1; r < C; ++r) cluster.map_shared_rank(s_u, peer(r))[tsu] = uv;
            ne_normals32(ne_philox_block(reps[rep].seed, reps[rep].replica, (unsigned)S.stream, (unsigned)ta,
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
        cta_sum_bcast<ND_, NF_>(cluster, pd, pf, um, s_red, s_slotP + (s_begin & 1) * 16 * NSV,
                                s_slotM + (s_begin & 1) * 16, rank, C, own_warps);
    }

    unsigned n_cand = 0, n_pair = 0;  // work counters (stencil entries visited, pairs < r_c)
    const float rc2 = tab.rc2f, rmin2 = tab.rmin2f, inv_h = tab.inv_h_rf;
    const int nk = tab.nk;
    // first interval above both the shared-memory window's start and r_min:
    // pairs below it take the checked path of pass 1
    const int kchk = max(k_lo, (int)(sqrtf(rmin2) * inv_h) + 2);
    const float dt = (float)S.dt;
    const float rho_maxf = (float)tab.rho_max;
    const float ihr_hi = (float)tab.inv_h_rho, ihr_lo = (float)(tab.inv_h_rho - (double)ihr_hi);
    // rank 0, thread SLOTS (owns no atom) keeps the replica's two works in
    // registers and writes them back at the end, only if the replica
    // completed the range; likewise x and v below, so a replica that raised
    // an error keeps its state of step s_begin and can be rerun from there
    const bool wthread = rank == 0 && threadIdx.x == SLOTS;
    double Wacc[2] = {0.0, 0.0};
    if (wthread) {
        Wacc[0] = Wg[2 * reps[rep].widx];
        Wacc[1] = Wg[2 * reps[rep].widx + 1];
    }
    double UE_prev = 0.0;  // the work thread: U_E at the positions of the previous step
    // barostat: the box and the lattice sites scale by mu_tot per axis from
    // the call's start (every thread holds the same values: they come from
    // the same sums); stencil vectors are multiplied by it
    double mu_tot[3] = {1.0, 1.0, 1.0};
    float muf[3] = {1.f, 1.f, 1.f}, mu_min = 1.f;

#pragma unroll 1
    for (long long it = 0; it <= n_steps; ++it) {
        const long long s = s_begin + it;
        const bool fin = it == n_steps;
        cluster.sync();  // u of step s and the partial sums for step s visible everywhere

        // ---------------- replica sums for step s: warp q < NP_ sums quantity q
        // over the CTAs (lane r holds CTA r; a fixed shuffle tree, C <= 16),
        // the energies in double-float, the sums for the mean removal in FP32.
        // They are read after the next __syncthreads.  max |u| is needed at
        // once, so every warp forms it itself.
        float umax;
        {
            const int q = threadIdx.x >> 5, r = threadIdx.x & 31;
            const float* sp = s_slotP + (s & 1) * 16 * NSV;
            if (q < ND_) {
                dfl acc = r < C ? dfl{sp[r * NSV + 2 * q], sp[r * NSV + 2 * q + 1]} : dfl{0.f, 0.f};
#pragma unroll
                for (int o = 8; o > 0; o >>= 1)
                    acc = df_add(acc, {__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)});
                if (r == 0) {
                    s_tot[2 * q] = acc.hi;
                    s_tot[2 * q + 1] = acc.lo;
                }
            } else if (q < NP_) {
                float acc = r < C ? sp[r * NSV + ND_ + q] : 0.f;
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (r == 0) s_tot[ND_ + q] = acc;
            }
            float um = r < C ? s_slotM[(s & 1) * 16 + r] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, o));
            umax = um;
        }
        // an atom beyond the stencil range (or a non-finite displacement): the
        // replica's result is void, so its cluster stops here instead of
        // scanning the whole stencil for the rest of the range.  Every CTA of
        // the cluster holds the same slot values and leaves at the same step.
        bool out = !(umax <= reps[rep].D);
        if constexpr (NPT) {
            // the scaled stencil must still cover r_c + 2 max|u|, and the box
            // must keep two periodic images more than 2 r_c apart
            const float need = ((float)tab.r_c + 2.f * umax) / mu_min - (float)tab.r_c;
            out = out || !(need <= 2.f * reps[rep].D);
            for (int c = 0; c < 3; ++c)
                out = out || !(mu_tot[c] * reps[rep].box0[c] > 2.0 * tab.r_c + 1.2);
        }
        if (out) {
            if (threadIdx.x == 0) {
                const int e = isnan(umax) ? ST_ENAN : ST_ERANGE;
                ne_set_status(status, e);
                ne_set_status(status + 1 + reps[rep].widx, e);
            }
            break;
        }

        // ---------------- pass 1: density, pair forces and energy, f'(r)/r of
        // every visit to TMEM (pair threads); the F'(rho) terms of the forces
        // follow in pass 2
        const float4 ui = s_u[sui];
        int m = 0, K, nq;  // pairs inside r_c; this thread's scan bound; the warp's visits
        int ql = -1;       // this thread's last visit inside r_c
        float fx = 0.f, fy = 0.f, fz = 0.f, ep = 0.f;
        float vxx = 0.f, vyy = 0.f, vzz = 0.f;  // diagonal virial (barostat only)
        dfl rho = {0.f, 0.f};
        {
            // every entry with |r0_j - r0_i| < r_c + |u_i| + max |u| (two
            // bins of margin against rounding of the bin index)
            float c = sqrtf(ui.x * ui.x + ui.y * ui.y + ui.z * ui.z) + umax;
            if constexpr (NPT) c = ((float)tab.r_c + c) / mu_min - (float)tab.r_c;  // in lattice units
            K = valid ? (int)s_K[skb + min(NKT - 1, (int)(c * inv_dK) + 2)] : 0;
            // every thread of the warp visits up to the warp's largest bound,
            // in whole batches of FRB (TMEM stores are warp-wide): entries
            // past a thread's own bound lie outside r_c for it, and the
            // stencil's NE_STENCIL_PAD far padding entries keep the last
            // batch inside the array
            const int Kw = __reduce_max_sync(0xffffffffu, K);
            nq = Kw > lane ? ((Kw - lane + TPA - 1) / TPA + FRB - 1) / FRB * FRB : 0;
            // rho as an unnormalised double-float: the running FP32 sum rh and
            // the exact rounding error of each addition (TwoSum) summed in rl
            float rh = 0.f, rl = 0.f;
            // one stencil visit (entry e, neighbour slot j, visit index qv):
            // the pair's terms of rho, the forces and the energy; returns
            // f'(r)/r inside r_c, else 0
            auto visit = [&](float4 e, int j, int qv) -> float {
                const float4 uj = s_u[j];
                if constexpr (NPT) {
                    e.x *= muf[0];
                    e.y *= muf[1];
                    e.z *= muf[2];
                }
                const float dx = e.x + uj.x - ui.x, dy = e.y + uj.y - ui.y, dz = e.z + uj.z - ui.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                float fr = 0.f;
                if (r2 < rc2) {
                    const float irh = rsqrtf(r2) * inv_h;  // 1 / (r h)
                    const float t = r2 * irh;              // r / h >= 0
                    const int kk = min((int)t, nk - 2);
                    const float w = t - (float)kk;
                    // intervals below kchk (r < ~1 A: the shared-memory window
                    // starts there, and r_min lies below it) are rare: their
                    // own branch checks r_min and reads global memory
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
                    // phi and dphi/dw together (Horner with derivative)
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
            // the first QMAX visits: neighbour slots from TMEM, f'(r)/r to TMEM
            const int nqa = min(nq, QMAX);
#pragma unroll 1
            for (int q0 = 0; q0 < nqa; q0 += FRB) {
                unsigned jw[FRB / 2];
                __syncwarp();
                ne_tm_ld_u4(tm_j + (unsigned)(q0 / 2), jw);
                float frv[FRB];
#pragma unroll
                for (int uq = 0; uq < FRB; ++uq) {
                    const int k = lane + TPA * (q0 + uq);
                    frv[uq] = visit(s_sv[stb + k], (int)((jw[uq >> 1] >> (16 * (uq & 1))) & 0xffffu), q0 + uq);
                }
                __syncwarp();
                ne_tm_st(tm_w + (unsigned)q0, frv);
            }
            // visits past QMAX: slots from the wrapped-cell tables, f'(r)/r
            // recomputed in pass 2
#pragma unroll 1
            for (int q = nqa; q < nq; ++q) {
                const int k = lane + TPA * q;
                const float4 e = s_sv[stb + k];
                const int code = __float_as_int(e.w);
                (void)visit(e, s_lxy[sxy + (code & 0xffff)] + s_lz[sz + ((unsigned)code >> 16)], q);
            }
            __syncwarp();
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");  // the stores land before pass 2 loads
            nq = __reduce_max_sync(0xffffffffu, ql) + 1;  // pass 2 stops after the warp's last pair
            rho = {rh, rl};
            n_cand += valid ? (unsigned)nq : 0u;
            n_pair += valid ? (unsigned)m : 0u;
            ep *= 0.5f;  // each pair energy is shared by the two atoms
            if (valid && lane == 1) s_rho[slot] = make_float2(rho.hi, rho.lo);
        }
        __syncthreads();
        // embedding of the owned atom: F(rho), F'(rho)
        float emb = 0.f;
        if (own) {
            const float2 r1_ = s_rho[threadIdx.x];  // owner = pair lane 0 of its slot
            const dfl rr = df_add(rho, {r1_.x, r1_.y});
            if (!(rr.hi < rho_maxf)) bad |= ST_ERANGE;
            // offset in the interval from the double-float rho: the product
            // with the high part of 1/h exact inside the FMA, the low parts added
            const int kk = min(max((int)(rr.hi * ihr_hi), 0), nk - 2);
            const float w = fmaf(rr.hi, ihr_hi, -(float)kk) + (rr.hi * ihr_lo + rr.lo * ihr_hi);
            const float4 c = __ldg(&tab.F32[kk]);
            emb = c.x + w * (c.y + w * (c.z + w * c.w));
            const float dF = (c.y + w * (2.f * c.z + 3.f * w * c.w)) * tab.inv_h_rhof;
            s_u[tsu].w = dF;
            for (int r = 1; r < C; ++r) cluster.map_shared_rank(s_u, peer(r))[tsu].w = dF;
            if (!isfinite(emb)) bad |= ST_ENAN;
        }
        cluster.sync();  // F' visible everywhere

        // ---------------- pass 2: embedding forces (F'_i + F'_j) f'(r) r_ij / r
        // over the visits of pass 1, f'(r)/r from TMEM (pair threads)
        {
            const float dFi = s_u[sui].w;
            const int nqt = min(nq, QMAX);
#pragma unroll 1
            for (int q0 = 0; q0 < nqt; q0 += FRB) {
                float frv[FRB];
                unsigned jw[FRB / 2];
                __syncwarp();
                ne_tm_ld_f8u4(tm_w + (unsigned)q0, tm_j + (unsigned)(q0 / 2), frv, jw);
#pragma unroll
                for (int uq = 0; uq < FRB; ++uq) {
                    if (frv[uq] != 0.f) {  // inside r_c (f' vanishes only at r_c)
                        const int k = lane + TPA * (q0 + uq);
                        float4 e = s_sv[stb + k];
                        const int j = (int)((jw[uq >> 1] >> (16 * (uq & 1))) & 0xffffu);
                        const float4 uj = s_u[j];
                        if constexpr (NPT) {
                            e.x *= muf[0];
                            e.y *= muf[1];
                            e.z *= muf[2];
                        }
                        const float dx = e.x + uj.x - ui.x, dy = e.y + uj.y - ui.y, dz = e.z + uj.z - ui.z;
                        const float sc = (dFi + uj.w) * frv[uq];
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
            for (int q = QMAX; q < nq; ++q) {
                const int k = lane + TPA * q;
                float4 e = s_sv[stb + k];
                const int code = __float_as_int(e.w);
                const int j = s_lxy[sxy + (code & 0xffff)] + s_lz[sz + ((unsigned)code >> 16)];
                const float4 uj = s_u[j];
                if constexpr (NPT) {
                    e.x *= muf[0];
                    e.y *= muf[1];
                    e.z *= muf[2];
                }
                const float dx = e.x + uj.x - ui.x, dy = e.y + uj.y - ui.y, dz = e.z + uj.z - ui.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < rc2)) continue;
                const float irh = rsqrtf(r2) * inv_h;
                const float t = r2 * irh;
                const int kk = min((int)t, nk - 2);
                const float w = t - (float)kk;
                const float4 g = kk >= k_lo ? s_tabF[kk - k_lo] : __ldg(&tab.pf32[2 * kk + 1]);
                const float sc = (dFi + uj.w) * ((g.y + w * (2.f * g.z + 3.f * w * g.w)) * irh);
                fx += sc * dx;
                fy += sc * dy;
                fz += sc * dz;
                if constexpr (NPT) {
                    vxx -= 0.5f * sc * dx * dx;
                    vyy -= 0.5f * sc * dy * dy;
                    vzz -= 0.5f * sc * dz * dz;
                }
            }
            if (valid && lane == 1) s_f[slot] = make_float4(fx, fy, fz, ep);
            if constexpr (NPT)
                if (valid && lane == 1) s_vir[slot] = make_float4(vxx, vyy, vzz, 0.f);
        }
        __syncthreads();
        if constexpr (NPT) {
            // the diagonal virial of this CTA's atoms at x_s (double-float per
            // axis: a fixed warp tree, then warp 0 over the warps), written
            // into every CTA of the cluster before the arrive below
            const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
            dfl vd[3] = {};
            if (own) {
                const float4 v1 = s_vir[threadIdx.x];
                vd[0] = df_add({vxx, 0.f}, {v1.x, 0.f});
                vd[1] = df_add({vyy, 0.f}, {v1.y, 0.f});
                vd[2] = df_add({vzz, 0.f}, {v1.z, 0.f});
            }
            if (w < own_warps) {
                warp_df_sum<3>(vd);
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
                warp_df_sum<3>(t);
                if (l < C) {
                    float* d = cluster.map_shared_rank(s_vcta, l) + rank * 6;
                    for (int a3 = 0; a3 < 3; ++a3) {
                        d[2 * a3] = t[a3].hi;
                        d[2 * a3 + 1] = t[a3].lo;
                    }
                }
            }
        }

        // ---------------- fused step of the owned atom
        // This CTA has finished reading u and F' of step s: arrive on the
        // cluster barrier now, integrate, and wait only before writing u of
        // step s + 1 into the other CTAs, which by then have all finished
        // reading step s too (the integration hides the barrier's latency).
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
        if (wthread) {
            // work increment of step s - 1, (lambda_s - lambda_{s-1}) dH/dlambda(x_{s-1}),
            // by a thread that owns no atom (s_tot holds the sums of step s
            // until the next cluster barrier)
            const double U0 = (double)s_tot[2 * P_U0] + (double)s_tot[2 * P_U0 + 1];
            if (it > 0) {
                const long long sp = s - 1;
                const double g = S.path == 0 ? U0 - UE_prev : U0;
                int wslot = -1;
                if (sp >= S.t_eq && sp < S.t_eq + S.t_s) wslot = 0;
                else if (sp >= 2 * S.t_eq + S.t_s && sp < 2 * S.t_eq + 2 * S.t_s) wslot = 1;
                if (wslot >= 0) {
                    Wacc[wslot] += (lam_tab[it] - lam_tab[it - 1]) * g;
                    if (wcum) {  // cumulative work of the switch: [0] = 0, [k + 1] after its step k
                        const long long k = wslot == 0 ? sp - S.t_eq : sp - (2 * S.t_eq + S.t_s);
                        double* wc = wcum + (size_t)(2 * reps[rep].widx + wslot) * (size_t)(S.t_s + 1);
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
            if (own) {
                const float4 f1_ = s_f[threadIdx.x];
                const float4 f = make_float4(fx + f1_.x, fy + f1_.y, fz + f1_.z, ep + f1_.w);
                const float F0[3] = {f.x, f.y, f.z};
                const int q = spq();
                const float c1 = R_.c1f, kf = k_of(q);
                const float hdt = spc ? R_.hdts[q] : R_.hdt_mf, c2 = spc ? R_.c2fs[q] : R_.c2f;
                const float wcm = spc ? R_.mfs[q] * R_.invM : 0.f;
                const float invN = 1.f / (float)n;
                float mFE[3], mxi[3];
                for (int c = 0; c < 3; ++c) {
                    if (spc) {  // -m_i sum_j k_j u_j / M, and sum_j m_j c2_j xi_j / M
                        mFE[c] = S.fix_cm ? -wcm * s_tot[T_UX + c] : 0.f;
                        mxi[c] = S.fix_cm ? s_tot[T_XX + c] * reps[rep].invM : 0.f;
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
                        if (!(fabsf(dlt) < 0.25f)) bad |= ST_ERANGE;  // > 250 A/ps at 1 fs, or NaN
                        xr[c] += (long long)__float2int_rn(dlt * 4294967296.f);
                        u[c] = fix_to_float(xr[c]);
                    }
                    // normals of the next step
                    ne_normals32(ne_philox_block(reps[rep].seed, reps[rep].replica, (unsigned)S.stream,
                                                 (unsigned)ta, (unsigned long long)(s + 1)),
                                 xi);
                }
            }
            asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
            if constexpr (NPT) {
                if (!fin) {
                    // the barostat step after the second drift (reading A23): the
                    // replica's diagonal virial at x_s from the C CTA partials
                    // (fixed order), then one overdamped Langevin step of ln V
                    // (isotropic) or of each ln L_a, with the first (or a-th)
                    // normal of Philox stream 5 at (atom 0, step s)
                    if (threadIdx.x == 0) {
                        const XRep& Rb = reps[rep];
                        double Wa[3];
                        for (int a3 = 0; a3 < 3; ++a3) {
                            dfl acc = {0.f, 0.f};
                            for (int r = 0; r < C; ++r) acc = df_add(acc, {s_vcta[r * 6 + 2 * a3], s_vcta[r * 6 + 2 * a3 + 1]});
                            Wa[a3] = (double)acc.hi + (double)acc.lo;
                        }
                        const double V = mu_tot[0] * Rb.box0[0] * mu_tot[1] * Rb.box0[1] * mu_tot[2] * Rb.box0[2];
                        const double lam = lam_tab[it + 1], dtd = S.dt;
                        double z[3];
                        ne_normals64(ne_philox_block(Rb.seed, Rb.replica, (unsigned)STREAM_BARO, 0u,
                                                     (unsigned long long)s),
                                     z);
                        const double noise = sqrt(2.0 * Rb.kT * Rb.mp * dtd / V);
                        if (Rb.npt == 2) {
                            for (int a3 = 0; a3 < 3; ++a3) {
                                const double drive = (Rb.dof / 3.0 * Rb.kT + lam * Wa[a3]) / V - Rb.P0;
                                s_mu[a3] = exp(Rb.mp * drive * dtd + noise * z[a3]);
                            }
                        } else {
                            const double drive = (Rb.dof * Rb.kT + lam * (Wa[0] + Wa[1] + Wa[2])) / (3.0 * V) - Rb.P0;
                            s_mu[0] = s_mu[1] = s_mu[2] = exp((Rb.mp * drive * dtd + noise * z[0]) / 3.0);
                        }
                    }
                    __syncthreads();
                    for (int a3 = 0; a3 < 3; ++a3) {
                        const double mu = s_mu[a3];
                        mu_tot[a3] *= mu;
                        muf[a3] = (float)mu_tot[a3];
                        if (own) {  // positions scale about the origin: the displacement from the scaled site by mu
                            xr[a3] = __double2ll_rn(mu * (double)xr[a3]);
                            u[a3] = fix_to_float(xr[a3]);
                        }
                    }
                    mu_min = fminf(muf[0], fminf(muf[1], muf[2]));
                }
            }
            if (own) {
                if (!fin) {
                    const float4 uv = make_float4(u[0], u[1], u[2], 0.f);
                    s_u[tsu] = uv;
                    for (int r = 1; r < C; ++r) cluster.map_shared_rank(s_u, peer(r))[tsu] = uv;
                }
                const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                const int q = spq();
                const float kf = k_of(q), wxi = spc ? R_.mfs[q] * R_.c2fs[q] : 1.f;
                pd[P_UE] = {0.5f * kf * u2, 0.f};
                for (int c = 0; c < 3; ++c) {
                    pf[P_UX - ND_ + c] = spc ? kf * u[c] : u[c];
                    pf[P_XX - ND_ + c] = spc ? wxi * xi[c] : xi[c];
                }
                un = sqrtf(u2);
                for (int c = 0; c < 3; ++c)
                    if (!isfinite(v[c])) bad |= ST_ENAN;
            }
            if (!fin)
                cta_sum_bcast<ND_, NF_>(cluster, pd, pf, un, s_red, s_slotP + ((s + 1) & 1) * 16 * NSV,
                                        s_slotM + ((s + 1) & 1) * 16, rank, C, own_warps);
        }
    }
    ne_tm_free(tm_base);  // every warp is past its last TMEM access
    if (bad) {
        ne_set_status(status, bad);
        ne_set_status(status + 1 + reps[rep].widx, bad);
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
    // every CTA's error bits for this replica are in its status word once the
    // cluster has passed this barrier (the fence orders the atomics first);
    // after it no CTA touches another's shared memory, so each may finish alone
    __threadfence();
    cluster.sync();
    int* s_fail = (int*)s_slotM;  // no longer in use
    if (threadIdx.x == 0) *s_fail = atomicOr(status + 1 + reps[rep].widx, 0);
    __syncthreads();
    if (*s_fail == 0) {
        if (own)
            for (int c = 0; c < 3; ++c) {
                // the site of the atom in the (scaled) box
                const long long site = NPT ? __double2ll_rn(mu_tot[c] * (double)site_fix(c)) : site_fix(c);
                xg[gi + c] = (double)(xr[c] + site) / XSCALE;
                vg[gi + c] = (double)v[c];
            }
        if (wthread) {
            Wg[2 * reps[rep].widx] = Wacc[0];
            Wg[2 * reps[rep].widx + 1] = Wacc[1];
            if (NPT && boxes_out)
                for (int c = 0; c < 3; ++c) boxes_out[3 * reps[rep].widx + c] = mu_tot[c] * reps[rep].box0[c];
        }
    }
}

}  // namespace

namespace {

// The kernel's launch attributes on the current device, raised only (a launch
// needs at least its shared memory and, above 8 CTAs, non-portable cluster
// sizes): the driver is called only when a launch needs more than was set
// before on the device.
template <bool NPT>
cudaError_t cluster_attributes(int C, size_t smem)
{
    static std::atomic<int> smem_set[64];
    static std::atomic<int> nonportable_set[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool cached = dev >= 0 && dev < 64;
    if (!cached || smem_set[dev].load() < (int)smem) {
        e = cudaFuncSetAttribute(k_cluster<NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (cached) smem_set[dev].store((int)smem);
    }
    if (C > 8 && (!cached || !nonportable_set[dev].load())) {
        e = cudaFuncSetAttribute(k_cluster<NPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        if (cached) nonportable_set[dev].store(1);
    }
    return cudaSuccess;
}

}  // namespace

namespace ne {

// Bytes of everything but the spline tables; the tables take what is left.
size_t cluster_smem_bytes(int n_max, int nb_nst_max, int lut_max, bool npt)
{
    size_t b = sizeof(float4) * (size_t)n_max + (sizeof(float4) + sizeof(float)) * (size_t)nb_nst_max +
               sizeof(int) * (size_t)lut_max + sizeof(unsigned short) * 4 * NKT;
    b = (b + 15) & ~(size_t)15;
    b += sizeof(float) * (2 * 16 * NSV + NSV);
    b += 16;  // alignment of s_f
    b += sizeof(float4) * SLOTS + sizeof(float2) * SLOTS + sizeof(float) * (32 + NWARP * NRED * 2) +
         sizeof(unsigned) * 4;
    if (npt) {  // s_vir, s_vred, s_vcta, s_mu and their alignments
        b = ((b + 15) & ~(size_t)15) + sizeof(float4) * SLOTS + sizeof(float) * (NWARP * 6 + 16 * 6);
        b = ((b + 7) & ~(size_t)7) + sizeof(double) * 4;
    }
    return ((b + 15) & ~(size_t)15) + 16;  // + alignment of the tables
}

int cluster_size_for(int n, int nb)
{
    int C = (n + SLOTS - 1) / SLOTS;
    if (C < 1) C = 1;
    while (atoms_per_cta(n, C, nb) > SLOTS) ++C;
    return C;
}

int cluster_atoms_per_cta() { return SLOTS; }

int cluster_threads_per_atom() { return TPA; }

int cluster_atoms_for(int n, int C, int nb) { return atoms_per_cta(n, C, nb); }

int cluster_max_active(int C, size_t smem)
{
    // the barostat instantiation has the same shape; the fixed-box kernel
    // stands for both in this count
    if (cluster_attributes<false>(C, smem) != cudaSuccess) {
        (void)cudaGetLastError();  // not a launch error: clear it, the caller reports 0 clusters
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_cluster<false>, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_lambda_table(const Sched& S, long long s_begin, long long count, double* out, cudaStream_t st)
{
    k_lambda_table<<<(int)std::min<long long>((count + 255) / 256, 1024), 256, 0, st>>>(S, s_begin, count, out);
    return cudaGetLastError();
}

cudaError_t launch_cluster(const XRep* reps, int n_rep, int C, size_t smem, const float4* st_vec,
                           const float* st_dist, double* x, double* v, double* W, int* status, const Sched& S,
                           long long s_begin, long long n_steps, const Tables& tab, unsigned long long* work,
                           int k_lo, double* lam_tab, double* wcum, cudaStream_t st, bool npt, double* boxes_out)
{
    cudaError_t e = npt ? cluster_attributes<true>(C, smem) : cluster_attributes<false>(C, smem);
    if (e != cudaSuccess) return e;
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
    if (npt)
        return cudaLaunchKernelEx(&cfg, k_cluster<true>, reps, st_vec, st_dist, x, v, W, status, S, s_begin, n_steps,
                                  tab, work, k_lo, (const double*)lam_tab, wcum, boxes_out);
    return cudaLaunchKernelEx(&cfg, k_cluster<false>, reps, st_vec, st_dist, x, v, W, status, S, s_begin, n_steps,
                              tab, work, k_lo, (const double*)lam_tab, wcum, boxes_out);
}

}  // namespace ne
