// ne_eam.cu -- EAM kernels of libne.so: spline tables, pass 1 (density rho_i,
// embedding F(rho_i), F'(rho_i), per-step short neighbour list), pass 2
// (pair + embedding forces, pair energy, Langevin noise of the step, and the
// per-replica totals), and the backward pass for dU/dtheta.
//
// EAM energy (Sec. II.B, eq. H with U = EAM):
//   U = sum_{i<j} phi(r_ij) + sum_i F(rho_i),   rho_i = sum_{j != i} f(r_ij)
//   F_i = sum_j [phi'(r_ij) + (F'(rho_i) + F'(rho_j)) f'(r_ij)] (r_j - r_i) / r_ij
// The full neighbour list holds each pair twice, so every atom sums its own
// rho and force without atomics; the pair energy takes 1/2 per direction.
//
// Pair kernels give TPA consecutive lanes to one atom; lane l takes list
// entries l, l+TPA, ...  The lists are interleaved so that, for a fixed
// iteration, the lanes of a warp read consecutive words.
#include "ne_internal.cuh"

namespace {

// ------------------------------------------------------------ tables
// theta (value y, slope m per knot) -> per-interval cubic in u in [0, 1):
// p(u) = c0 + c1 u + c2 u^2 + c3 u^3 with c0 = y0, c1 = h m0,
// c2 = 3 (y1 - y0) - 2 h m0 - h m1, c3 = 2 (y0 - y1) + h m0 + h m1 -- the
// cubic Hermite interpolant written in the power basis.
__global__ void k_tables(const double* __restrict__ theta, int nk, double r_c, double rho_max,
                         float4* pf32, ned4* pf64, float4* F32, ned4* F64)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk - 1) return;
    for (int fn = 0; fn < 3; ++fn) {
        double h = (fn == 2 ? rho_max : r_c) / (nk - 1);
        const double* t = theta + (size_t)fn * nk * 2;
        double y0 = t[2 * k], m0 = t[2 * k + 1], y1 = t[2 * k + 2], m1 = t[2 * k + 3];
        ned4 c;
        c.x = y0;
        c.y = h * m0;
        c.z = 3.0 * (y1 - y0) - 2.0 * h * m0 - h * m1;
        c.w = 2.0 * (y0 - y1) + h * m0 + h * m1;
        float4 cf = make_float4((float)c.x, (float)c.y, (float)c.z, (float)c.w);
        if (fn < 2) {
            pf64[2 * k + fn] = c;
            pf32[2 * k + fn] = cf;
        } else {
            F64[k] = c;
            F32[k] = cf;
        }
    }
}

template <typename T>
struct V3 {
    T x, y, z;
};

// Position of atom i for the pair kernels: the wrapped FP32 copy (mixed) or
// the unwrapped FP64 state (FP64 path).
template <bool MIXED>
struct Pos;
template <>
struct Pos<true> {
    using R = float;
    static __device__ __forceinline__ V3<float> load(const DevBatch& B, int i)
    {
        float4 p = B.pos32[i];
        return {p.x, p.y, p.z};
    }
};
template <>
struct Pos<false> {
    using R = double;
    static __device__ __forceinline__ V3<double> load(const DevBatch& B, int i)
    {
        return {B.x[3 * i], B.x[3 * i + 1], B.x[3 * i + 2]};
    }
};

__device__ __forceinline__ float mi(float d, float L, float invL) { return d - L * rintf(d * invL); }
__device__ __forceinline__ double mi(double d, double L, double invL) { return d - L * rint(d * invL); }

template <typename R>
__device__ __forceinline__ R lane_sum(R v, int tpa)
{
    for (int o = tpa >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------ pass 1
// Mixed precision keeps GB300's FP64 pipe (1/64 of FP32) out of the pair
// loop and the sums: rho as an unnormalised double-float (the FP32 running
// sum and the TwoSum error of each addition), combined over the lanes and
// the block in double-float; the interval of F from the double-float rho
// with the high part of 1/h exact in the FMA (the crystal runner's forms).
template <bool MIXED, int TPA>
__global__ void __launch_bounds__(NE_TILE* TPA) k_density(DevBatch B)
{
    using R = typename Pos<MIXED>::R;
    __shared__ double red[NE_TILE * TPA];
    const int tile = blockIdx.x;
    const int rep = B.tile_rep[tile];
    const RepDev& P = B.rep[rep];
    const int local = threadIdx.x / TPA, lane = threadIdx.x % TPA;
    const int a = (tile - P.tile0) * NE_TILE + local;
    const bool valid = a < P.n;
    const int i = P.off + (valid ? a : 0);
    const R L0 = (R)P.L[0], L1 = (R)P.L[1], L2 = (R)P.L[2];
    const R iL0 = (R)P.invL[0], iL1 = (R)P.invL[1], iL2 = (R)P.invL[2];
    const R rc2 = MIXED ? (R)B.tab.rc2f : (R)(B.tab.r_c * B.tab.r_c);
    const R rmin2 = (R)(NE_RMIN * NE_RMIN);
    const R inv_h = MIXED ? (R)B.tab.inv_h_rf : (R)B.tab.inv_h_r;
    const int nk = B.tab.nk;
    const int cap = NE_SMAX / TPA;
    double rho = 0.0;           // FP64 path
    float rh = 0.f, rl = 0.f;   // mixed: running sum and TwoSum errors
    int m = 0, bad = 0;
    if (valid) {
        const V3<R> pi = Pos<MIXED>::load(B, i);
        if (!isfinite(pi.x) || !isfinite(pi.y) || !isfinite(pi.z)) bad |= ST_ENAN;
        const int cnt = min(B.ncnt[i], NE_NMAX);
        for (int k = lane; k < cnt; k += TPA) {
            const int jn = B.nbr[ne_nbr_index(k, i, B.n_tot, TPA)];
            const V3<R> pj = Pos<MIXED>::load(B, jn);
            R dx = mi(pj.x - pi.x, L0, iL0), dy = mi(pj.y - pi.y, L1, iL1), dz = mi(pj.z - pi.z, L2, iL2);
            R r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < rc2) {
                if (r2 < rmin2) bad |= ST_ERANGE;
                R r = sqrt(r2);
                R t = r * inv_h;
                int kk = min(max((int)t, 0), nk - 2);
                R u = t - (R)kk;
                R fr;
                if constexpr (MIXED) {
                    float4 c = __ldg(&B.tab.pf32[2 * kk + 1]);
                    fr = (R)(c.x + (float)u * (c.y + (float)u * (c.z + (float)u * c.w)));
                    const float s_ = rh + (float)fr, bp = s_ - rh;
                    rl += (rh - (s_ - bp)) + ((float)fr - bp);
                    rh = s_;
                } else {
                    ned4 c = B.tab.pf64[2 * kk + 1];
                    fr = (R)(c.x + (double)u * (c.y + (double)u * (c.z + (double)u * c.w)));
                    rho += (double)fr;
                }
                if (m < cap)
                    B.sl[(m * B.n_tot + i) * TPA + lane] = jn;
                else
                    bad |= ST_ENEIGH;
                ++m;
            }
        }
        B.scnt[i * TPA + lane] = min(m, cap);
    }
    dff rr = {0.f, 0.f};
    if constexpr (MIXED) {
        rr = dff_add({rh, 0.f}, {rl, 0.f});  // normalised
        for (int o = TPA >> 1; o > 0; o >>= 1)
            rr = dff_add(rr, {__shfl_xor_sync(0xffffffffu, rr.hi, o), __shfl_xor_sync(0xffffffffu, rr.lo, o)});
        rho = (double)rr.hi + (double)rr.lo;
    } else {
        rho = lane_sum(rho, TPA);
    }
    double Femb = 0.0;
    float Femb32 = 0.f;
    if (valid && lane == 0) {
        if (!(rho < B.tab.rho_max)) bad |= ST_ERANGE;
        double dF;
        if constexpr (MIXED) {
            const float ihr_hi = (float)B.tab.inv_h_rho, ihr_lo = (float)(B.tab.inv_h_rho - (double)ihr_hi);
            const int kk = min(max((int)(rr.hi * ihr_hi), 0), nk - 2);
            const float u = fmaf(rr.hi, ihr_hi, -(float)kk) + (rr.hi * ihr_lo + rr.lo * ihr_hi);
            float4 c = __ldg(&B.tab.F32[kk]);
            Femb32 = c.x + u * (c.y + u * (c.z + u * c.w));
            dF = (double)((c.y + u * (2.f * c.z + 3.f * u * c.w)) * (float)B.tab.inv_h_rho);
            float4 p = B.pos32[i];
            B.posF[i] = make_float4(p.x, p.y, p.z, (float)dF);
            if (!isfinite(Femb32)) bad |= ST_ENAN;
        } else {
            double t = rho * B.tab.inv_h_rho;
            int kk = min(max((int)t, 0), nk - 2);
            double u = t - kk;
            ned4 c = B.tab.F64[kk];
            Femb = c.x + u * (c.y + u * (c.z + u * c.w));
            dF = (c.y + u * (2.0 * c.z + 3.0 * u * c.w)) * B.tab.inv_h_rho;
            B.dF64[i] = dF;
        }
        if (B.rho) B.rho[i] = rho;
        if (!isfinite(Femb)) bad |= ST_ENAN;
    }
    if (bad) ne_set_status(B.status, bad);
    if constexpr (MIXED) {
        // the tile's embedding energy in double-float: a fixed tree in each
        // warp, then warp 0 over the warps in order
        const dff e = dff_warp_sum({Femb32, 0.f});
        float2* wsum = (float2*)red;
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
        if (l == 0) wsum[w] = make_float2(e.hi, e.lo);
        __syncthreads();
        if (w == 0) {
            const dff t = dff_warp_sum(l < nw ? dff{wsum[l].x, wsum[l].y} : dff{0.f, 0.f});
            if (l == 0) B.partA[(size_t)tile * NPA + PA_UEMB] = (double)t.hi + (double)t.lo;
        }
    } else {
        red[threadIdx.x] = Femb;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) B.partA[(size_t)tile * NPA + PA_UEMB] = red[0];
    }
}

// ------------------------------------------------------------ pass 2
// VIR: also the configurational virial (only runs with a barostat need it)
template <bool MIXED, int TPA, bool VIR>
__global__ void __launch_bounds__(NE_TILE* TPA)
    k_force(DevBatch B, Sched S, const long long* __restrict__ step_base, int j, int want_noise)
{
    using R = typename Pos<MIXED>::R;
    __shared__ double red[VIR ? 11 : 7][NE_TILE * TPA];
    __shared__ int s_last;
    const int tile = blockIdx.x;
    const int rep = B.tile_rep[tile];
    const RepDev& P = B.rep[rep];
    const int local = threadIdx.x / TPA, lane = threadIdx.x % TPA;
    const int a = (tile - P.tile0) * NE_TILE + local;
    const bool valid = a < P.n;
    const int i = P.off + (valid ? a : 0);
    const R L0 = (R)P.L[0], L1 = (R)P.L[1], L2 = (R)P.L[2];
    const R iL0 = (R)P.invL[0], iL1 = (R)P.invL[1], iL2 = (R)P.invL[2];
    const R inv_h = MIXED ? (R)B.tab.inv_h_rf : (R)B.tab.inv_h_r;
    const int nk = B.tab.nk;
    R fx = 0, fy = 0, fz = 0, ep = 0, vir = 0;  // vir: -(1/2) sum_j r dU/dr (the pair's half)
    R vxx = 0, vyy = 0, vzz = 0;                  // its diagonal: -(1/2) sum_j r_a^2 / r dU/dr
    if (valid) {
        V3<R> pi;
        R dFi;
        if constexpr (MIXED) {
            float4 p = B.posF[i];
            pi.x = (R)p.x;
            pi.y = (R)p.y;
            pi.z = (R)p.z;
            dFi = (R)p.w;
        } else {
            pi = Pos<false>::load(B, i);
            dFi = (R)B.dF64[i];
        }
        const int m = B.scnt[i * TPA + lane];
        for (int q = 0; q < m; ++q) {
            const int jn = B.sl[(q * B.n_tot + i) * TPA + lane];
            V3<R> pj;
            R dFj;
            if constexpr (MIXED) {
                float4 p = B.posF[jn];
                pj.x = (R)p.x;
                pj.y = (R)p.y;
                pj.z = (R)p.z;
                dFj = (R)p.w;
            } else {
                pj = Pos<false>::load(B, jn);
                dFj = (R)B.dF64[jn];
            }
            R dx = mi(pj.x - pi.x, L0, iL0), dy = mi(pj.y - pi.y, L1, iL1), dz = mi(pj.z - pi.z, L2, iL2);
            R r2 = dx * dx + dy * dy + dz * dz;
            R r = sqrt(r2);
            R ir = (R)1 / r;
            R t = r * inv_h;
            int kk = min(max((int)t, 0), nk - 2);
            R u = t - (R)kk;
            R phi, dphi, df;
            if constexpr (MIXED) {
                float4 c = __ldg(&B.tab.pf32[2 * kk]);
                float4 g = __ldg(&B.tab.pf32[2 * kk + 1]);
                float uf = (float)u;
                phi = c.x + uf * (c.y + uf * (c.z + uf * c.w));
                dphi = (c.y + uf * (2.f * c.z + 3.f * uf * c.w)) * (float)inv_h;
                df = (g.y + uf * (2.f * g.z + 3.f * uf * g.w)) * (float)inv_h;
            } else {
                ned4 c = B.tab.pf64[2 * kk];
                ned4 g = B.tab.pf64[2 * kk + 1];
                phi = c.x + u * (c.y + u * (c.z + u * c.w));
                dphi = (c.y + u * (2.0 * c.z + 3.0 * u * c.w)) * inv_h;
                df = (g.y + u * (2.0 * g.z + 3.0 * u * g.w)) * inv_h;
            }
            R s = (dphi + (dFi + dFj) * df) * ir;
            fx += s * dx;
            fy += s * dy;
            fz += s * dz;
            ep += (R)0.5 * phi;
            if constexpr (VIR) {
                vir -= (R)0.5 * s * r2;
                vxx -= (R)0.5 * s * dx * dx;
                vyy -= (R)0.5 * s * dy * dy;
                vzz -= (R)0.5 * s * dz * dz;
            }
        }
    }
    fx = lane_sum(fx, TPA);
    fy = lane_sum(fy, TPA);
    fz = lane_sum(fz, TPA);
    // the tile's totals: pair energy and virials from every lane's partial,
    // forces and noise from the atom's lane 0
    constexpr int NQ = VIR ? 11 : 7;
    double v[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    v[0] = (double)ep;
    if constexpr (VIR) {
        v[7] = (double)vir;
        v[8] = (double)vxx;
        v[9] = (double)vyy;
        v[10] = (double)vzz;
    }
    if (valid && lane == 0) {
        if constexpr (MIXED) {
            B.f32[i] = make_float4((float)fx, (float)fy, (float)fz, 0.f);
        } else {
            B.f64[3 * i] = (double)fx;
            B.f64[3 * i + 1] = (double)fy;
            B.f64[3 * i + 2] = (double)fz;
        }
        v[1] = (double)fx;
        v[2] = (double)fy;
        v[3] = (double)fz;
        if (want_noise) {
            const long long s = *step_base + j;
            uint4 w = ne_philox_block(P.seed, P.replica, (unsigned)S.stream, (unsigned)a,
                                      (unsigned long long)s);
            if constexpr (MIXED) {
                float z[3];
                ne_normals32(w, z);
                B.xi32[3 * i] = z[0];
                B.xi32[3 * i + 1] = z[1];
                B.xi32[3 * i + 2] = z[2];
                v[4] = z[0];
                v[5] = z[1];
                v[6] = z[2];
            } else {
                double z[3];
                ne_normals64(w, z);
                B.xi64[3 * i] = z[0];
                B.xi64[3 * i + 1] = z[1];
                B.xi64[3 * i + 2] = z[2];
                v[4] = z[0];
                v[5] = z[1];
                v[6] = z[2];
            }
            if (P.nsp) {  // the velocity increments' momentum: sum m_j c2_j xi_j
                const int q = P.sp[a];
                const double wq = P.ms[q] * P.c2s[q];
                v[4] *= wq;
                v[5] *= wq;
                v[6] *= wq;
            }
        }
    }
    double tq[11];  // the totals, in thread 0
    if constexpr (MIXED) {
        // FP32 values summed as double-float (GB300's FP64 pipe kept out): a
        // fixed tree in each warp, then warp 0 over the warps in order
        float2* wsum = (float2*)&red[0][0];  // [NQ][warps]
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int q = 0; q < NQ; ++q) {
            const dff t = dff_warp_sum({(float)v[q], 0.f});
            if (l == 0) wsum[q * nw + w] = make_float2(t.hi, t.lo);
        }
        __syncthreads();
        if (w == 0)
            for (int q = 0; q < NQ; ++q) {
                const dff t = dff_warp_sum(l < nw ? dff{wsum[q * nw + l].x, wsum[q * nw + l].y} : dff{0.f, 0.f});
                tq[q] = (double)t.hi + (double)t.lo;
            }
    } else {
        for (int q = 0; q < NQ; ++q) red[q][threadIdx.x] = v[q];
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w)
                for (int q = 0; q < NQ; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
            __syncthreads();
        }
        for (int q = 0; q < NQ; ++q) tq[q] = red[q][0];
    }
    if (threadIdx.x == 0) {
        double* pa = B.partA + (size_t)tile * NPA;
        pa[PA_UPAIR] = tq[0];
        pa[PA_F0X] = tq[1];
        pa[PA_F0Y] = tq[2];
        pa[PA_F0Z] = tq[3];
        pa[PA_XIX] = tq[4];
        pa[PA_XIY] = tq[5];
        pa[PA_XIZ] = tq[6];
        pa[PA_VIR] = VIR ? tq[VIR ? 7 : 0] : 0.0;
        pa[PA_VXX] = VIR ? tq[VIR ? 8 : 0] : 0.0;
        pa[PA_VYY] = VIR ? tq[VIR ? 9 : 0] : 0.0;
        pa[PA_VZZ] = VIR ? tq[VIR ? 10 : 0] : 0.0;
        __threadfence();
        unsigned prev = atomicAdd(&B.tile_done[rep], 1u);
        s_last = (prev == (unsigned)P.ntile - 1u);
    }
    __syncthreads();
    if (s_last) {
        // Last tile of this replica: fixed-order sums of every tile partial,
        // one warp per quantity (a replica of 65,536 atoms has 1,024 tiles)
        __threadfence();
        const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int q = w; q < NTOT; q += nw) {
            const double acc = q < NPA ? ne_warp_tile_sum(B.partA, NPA, q, P.tile0, P.ntile)
                                       : ne_warp_tile_sum(B.partB, NPB, q - NPA, P.tile0, P.ntile);
            if ((threadIdx.x & 31) == 0) B.tot[(size_t)rep * NTOT + q] = acc;
        }
        if (threadIdx.x == 0) B.tile_done[rep] = 0u;
    }
}

// ------------------------------------------------------------ backward
// dU/dtheta: U is linear in the phi and F knot parameters; the f knots enter
// through rho_i, weighted by F'(rho_i).  The FP64 kernel walks the full
// list, each pair from both atoms: phi takes 1/2 per direction, f takes
// F'(rho_i) from atom i's side only; the mixed kernel takes each pair once,
// phi whole and f with F'(rho_i) + F'(rho_j) (half the bin atomics).
// Hermite basis on interval k with u in [0, 1) and spacing h:
// (h00, h h10, h01, h h11) multiply (y_k, m_k, y_{k+1}, m_{k+1}).
__device__ __forceinline__ void hermite_w(double u, double h, double w[4])
{
    double u2 = u * u, u3 = u2 * u;
    w[0] = 2 * u3 - 3 * u2 + 1;
    w[1] = (u3 - 2 * u2 + u) * h;
    w[2] = -2 * u3 + 3 * u2;
    w[3] = (u3 - u2) * h;
}

__device__ __forceinline__ void hermite_wf(float u, float h, float w[4])
{
    float u2 = u * u, u3 = u2 * u;
    w[0] = 2 * u3 - 3 * u2 + 1;
    w[1] = (u3 - 2 * u2 + u) * h;
    w[2] = -2 * u3 + 3 * u2;
    w[3] = (u3 - u2) * h;
}

// The weight gE of a backward launch: the host's value, or, inside a run,
// gw[step - s_off] read on the device for step = *ctr + j, so a captured
// graph replays the per-step weights.  A zero weight skips the launch's work.
struct BwdWeight {
    double gE;
    const double* gw;
    const long long* ctr;
    int j;
    long long s_off;
};

__device__ __forceinline__ double bwd_weight(const BwdWeight& W)
{
    return W.gw ? W.gw[*W.ctr + W.j - W.s_off] : W.gE;
}

// Mixed precision.  phi and f (8 adds a pair): FP32 basis weights, the
// slope weights without their factor h, into per-block FP32 bins in shared
// memory (a block is the SM's only one, with BWD_THREADS threads working on
// BWD_THREADS / (NE_TILE * TPA) tiles at once), flushed to global memory and
// summed over the blocks in FP64 by k_bins_reduce.  F (4 adds an atom, on the
// few intervals a crystal's densities fall in): one global array of 64-bit
// fixed-point bins, 2^-32 per unit, cleared before the launch, the lanes of a
// warp on one interval adding their weights before one integer atomic add
// each (exact, so the order of the adds does not matter).
// (64-bit shared-memory bins for phi and f too made the whole gradient
// bitwise reproducible but the kernel 1.7x slower: 64-bit shared atomics are
// slower than FP32 ones on this SM.)  Bins are function-major, then
// value/slope, then knot (bin_index), so a warp's adds at random intervals
// spread over the shared-memory banks.
constexpr int BWD_THREADS = 1024;
constexpr double BWD_FIX = 4294967296.0;  // 2^32

// bin of knot parameter (function fn, knot k, c = 0 value / 1 slope); the
// knot parameters theta themselves are [fn][k][c]
__host__ __device__ __forceinline__ int bin_index(int fn, int k, int c, int nk) { return (2 * fn + c) * nk + k; }

// The global bins buffer: the 2 nk 64-bit F bins first (cleared by each
// launch), then each block's 4 nk FP32 phi/f bins
__host__ __device__ __forceinline__ size_t bwd_block_bytes(int nk) { return sizeof(float) * 4 * (size_t)nk; }
__host__ __device__ __forceinline__ size_t bwd_f_bytes(int nk) { return sizeof(unsigned long long) * 2 * (size_t)nk; }

template <int TPA>
__global__ void __launch_bounds__(BWD_THREADS, 1)
    k_backward_mixed(DevBatch B, unsigned char* __restrict__ bins, BwdWeight W)
{
    constexpr int TPB = NE_TILE * TPA, TILES = BWD_THREADS / TPB;
    if (bwd_weight(W) == 0.0) return;
    extern __shared__ __align__(16) unsigned char sbytes[];
    const int nk = B.tab.nk;
    float* const spf = (float*)sbytes;  // [4 nk] phi, f
    unsigned long long* const gF = (unsigned long long*)bins;  // global F bins: F's bin_index - 4 nk
    for (int q = threadIdx.x; q < 4 * nk; q += blockDim.x) spf[q] = 0.f;
    __syncthreads();
    const float inv_h = B.tab.inv_h_rf;
    const float fix = (float)BWD_FIX;
    const int sub = threadIdx.x / TPB, tt = threadIdx.x % TPB;
    for (int tile = blockIdx.x * TILES + sub; tile < B.n_tiles; tile += gridDim.x * TILES) {
        const int rep = B.tile_rep[tile];
        const RepDev& P = B.rep[rep];
        const int local = tt / TPA, lane = tt % TPA;
        const int a = (tile - P.tile0) * NE_TILE + local;
        if (a < P.n) {
            const int i = P.off + a;
            const float Lf0 = (float)P.L[0], Lf1 = (float)P.L[1], Lf2 = (float)P.L[2];
            const float iL0 = (float)P.invL[0], iL1 = (float)P.invL[1], iL2 = (float)P.invL[2];
            float4 pi = B.posF[i];
            const float dFi = pi.w;
            const int m = B.scnt[i * TPA + lane];
            for (int q = 0; q < m; ++q) {
                const int jn = B.sl[(q * B.n_tot + i) * TPA + lane];
                // each pair once, from its lower-index atom: the short lists
                // are symmetric (the minimum-image difference of j and i is
                // the exact negative of that of i and j, so both atoms see
                // the same r), and the pair adds phi's basis weights whole
                // and f's times F'_i + F'_j
                if (jn < i) continue;
                float4 pj = B.posF[jn];
                float dx = mi(pj.x - pi.x, Lf0, iL0), dy = mi(pj.y - pi.y, Lf1, iL1),
                      dz = mi(pj.z - pi.z, Lf2, iL2);
                float r = sqrtf(dx * dx + dy * dy + dz * dz);
                float t = r * inv_h;
                int kk = min(max((int)t, 0), nk - 2);
                float w[4];
                hermite_wf(t - (float)kk, 1.f, w);  // slope weights without h
                // w = (y_kk, m_kk / h, y_kk+1, m_kk+1 / h) weights
                const float dFij = dFi + pj.w;
                for (int c = 0; c < 4; ++c) {
                    atomicAdd(spf + bin_index(0, kk + (c >> 1), c & 1, nk), w[c]);
                    atomicAdd(spf + bin_index(1, kk + (c >> 1), c & 1, nk), dFij * w[c]);
                }
            }
            if (lane == 0) {
                double t = B.rho[i] * B.tab.inv_h_rho;
                int kk = min(max((int)t, 0), nk - 2);
                float w[4];
                hermite_wf((float)(t - kk), 1.f, w);  // slope weights without h
                // the densities of a crystal fall in a few F intervals, so the
                // atoms of a warp mostly share one: the lanes on an interval
                // add their fixed-point weights and one of them does the
                // atomic adds, instead of all of them contending for the bins
                long long wq[4];
                for (int c = 0; c < 4; ++c) wq[c] = __float2ll_rn(w[c] * fix);
                const unsigned act = __activemask();
                const unsigned grp = __match_any_sync(act, kk);
                long long g[4] = {0, 0, 0, 0};
                for (unsigned rest = act; rest; rest &= rest - 1) {
                    const int src = __ffs(rest) - 1;
                    for (int c = 0; c < 4; ++c) {
                        const long long v = __shfl_sync(act, wq[c], src);
                        if (grp & (1u << src)) g[c] += v;
                    }
                }
                if ((int)(threadIdx.x & 31) == __ffs(grp) - 1)
                    for (int c = 0; c < 4; ++c)
                        atomicAdd(gF + (bin_index(2, kk + (c >> 1), c & 1, nk) - 4 * nk), (unsigned long long)g[c]);
            }
        }
    }
    __syncthreads();
    float* opf = (float*)(bins + bwd_f_bytes(nk) + (size_t)blockIdx.x * bwd_block_bytes(nk));
    for (int q = threadIdx.x; q < 4 * nk; q += blockDim.x) opf[q] = spf[q];
}

// gtheta[q] (+)= gE * (the bin total of parameter q): a block of BR_COLS x
// BR_SEG threads takes BR_COLS knot parameters.  phi and f: segment g adds
// the blocks b = g, g + BR_SEG, ... in FP64, then the segments in a fixed
// order; F: the global fixed-point bin (2^-32), cleared before each backward
// launch.  A slope total is scaled by h once.
constexpr int BR_COLS = 32, BR_SEG = 8;

__global__ void __launch_bounds__(BR_COLS* BR_SEG)
    k_bins_reduce(unsigned char* __restrict__ bins, int n_blocks, int nk, double h_r, double h_rho, BwdWeight W,
                  double* __restrict__ gtheta, int accumulate)
{
    __shared__ double part[BR_SEG][BR_COLS];
    const int nb = 6 * nk;
    const int col = threadIdx.x % BR_COLS, g = threadIdx.x / BR_COLS;
    const int q = blockIdx.x * BR_COLS + col;  // knot parameter [fn][k][c]
    const double gE = bwd_weight(W);
    if (gE == 0.0) return;
    const size_t stride = bwd_block_bytes(nk);
    const int fn = q / (2 * nk), k = (q % (2 * nk)) >> 1, c = q & 1;
    const int bq = bin_index(fn, k, c, nk);
    double acc = 0.0;
    if (q < nb && fn < 2)
        for (int b = g; b < n_blocks; b += BR_SEG)
            acc += (double)((const float*)(bins + bwd_f_bytes(nk) + (size_t)b * stride))[bq];
    part[g][col] = acc;
    __syncthreads();
    if (g == 0 && q < nb) {
        double t = 0.0;
        if (fn < 2) {
            for (int h = 0; h < BR_SEG; ++h) t += part[h][col];
        } else {
            t = (double)(long long)((const unsigned long long*)bins)[bq - 4 * nk] * (1.0 / BWD_FIX);
        }
        if (c) t *= fn < 2 ? h_r : h_rho;
        gtheta[q] = (accumulate ? gtheta[q] : 0.0) + gE * t;
    }
}

// FP64 path: FP64 basis weights added straight into gtheta (pre-zeroed) with
// FP64 atomics, scaled by gE.
template <int TPA>
__global__ void __launch_bounds__(NE_TILE* TPA) k_backward_fp64(DevBatch B, BwdWeight W, double* gtheta)
{
    const double gE = bwd_weight(W);
    if (gE == 0.0) return;
    const int nk = B.tab.nk;
    const int tile = blockIdx.x;
    const int rep = B.tile_rep[tile];
    const RepDev& P = B.rep[rep];
    const int local = threadIdx.x / TPA, lane = threadIdx.x % TPA;
    const int a = (tile - P.tile0) * NE_TILE + local;
    if (a >= P.n) return;
    const int i = P.off + a;
    const double dFi = B.dF64[i];
    const double xi = B.x[3 * i], yi = B.x[3 * i + 1], zi = B.x[3 * i + 2];
    const int m = B.scnt[i * TPA + lane];
    for (int q = 0; q < m; ++q) {
        const int jn = B.sl[(q * B.n_tot + i) * TPA + lane];
        double dx = mi(B.x[3 * jn] - xi, P.L[0], P.invL[0]);
        double dy = mi(B.x[3 * jn + 1] - yi, P.L[1], P.invL[1]);
        double dz = mi(B.x[3 * jn + 2] - zi, P.L[2], P.invL[2]);
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        double t = r * B.tab.inv_h_r;
        int kk = min(max((int)t, 0), nk - 2);
        double w[4];
        hermite_w(t - kk, B.tab.h_r, w);
        for (int c = 0; c < 4; ++c) {
            atomicAdd(gtheta + 2 * kk + c, gE * 0.5 * w[c]);
            atomicAdd(gtheta + 2 * nk + 2 * kk + c, gE * dFi * w[c]);
        }
    }
    if (lane == 0) {
        double t = B.rho[i] * B.tab.inv_h_rho;
        int kk = min(max((int)t, 0), nk - 2);
        double w[4];
        hermite_w(t - kk, B.tab.h_rho, w);
        for (int c = 0; c < 4; ++c) atomicAdd(gtheta + 4 * nk + 2 * kk + c, gE * w[c]);
    }
}

// Configurational virial for the pressure (Sec. III.A: the lattice
// parameter at zero pressure): W = sum_{i<j} r_ij . F_ij = -sum_{i<j} r dU/dr
// with dU/dr = phi'(r) + (F'_i + F'_j) f'(r), in FP64 after an FP64 density
// pass.  Each pair is seen from both atoms, so every visit adds half.  Tile
// partials in fixed order; P = (N_dof k_B T + W) / (3 V).
template <int TPA>
__global__ void __launch_bounds__(NE_TILE* TPA) k_virial(DevBatch B)
{
    __shared__ double red[NE_TILE * TPA];
    const int nk = B.tab.nk;
    const int tile = blockIdx.x;
    const RepDev& P = B.rep[B.tile_rep[tile]];
    const int local = threadIdx.x / TPA, lane = threadIdx.x % TPA;
    const int a = (tile - P.tile0) * NE_TILE + local;
    double w = 0.0;
    if (a < P.n) {
        const int i = P.off + a;
        const V3<double> pi = Pos<false>::load(B, i);
        const double dFi = B.dF64[i];
        const int m = B.scnt[i * TPA + lane];
        for (int q = 0; q < m; ++q) {
            const int jn = B.sl[(q * B.n_tot + i) * TPA + lane];
            const V3<double> pj = Pos<false>::load(B, jn);
            const double dx = mi(pj.x - pi.x, P.L[0], P.invL[0]);
            const double dy = mi(pj.y - pi.y, P.L[1], P.invL[1]);
            const double dz = mi(pj.z - pi.z, P.L[2], P.invL[2]);
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            const double t = r * B.tab.inv_h_r;
            const int kk = min(max((int)t, 0), nk - 2);
            const double u = t - kk;
            const ned4 c = B.tab.pf64[2 * kk];
            const ned4 g = B.tab.pf64[2 * kk + 1];
            const double dphi = (c.y + u * (2.0 * c.z + 3.0 * u * c.w)) * B.tab.inv_h_r;
            const double df = (g.y + u * (2.0 * g.z + 3.0 * u * g.w)) * B.tab.inv_h_r;
            w -= 0.5 * (dphi + (dFi + B.dF64[jn]) * df) * r;
        }
    }
    red[threadIdx.x] = w;
    __syncthreads();
    for (int h = NE_TILE * TPA / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) B.partA[tile] = red[0];
}

// Sum of n tile partials in tile order (one thread: deterministic).
__global__ void k_sum_tiles(const double* part, int n, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double acc = 0.0;
        for (int t = 0; t < n; ++t) acc += part[t];
        *out = acc;
    }
}

template <bool MIXED>
void density_tpa(const DevBatch& B, cudaStream_t st)
{
    dim3 g(B.n_tiles);
    switch (B.tpa) {
    case 1: k_density<MIXED, 1><<<g, NE_TILE * 1, 0, st>>>(B); break;
    case 2: k_density<MIXED, 2><<<g, NE_TILE * 2, 0, st>>>(B); break;
    case 4: k_density<MIXED, 4><<<g, NE_TILE * 4, 0, st>>>(B); break;
    default: k_density<MIXED, 8><<<g, NE_TILE * 8, 0, st>>>(B); break;
    }
}

template <bool MIXED>
void force_tpa(const DevBatch& B, const Sched& S, const long long* sb, int j, int wn,
               cudaStream_t st)
{
    dim3 g(B.n_tiles);
    if (B.npt_any) {
        switch (B.tpa) {
        case 1: k_force<MIXED, 1, true><<<g, NE_TILE * 1, 0, st>>>(B, S, sb, j, wn); break;
        case 2: k_force<MIXED, 2, true><<<g, NE_TILE * 2, 0, st>>>(B, S, sb, j, wn); break;
        case 4: k_force<MIXED, 4, true><<<g, NE_TILE * 4, 0, st>>>(B, S, sb, j, wn); break;
        default: k_force<MIXED, 8, true><<<g, NE_TILE * 8, 0, st>>>(B, S, sb, j, wn); break;
        }
        return;
    }
    switch (B.tpa) {
    case 1: k_force<MIXED, 1, false><<<g, NE_TILE * 1, 0, st>>>(B, S, sb, j, wn); break;
    case 2: k_force<MIXED, 2, false><<<g, NE_TILE * 2, 0, st>>>(B, S, sb, j, wn); break;
    case 4: k_force<MIXED, 4, false><<<g, NE_TILE * 4, 0, st>>>(B, S, sb, j, wn); break;
    default: k_force<MIXED, 8, false><<<g, NE_TILE * 8, 0, st>>>(B, S, sb, j, wn); break;
    }
}

}  // namespace

namespace ne {

void launch_tables(const double* theta, int nk, double r_c, double rho_max, float4* pf32,
                   ned4* pf64, float4* F32, ned4* F64, cudaStream_t st)
{
    int n = nk - 1;
    k_tables<<<(n + 255) / 256, 256, 0, st>>>(theta, nk, r_c, rho_max, pf32, pf64, F32, F64);
}

void launch_density(const DevBatch& B, bool mixed, const long long*, int, cudaStream_t st)
{
    if (mixed)
        density_tpa<true>(B, st);
    else
        density_tpa<false>(B, st);
}

void launch_force(const DevBatch& B, const Sched& S, bool mixed, const long long* step_base, int j,
                  int want_noise, cudaStream_t st)
{
    if (mixed)
        force_tpa<true>(B, S, step_base, j, want_noise, st);
    else
        force_tpa<false>(B, S, step_base, j, want_noise, st);
}

cudaError_t prepare_backward(const DevBatch& B)
{
    const int smem = (int)bwd_block_bytes(B.tab.nk);
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    switch (B.tpa) {
    case 1: return cudaFuncSetAttribute(k_backward_mixed<1>, a, smem);
    case 2: return cudaFuncSetAttribute(k_backward_mixed<2>, a, smem);
    case 4: return cudaFuncSetAttribute(k_backward_mixed<4>, a, smem);
    default: return cudaFuncSetAttribute(k_backward_mixed<8>, a, smem);
    }
}

size_t backward_block_bytes(int nk) { return bwd_block_bytes(nk); }

size_t backward_bins_bytes(int nk, int n_blocks)
{
    return bwd_f_bytes(nk) + bwd_block_bytes(nk) * (size_t)n_blocks;
}

bool backward_fits(int nk)
{
    int dev = 0, smem_max = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return bwd_block_bytes(nk) <= (size_t)smem_max;
}

int backward_bin_blocks(const DevBatch& B)
{
    // one block per SM (the bins fill its shared memory), no more than the
    // tiles need
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
            (void)cudaGetLastError();
            sms = 148;
        }
    }
    const int per = BWD_THREADS / (NE_TILE * (B.tpa < 1 ? 1 : B.tpa));
    const int need = (B.n_tiles + per - 1) / per;
    const int nb = need < sms ? need : sms;
    return nb < 1 ? 1 : nb;
}

void launch_virial(const DevBatch& B, double* out, cudaStream_t st)
{
    dim3 g(B.n_tiles);
    switch (B.tpa) {
    case 1: k_virial<1><<<g, NE_TILE * 1, 0, st>>>(B); break;
    case 2: k_virial<2><<<g, NE_TILE * 2, 0, st>>>(B); break;
    case 4: k_virial<4><<<g, NE_TILE * 4, 0, st>>>(B); break;
    default: k_virial<8><<<g, NE_TILE * 8, 0, st>>>(B); break;
    }
    k_sum_tiles<<<1, 32, 0, st>>>(B.partA, B.n_tiles, out);
}

void launch_backward(const DevBatch& B, bool mixed, double gE, double* gx, double* gtheta,
                     float* bins, int n_bin_blocks, bool accumulate, cudaStream_t st, const double* gw,
                     const long long* ctr, int j, long long s_off, bool set_attr)
{
    (void)gx;
    const int nk = B.tab.nk;
    const int nb = 3 * nk * 2;
    const BwdWeight W{gE, gw, ctr, j, s_off};
    if (mixed) {
        size_t smem = bwd_block_bytes(nk);
        cudaMemsetAsync(bins, 0, bwd_f_bytes(nk), st);  // the global F bins
#define NE_BWD(T)                                                                                        \
    if (set_attr) cudaFuncSetAttribute(k_backward_mixed<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    k_backward_mixed<T><<<n_bin_blocks, BWD_THREADS, smem, st>>>(B, (unsigned char*)bins, W)
        switch (B.tpa) {
        case 1: NE_BWD(1); break;
        case 2: NE_BWD(2); break;
        case 4: NE_BWD(4); break;
        default: NE_BWD(8); break;
        }
#undef NE_BWD
        k_bins_reduce<<<(nb + BR_COLS - 1) / BR_COLS, BR_COLS * BR_SEG, 0, st>>>(
            (unsigned char*)bins, n_bin_blocks, nk, B.tab.h_r, B.tab.h_rho, W, gtheta, accumulate ? 1 : 0);
    } else {
        if (!accumulate) cudaMemsetAsync(gtheta, 0, sizeof(double) * nb, st);
        dim3 g(B.n_tiles);
        switch (B.tpa) {
        case 1: k_backward_fp64<1><<<g, NE_TILE * 1, 0, st>>>(B, W, gtheta); break;
        case 2: k_backward_fp64<2><<<g, NE_TILE * 2, 0, st>>>(B, W, gtheta); break;
        case 4: k_backward_fp64<4><<<g, NE_TILE * 4, 0, st>>>(B, W, gtheta); break;
        default: k_backward_fp64<8><<<g, NE_TILE * 8, 0, st>>>(B, W, gtheta); break;
        }
    }
}

}  // namespace ne
