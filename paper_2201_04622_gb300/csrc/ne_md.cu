// ne_md.cu -- dynamics kernels of libne.so: neighbour-list build, the fused
// lambda-blend + Einstein spring + work increment + BAOAB Langevin step,
// Maxwell-Boltzmann initial velocities, the spring energy, and small
// reductions (msd samples, exported energies/forces).
#include "ne_internal.cuh"

namespace {

__device__ __forceinline__ double wrap(double x, double L, double invL) { return x - L * floor(x * invL); }

// ------------------------------------------------------------ neighbours
// Rebuild of the candidate list of every replica whose flag is set (or of
// all replicas, when forced), in two launches:
//   k_nl_bin   one block per replica: reference positions (the lattice
//              sites at the start of a run, the current positions after an
//              atom strayed more than skin/2), wrapped; cell binning with
//              cells of edge >= r_c + skin; counting sort by cell (count,
//              exclusive scan, scatter) and an insertion sort inside each
//              cell so the order does not depend on the atomics;
//   k_nl_list  one thread per atom on every SM: all atoms of the 27
//              surrounding cells (all atoms when the box holds < 3 cells per
//              axis) within r_c + skin, minimum image, FP32 distances with a
//              1e-3 A margin so that rounding never drops a pair.
// Both return at once for replicas that need no rebuild.  The per-atom part
// of the binning (wrapped position, cell in FP64) runs first in k_nl_prep,
// one block per tile, so a large replica's FP64 work spreads over the SMs.
__global__ void __launch_bounds__(NE_TILE) k_nl_prep(DevBatch B, int force, int from_sites)
{
    const int tile = blockIdx.x;
    const int rep = B.tile_rep[tile];
    if (!(force || B.flags[rep] != 0)) return;
    const RepDev& P = B.rep[rep];
    const int a = (tile - P.tile0) * NE_TILE + threadIdx.x;
    if (a >= P.n) return;
    const int i = P.off + a;
    const double* X = from_sites ? B.x0 : B.x;
    double w[3];
    for (int d = 0; d < 3; ++d) w[d] = wrap(X[3 * i + d], P.L[d], P.invL[d]);
    B.pbuild[i] = make_float4((float)w[0], (float)w[1], (float)w[2], 0.f);
    if (P.nc[0] == 0) return;
    int c3[3];
    for (int d = 0; d < 3; ++d) {
        const int q = (int)(w[d] * P.invL[d] * P.nc[d]);
        c3[d] = min(max(q, 0), P.nc[d] - 1);
    }
    B.cellof[i] = (c3[0] * P.nc[1] + c3[1]) * P.nc[2] + c3[2];
}

__global__ void __launch_bounds__(512) k_nl_bin(DevBatch B, int force, int from_sites)
{
    const int rep = blockIdx.x;
    const RepDev& P = B.rep[rep];
    const int tid = threadIdx.x, bs = blockDim.x;
    const int go = force || B.flags[rep] != 0;
    __syncthreads();
    if (tid == 0) {
        B.building[rep] = go;
        B.flags[rep] = 0;
        if (go) atomicAdd(B.rebuilds, 1ull);
    }
    if (!go) return;
    (void)from_sites;  // positions were wrapped and binned by k_nl_prep
    const int n = P.n, off = P.off;
    if (P.nc[0] == 0) return;
    const int nc0 = P.nc[0], nc1 = P.nc[1], nc2 = P.nc[2];
    const int ncell = nc0 * nc1 * nc2;
    int* start = B.cstart + P.cell_off + rep;  // ncell + 1 entries
    int* fill = B.cfill + P.cell_off;
    for (int c = tid; c <= ncell; c += bs) start[c] = 0;
    for (int c = tid; c < ncell; c += bs) fill[c] = 0;
    __syncthreads();
    for (int a = tid; a < n; a += bs) atomicAdd(&start[B.cellof[off + a] + 1], 1);
    __syncthreads();
    // inclusive scan of start[1..ncell] by the whole block: each thread sums
    // a contiguous chunk of cells, a shared-memory scan over the chunk
    // totals gives each chunk's offset, then each thread writes its chunk
    {
        __shared__ int s_chunk[512];
        const int per = (ncell + bs - 1) / bs;
        const int c0 = 1 + tid * per, c1 = min(ncell + 1, c0 + per);
        int tot = 0;
        for (int c = c0; c < c1; ++c) tot += start[c];
        s_chunk[tid] = tot;
        __syncthreads();
        for (int o = 1; o < bs; o <<= 1) {  // Hillis-Steele inclusive scan over the chunk totals
            const int v = tid >= o ? s_chunk[tid - o] : 0;
            __syncthreads();
            s_chunk[tid] += v;
            __syncthreads();
        }
        int run = tid > 0 ? s_chunk[tid - 1] : 0;
        for (int c = c0; c < c1; ++c) {
            run += start[c];
            start[c] = run;
        }
    }
    __syncthreads();
    for (int a = tid; a < n; a += bs) {
        const int c = B.cellof[off + a];
        const int pos = atomicAdd(&fill[c], 1);
        B.sorted[off + start[c] + pos] = a;
    }
    __syncthreads();
    // sort each cell's atoms by index: in a thread-local copy when the cell
    // holds at most NE_CELL_LOCAL atoms (the common case), else in place
    constexpr int NE_CELL_LOCAL = 64;
    for (int c = tid; c < ncell; c += bs) {
        int* sl = B.sorted + off + start[c];
        const int len = start[c + 1] - start[c];
        if (len <= NE_CELL_LOCAL) {
            int loc[NE_CELL_LOCAL];
            for (int p = 0; p < len; ++p) {
                const int key = sl[p];
                int q = p - 1;
                while (q >= 0 && loc[q] > key) {
                    loc[q + 1] = loc[q];
                    --q;
                }
                loc[q + 1] = key;
            }
            for (int p = 0; p < len; ++p) sl[p] = loc[p];
        } else {
            for (int p = 1; p < len; ++p) {
                int key = sl[p], q = p - 1;
                while (q >= 0 && sl[q] > key) {
                    sl[q + 1] = sl[q];
                    --q;
                }
                sl[q + 1] = key;
            }
        }
    }
}

__global__ void __launch_bounds__(NE_TILE) k_nl_list(DevBatch B)
{
    const int tile = blockIdx.x;
    const int rep = B.tile_rep[tile];
    if (!B.building[rep]) return;
    const RepDev& P = B.rep[rep];
    const int a = (tile - P.tile0) * NE_TILE + threadIdx.x;
    if (a >= P.n) return;
    const int off = P.off, i = off + a, tpa = B.tpa;
    const float L0 = (float)P.L[0], L1 = (float)P.L[1], L2 = (float)P.L[2];
    const float iL0 = (float)P.invL[0], iL1 = (float)P.invL[1], iL2 = (float)P.invL[2];
    const float rl = sqrtf((float)P.rlist2) + 1e-3f;
    const float rl2 = rl * rl;
    const float4 pi = B.pbuild[i];
    int cnt = 0, bad = 0;
    auto test = [&](int b) {
        if (b == a) return;
        const int j = off + b;
        const float4 pj = B.pbuild[j];
        float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        dx -= L0 * rintf(dx * iL0);
        dy -= L1 * rintf(dy * iL1);
        dz -= L2 * rintf(dz * iL2);
        if (dx * dx + dy * dy + dz * dz < rl2) {
            if (cnt < NE_NMAX) B.nbr[ne_nbr_index(cnt, i, B.n_tot, tpa)] = j;
            ++cnt;
        }
    };
    if (P.nc[0] == 0) {
        for (int b = 0; b < P.n; ++b) test(b);
    } else {
        const int nc0 = P.nc[0], nc1 = P.nc[1], nc2 = P.nc[2];
        const int* start = B.cstart + P.cell_off + rep;
        const int c = B.cellof[i];
        const int cx = c / (nc1 * nc2), cy = (c / nc2) % nc1, cz = c % nc2;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    const int o = (((cx + dx + nc0) % nc0) * nc1 + (cy + dy + nc1) % nc1) * nc2 +
                                  (cz + dz + nc2) % nc2;
                    for (int p = start[o]; p < start[o + 1]; ++p) test(B.sorted[off + p]);
                }
    }
    if (cnt > NE_NMAX) bad |= ST_ENEIGH;
    B.ncnt[i] = min(cnt, NE_NMAX);
    if (bad) ne_set_status(B.status, bad);
}

// ------------------------------------------------------------ fused step
// Total force of H(lambda) on atom i from the EAM force F0, the spring force
// F_E = -k u and, with the centre of mass fixed, their replica means:
//   Frenkel-Ladd (eq. interp): (1 - lambda) F0 + lambda F_E
//   reversible scaling (eq. H_rs): lambda F0
__device__ __forceinline__ double blend(int path, double lam, double F0, double FE)
{
    return path == 0 ? (1.0 - lam) * F0 + lam * FE : lam * F0;
}

// One thread per atom.  With s the global step and Lambda(s) the schedule:
//   do_close: v += dt/2m F(x_s; Lambda(s))      (second half kick of step s-1)
//   do_open:  W += (Lambda(s+1) - Lambda(s)) dH/dlambda(x_s)   (first thread
//             of the replica; the discrete work sum of Sec. II.A)
//             v += dt/2m F(x_s; Lambda(s+1));  x += dt/2 v;
//             v = c1 v + c2 (xi - mean xi);    x += dt/2 v
// then the tile partials at the resulting x (U_E, sum u, sum |u|^2) and the
// kinetic energy of the completed velocity v_s, the FP32 wrapped copy of x
// and the displacement check against the list-build positions.
//
// With the barostat (RepDev.npt), after the second drift ln V takes one
// Euler-Maruyama step of the overdamped Langevin equation whose stationary
// density is V^(N'+1) exp(-(lambda U + P0 V)/kT) at fixed scaled
// coordinates (N' = dof / 3; the Ito drift includes the derivative of the
// mobility kT m / V, which cancels the Jacobian's kT / V):
//   d ln V = m [(dof kT + lambda W)/(3V) - P0] dt + sqrt(2 kT m dt / V) eta,
// W the virial at x_s (replica totals of pass 2 of this step), eta the first
// normal of Philox stream 5 at (atom 0, step s).  Every block computes the
// same factor; positions scale about the origin here, the box in k_npt_box
// after this kernel.
//
// Per axis (RepDev.npt = 2, for non-cubic cells such as hcp, whose c/a the
// isotropic form cannot change): each eps_a = ln L_a takes the same kind of
// step with the measure dL_x dL_y dL_z,
//   d eps_a = m [(dof/3 kT + lambda W_a)/V - P0] dt + sqrt(2 kT m dt / V) eta_a,
// W_a = -dU/d eps_a the a-th diagonal element of the virial, eta_a the a-th
// normal of the same Philox block; coordinate a and edge a scale by e^(d eps_a).
__device__ inline void npt_scale(const RepDev& P, const double* T, double lam, long long s, double dt,
                                 double mu[3])
{
    const double V = P.L[0] * P.L[1] * P.L[2];
    double z[3];
    ne_normals64(ne_philox_block(P.seed, P.replica, (unsigned)STREAM_BARO, 0u, (unsigned long long)s), z);
    const double noise = sqrt(2.0 * P.kT * P.mp * dt / V);
    if (P.npt == 2) {
        for (int c = 0; c < 3; ++c) {
            const double drive = (P.dof / 3.0 * P.kT + lam * T[TOT_VXX + c]) / V - P.P0;
            mu[c] = exp(P.mp * drive * dt + noise * z[c]);
        }
        return;
    }
    const double drive = (P.dof * P.kT + lam * T[TOT_VIR]) / (3.0 * V) - P.P0;
    const double deps = P.mp * drive * dt + noise * z[0];
    mu[0] = mu[1] = mu[2] = exp(deps / 3.0);
}

// The work increment (lambda_{s+1} - lambda_s) dH/dlambda(x_s) of replica
// rep into W (and its cumulative record and trace row), by one thread.
__device__ void step_work(const DevBatch& B, const Sched& S, const double* T, int rep, long long s, double lam_s,
                          double lam_n)
{
    const double U0 = T[TOT_UEMB] + T[TOT_UPAIR];
    const double g = S.path == 0 ? U0 - T[TOT_UE] : U0;
    const double dW = (lam_n - lam_s) * g;
    int slot = -1;
    long long k = 0;
    if (S.kind == SCHED_FIXED) {
        slot = 0;
    } else if (s >= S.t_eq && s < S.t_eq + S.t_s) {
        slot = 0;
        k = s - S.t_eq;
    } else if (s >= 2 * S.t_eq + S.t_s && s < 2 * S.t_eq + 2 * S.t_s) {
        slot = 1;
        k = s - (2 * S.t_eq + S.t_s);
    }
    if (slot >= 0) {
        double* W = B.W + (S.kind == SCHED_FIXED ? rep : 2 * rep + slot);
        *W += dW;
        if (B.Wcum && S.kind == SCHED_SWITCH) {
            double* wc = B.Wcum + ((size_t)(2 * rep + slot)) * (S.t_s + 1);
            if (k == 0) wc[0] = 0.0;
            wc[k + 1] = *W;
        }
    }
    if (B.trace && s % B.trace_stride == 0 && s / B.trace_stride < B.trace_rows) {
        double* row = B.trace + 8 * (s / B.trace_stride);
        row[0] = (double)s;
        row[1] = lam_s;
        row[2] = g;
        row[3] = U0;
        row[4] = T[TOT_UE];
        row[6] = B.W[2 * rep];
        row[7] = B.W[2 * rep + 1];
        if (slot == 0) row[6] -= dW;
        if (slot == 1) row[7] -= dW;
    }
}

template <bool MIXED>
__global__ void __launch_bounds__(NE_TILE)
    k_step(DevBatch B, Sched S, const long long* __restrict__ step_base, int j, int do_close, int do_open)
{
    __shared__ double red[NPB][NE_TILE];
    const int tile = blockIdx.x;
    const int rep = B.tile_rep[tile];
    const RepDev& P = B.rep[rep];
    const int a = (tile - P.tile0) * NE_TILE + threadIdx.x;
    const bool valid = a < P.n;
    const int i = P.off + (valid ? a : 0);
    const long long s = *step_base + j;
    const double* T = B.tot + (size_t)rep * NTOT;
    const double lam_s = ne_sched_lambda(S, s);
    const double lam_n = ne_sched_lambda(S, s + 1);
    const double invN = 1.0 / P.n;
    double part[NPB] = {0, 0, 0, 0, 0, 0};
    int bad = 0;
    if (valid) {
        double x[3], v[3], u[3], F0[3], mF0[3], mFE[3];
        double Lb[3] = {P.L[0], P.L[1], P.L[2]};  // box after this step (the barostat scales it)
        for (int c = 0; c < 3; ++c) {
            x[c] = B.x[3 * i + c];
            v[c] = B.v[3 * i + c];
            u[c] = x[c] - B.x0[3 * i + c];
        }
        if constexpr (MIXED) {
            float4 f = B.f32[i];
            F0[0] = f.x;
            F0[1] = f.y;
            F0[2] = f.z;
        } else {
            F0[0] = B.f64[3 * i];
            F0[1] = B.f64[3 * i + 1];
            F0[2] = B.f64[3 * i + 2];
        }
        // this atom's mass, spring, noise amplitude and half-step factor
        // (one species, or its species' entries)
        const int q = P.nsp ? (int)P.sp[a] : 0;
        const double mi = P.nsp ? P.ms[q] : P.m, ki = P.nsp ? P.ks[q] : P.k;
        const double c2i = P.nsp ? P.c2s[q] : P.c2, hdti = P.nsp ? P.hdts[q] : P.hdt_m;
        for (int c = 0; c < 3; ++c) {
            if (P.nsp) {  // mass-weighted constraint: F_i -= m_i sum_j F_j / M
                mF0[c] = S.fix_cm ? mi * T[TOT_F0X + c] / P.M : 0.0;
                mFE[c] = S.fix_cm ? -mi * T[TOT_UX + c] / P.M : 0.0;  // TOT_UX: sum_j k_j u_j
            } else {
                mF0[c] = S.fix_cm ? T[TOT_F0X + c] * invN : 0.0;
                mFE[c] = S.fix_cm ? -P.k * T[TOT_UX + c] * invN : 0.0;
            }
        }
        if (do_close) {
            for (int c = 0; c < 3; ++c)
                v[c] += hdti * blend(S.path, lam_s, F0[c] - mF0[c], -ki * u[c] - mFE[c]);
        }
        part[PB_KE] = 0.5 * mi * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (do_open) {
            // velocity increments of the thermostat: c2 (xi - mean xi) for one
            // species; c2_i xi_i - sum_j m_j c2_j xi_j / M with species tables
            double dv[3];
            for (int c = 0; c < 3; ++c) {
                const double xi = MIXED ? (double)B.xi32[3 * i + c] : B.xi64[3 * i + c];
                if (P.nsp) dv[c] = c2i * xi - (S.fix_cm ? T[TOT_XIX + c] / P.M : 0.0);
                else dv[c] = P.c2 * (S.fix_cm ? xi - T[TOT_XIX + c] * invN : xi);
            }
            for (int c = 0; c < 3; ++c) {
                v[c] += hdti * blend(S.path, lam_n, F0[c] - mF0[c], -ki * u[c] - mFE[c]);
                x[c] += 0.5 * S.dt * v[c];
                v[c] = P.c1 * v[c] + dv[c];
                x[c] += 0.5 * S.dt * v[c];
            }
            if (P.npt) {
                double mu[3];
                npt_scale(P, T, lam_n, s, S.dt, mu);
                for (int c = 0; c < 3; ++c) {
                    x[c] *= mu[c];
                    Lb[c] = mu[c] * P.L[c];
                }
            }
            for (int c = 0; c < 3; ++c) u[c] = x[c] - B.x0[3 * i + c];
        }
        for (int c = 0; c < 3; ++c) {
            if (!isfinite(x[c]) || !isfinite(v[c])) bad |= ST_ENAN;
            B.x[3 * i + c] = x[c];
            B.v[3 * i + c] = v[c];
            part[PB_UX + c] = P.nsp ? ki * u[c] : u[c];
        }
        part[PB_U2] = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        part[PB_UE] = 0.5 * ki * part[PB_U2];
        // FP32 wrapped copy and displacement since the list build
        float w[3];
        for (int c = 0; c < 3; ++c) w[c] = (float)wrap(x[c], Lb[c], 1.0 / Lb[c]);
        if constexpr (MIXED) B.pos32[i] = make_float4(w[0], w[1], w[2], 0.f);
        float4 pb = B.pbuild[i];
        float d0 = w[0] - pb.x, d1 = w[1] - pb.y, d2 = w[2] - pb.z;
        const float L0 = (float)Lb[0], L1 = (float)Lb[1], L2 = (float)Lb[2];
        d0 -= L0 * rintf(d0 / L0);
        d1 -= L1 * rintf(d1 / L1);
        d2 -= L2 * rintf(d2 / L2);
        if (d0 * d0 + d1 * d1 + d2 * d2 > P.half_skin2) B.flags[rep] = 1;
    }
    if (bad) ne_set_status(B.status, bad);
    if (do_open && valid && a == 0) step_work(B, S, T, rep, s, lam_s, lam_n);
    for (int q = 0; q < NPB; ++q) red[q][threadIdx.x] = part[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < NPB; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* pb = B.partB + (size_t)tile * NPB;
        for (int q = 0; q < NPB; ++q) pb[q] = red[q][0];
    }
}

// The mixed-precision step: the same steps as k_step, with the velocity
// arithmetic (kicks, thermostat) in FP32, each drift added to the FP64
// position once, and the tile sums in double-float -- the crystal runner's
// precision, keeping GB300's FP64 pipe (1/64 of FP32) to a few conversions
// an atom.  Thread 0 forms the block's replica scalars (lambda at s and s + 1,
// the centre-of-mass means, the barostat's factors, the box after it) in FP64
// once and the second warp the FP32 mass, spring and thermostat tables.
__global__ void __launch_bounds__(NE_TILE)
    k_step_mixed(DevBatch B, Sched S, const long long* __restrict__ step_base, int j, int do_close, int do_open)
{
    __shared__ double s_lam[2], s_mu[3];
    __shared__ float s_mean[9];  // mean F0, spring and noise terms (see below)
    __shared__ float s_box[8];   // box and 1 / box after this step's scaling, c1, (skin / 2)^2
    __shared__ float s_tab[4][NE_MAX_SPECIES_DEV + 1];  // m, k, c2, dt / 2m: species 0.., the replica's last
    __shared__ float2 s_w[NPB][NE_TILE / 32];
    const int tile = blockIdx.x;
    const int rep = B.tile_rep[tile];
    const RepDev& P = B.rep[rep];
    const int a = (tile - P.tile0) * NE_TILE + threadIdx.x;
    const bool valid = a < P.n;
    const int i = P.off + (valid ? a : 0);
    const long long s = *step_base + j;
    const double* T = B.tot + (size_t)rep * NTOT;
    if (threadIdx.x < 32) {
        // the replica scalars, one a lane, the lanes running the same
        // instructions (GB300 issues an FP64 warp instruction at the same cost
        // for one lane as for 32, so a serial chain on one thread held the
        // whole block): lambda at s and s + 1 in lanes of each parity; the
        // barostat's factors (lane 0); one division for the centre-of-mass
        // means (lanes 0-8: mean F0, the spring's mean and the noise mean,
        // per unit mass with species tables, mass-weighted) and 1 / box
        // (lanes 9-11); the box (lanes 12-14), c1 and (skin / 2)^2
        const int l = threadIdx.x, c = l % 3;
        const double lam = ne_sched_lambda(S, s + (l & 1));
        if (l < 2) s_lam[l] = lam;
        double mu[3] = {1.0, 1.0, 1.0};
        if (do_open && P.npt) {
            const double lam_n1 = __shfl_sync(0xffffffffu, lam, 1);
            if (l == 0) npt_scale(P, T, lam_n1, s, S.dt, mu);
            for (int q = 0; q < 3; ++q) mu[q] = __shfl_sync(0xffffffffu, mu[q], 0);
        }
        const double muc = c == 0 ? mu[0] : (c == 1 ? mu[1] : mu[2]);
        double num, den = P.nsp ? P.M : (double)P.n;
        if (l < 3) num = T[TOT_F0X + c];
        else if (l < 6) num = -(P.nsp ? 1.0 : P.k) * T[TOT_UX + c];
        else if (l < 9) num = T[TOT_XIX + c];
        else {
            num = P.invL[c];
            den = muc;
        }
        const double quo = num / den;
        if (l < 9) s_mean[l] = S.fix_cm ? (float)quo : 0.f;
        else if (l < 12) s_box[3 + c] = (float)quo;
        else if (l < 15) s_box[c] = (float)(muc * P.L[c]);
        else if (l == 15) s_box[6] = (float)P.c1;
        else if (l == 16) s_box[7] = (float)P.half_skin2;
        if (l < 3) s_mu[l] = muc;
    } else if (threadIdx.x >= 32 && threadIdx.x < 33 + NE_MAX_SPECIES_DEV) {
        const int t = threadIdx.x - 32;
        const bool r1 = t == NE_MAX_SPECIES_DEV;  // the replica's single-species values
        const int ts = r1 ? 0 : t;
        if (r1 || t < P.nsp) {
            s_tab[0][t] = (float)(r1 ? P.m : P.ms[ts]);
            s_tab[1][t] = (float)(r1 ? P.k : P.ks[ts]);
            s_tab[2][t] = (float)(r1 ? P.c2 : P.c2s[ts]);
            s_tab[3][t] = (float)(r1 ? P.hdt_m : P.hdts[ts]);
        }
    }
    __syncthreads();
    const double lam_s = s_lam[0], lam_n = s_lam[1];
    const float ls = (float)lam_s, ln = (float)lam_n;
    float part[NPB] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int bad = 0;
    if (valid) {
        double x[3];
        float v[3], u[3], F0[3], mF0[3], mFE[3];
        const float4 f = B.f32[i];
        F0[0] = f.x;
        F0[1] = f.y;
        F0[2] = f.z;
        for (int c = 0; c < 3; ++c) {
            x[c] = B.x[3 * i + c];
            v[c] = (float)B.v[3 * i + c];
            u[c] = (float)(x[c] - B.x0[3 * i + c]);
        }
        const int q = P.nsp ? (int)P.sp[a] : NE_MAX_SPECIES_DEV;
        const float mi = s_tab[0][q], ki = s_tab[1][q], c2i = s_tab[2][q], hdti = s_tab[3][q];
        const float wm = P.nsp ? mi : 1.f;  // F_i -= m_i sum_j F_j / M with species tables
        for (int c = 0; c < 3; ++c) {
            mF0[c] = wm * s_mean[c];
            mFE[c] = wm * s_mean[3 + c];
        }
        auto blendf = [&](float lam, float a0, float ae) { return S.path == 0 ? (1.f - lam) * a0 + lam * ae : lam * a0; };
        if (do_close)
            for (int c = 0; c < 3; ++c) v[c] += hdti * blendf(ls, F0[c] - mF0[c], -ki * u[c] - mFE[c]);
        part[PB_KE] = 0.5f * mi * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (do_open) {
            for (int c = 0; c < 3; ++c) {
                const float xi = B.xi32[3 * i + c];
                const float dv = P.nsp ? c2i * xi - s_mean[6 + c] : c2i * (xi - s_mean[6 + c]);
                v[c] += hdti * blendf(ln, F0[c] - mF0[c], -ki * u[c] - mFE[c]);
                const float v1 = v[c];
                v[c] = s_box[6] * v[c] + dv;
                const float dx = 0.5f * (float)S.dt * (v1 + v[c]);
                if (!isfinite(dx)) bad |= ST_ENAN;
                x[c] += (double)dx;
            }
            if (P.npt)
                for (int c = 0; c < 3; ++c) x[c] *= s_mu[c];
            // from x itself, so that a run resumed from (x, v) forms the same totals
            for (int c = 0; c < 3; ++c) u[c] = (float)(x[c] - B.x0[3 * i + c]);
        }
        for (int c = 0; c < 3; ++c) {
            if (!isfinite(v[c])) bad |= ST_ENAN;
            B.x[3 * i + c] = x[c];
            B.v[3 * i + c] = (double)v[c];
            part[PB_UX + c] = P.nsp ? ki * u[c] : u[c];
        }
        part[PB_U2] = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        part[PB_UE] = 0.5f * ki * part[PB_U2];
        // FP32 wrapped copy and displacement since the list build: the image
        // index in FP32, the shift (only for an atom outside the box) in FP64
        float w[3];
        for (int c = 0; c < 3; ++c) {
            w[c] = (float)x[c];
            const float n = floorf(w[c] * s_box[3 + c]);
            if (n != 0.f) w[c] = (float)(x[c] - s_mu[c] * P.L[c] * (double)n);
        }
        B.pos32[i] = make_float4(w[0], w[1], w[2], 0.f);
        const float4 pb = B.pbuild[i];
        float d[3] = {w[0] - pb.x, w[1] - pb.y, w[2] - pb.z}, d2 = 0.f;
        for (int c = 0; c < 3; ++c) {
            d[c] = fmaf(-s_box[c], rintf(d[c] * s_box[3 + c]), d[c]);
            d2 = fmaf(d[c], d[c], d2);
        }
        if (d2 > s_box[7]) B.flags[rep] = 1;
    }
    if (bad) ne_set_status(B.status, bad);
    if (do_open && valid && a == 0) step_work(B, S, T, rep, s, lam_s, lam_n);
    // the tile's partials in double-float: a fixed tree in each warp, then
    // the two warps in order
    const int wp = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int q = 0; q < NPB; ++q) {
        const dff t = dff_warp_sum({part[q], 0.f});
        if (l == 0) s_w[q][wp] = make_float2(t.hi, t.lo);
    }
    __syncthreads();
    if (threadIdx.x < NPB) {
        dff t = {0.f, 0.f};
        for (int w2 = 0; w2 < NE_TILE / 32; ++w2) t = dff_add(t, {s_w[threadIdx.x][w2].x, s_w[threadIdx.x][w2].y});
        B.partB[(size_t)tile * NPB + threadIdx.x] = (double)t.hi + (double)t.lo;
    }
}

// Trace temperature column: KE of v_s (tile partials of the step kernel of
// step s) summed in fixed order after that kernel.
__global__ void k_trace_T(DevBatch B, const long long* __restrict__ step_base, int j)
{
    const long long s = *step_base + j;
    if (!B.trace || s % B.trace_stride != 0 || s / B.trace_stride >= B.trace_rows) return;
    const RepDev& P = B.rep[0];
    const double ke = ne_warp_tile_sum(B.partB, NPB, PB_KE, P.tile0, P.ntile);
    const double kB = 8.617333262e-5;
    if (threadIdx.x == 0) B.trace[8 * (s / B.trace_stride) + 5] = 2.0 * ke / (P.dof * kB);
}

__global__ void k_advance(long long* step_base, long long by) { *step_base += by; }

// Box of every barostatted replica after the step kernel of step s (same
// scale factor as that kernel).  A box whose cells became shorter than
// r_c + skin, or whose edge fell below 2 (r_c + skin), is reported
// (NE_ERANGE) and left unchanged.
__global__ void k_npt_box(DevBatch B, Sched S, const long long* __restrict__ step_base, int j)
{
    const int rep = blockIdx.x;
    if (rep >= B.n_rep || threadIdx.x != 0) return;
    RepDev& P = const_cast<RepDev*>(B.rep)[rep];
    if (!P.npt) return;
    const long long s = *step_base + j;
    double mu[3];
    npt_scale(P, B.tot + (size_t)rep * NTOT, ne_sched_lambda(S, s + 1), s, S.dt, mu);
    const double rl = sqrt(P.rlist2);
    for (int c = 0; c < 3; ++c) {
        const double L = mu[c] * P.L[c];
        if (!(L > 2.0 * rl) || (P.nc[c] > 0 && !(L / P.nc[c] >= rl))) {
            ne_set_status(B.status, ST_ERANGE);
            return;
        }
    }
    for (int c = 0; c < 3; ++c) {
        P.L[c] *= mu[c];
        P.invL[c] = 1.0 / P.L[c];
    }
}

__global__ void k_noise(unsigned long long seed, unsigned replica, int stream, long long step, int n,
                        int mixed, double* z)
{
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        uint4 w = ne_philox_block(seed, replica, (unsigned)stream, (unsigned)a, (unsigned long long)step);
        if (mixed) {
            float f[3];
            ne_normals32(w, f);
            for (int c = 0; c < 3; ++c) z[3 * a + c] = f[c];
        } else {
            double d[3];
            ne_normals64(w, d);
            for (int c = 0; c < 3; ++c) z[3 * a + c] = d[c];
        }
    }
}

// FP32 copy of the positions wrapped into the box (pass-1/2 input of the
// mixed path when no step kernel has produced it).
__global__ void k_wrap32(DevBatch B)
{
    const int tile = blockIdx.x;
    const RepDev& P = B.rep[B.tile_rep[tile]];
    const int a = (tile - P.tile0) * NE_TILE + threadIdx.x;
    if (a >= P.n) return;
    const int i = P.off + a;
    B.pos32[i] = make_float4((float)wrap(B.x[3 * i], P.L[0], P.invL[0]),
                             (float)wrap(B.x[3 * i + 1], P.L[1], P.invL[1]),
                             (float)wrap(B.x[3 * i + 2], P.L[2], P.invL[2]), 0.f);
}

// ------------------------------------------------------------ velocities
// Philox normals (stream 1, step 0) times sqrt(kT/m); mean removed when the
// centre of mass is fixed; rescaled to exactly T over the free dof.
// Velocity start: Maxwell-Boltzmann from Philox normals, the centre-of-mass
// momentum removed, then scaled to T exactly.  Three launches over the
// tiles (draw, centre, scale); each block forms its replica's sums from the
// tile partials in a fixed order (the partA slots of pass 1 and 2, which a
// force evaluation rewrites before it reads them), so the FP64 Box-Muller of
// a large replica spreads over the SMs instead of one block doing it all.
__device__ __forceinline__ double tile_sum64(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = NE_TILE / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double t = red[0];
    __syncthreads();
    return t;
}

__device__ __forceinline__ double init_mass(const RepDev& P, int a) { return P.nsp ? P.ms[P.sp[a]] : P.m; }

__global__ void __launch_bounds__(NE_TILE) k_init_v_draw(DevBatch B)
{
    __shared__ double red[NE_TILE];
    const int tile = blockIdx.x;
    const RepDev& P = B.rep[B.tile_rep[tile]];
    const int a = (tile - P.tile0) * NE_TILE + threadIdx.x;
    // with species tables atom a has sd = sqrt(kT / m_a), and the momentum
    // sum_a m_a v_a / M is removed (the mass-weighted centre of mass)
    double sum[3] = {0, 0, 0};
    if (a < P.n) {
        const double sd = sqrt(P.kT / init_mass(P, a));
        const double w = P.nsp ? init_mass(P, a) / P.M : 1.0;
        double z[3];
        ne_normals64(ne_philox_block(P.seed, P.replica, STREAM_INITV, (unsigned)a, 0ull), z);
        for (int c = 0; c < 3; ++c) {
            B.v[3 * (P.off + a) + c] = sd * z[c];
            sum[c] = w * sd * z[c];
        }
    }
    for (int c = 0; c < 3; ++c) {
        const double t = tile_sum64(sum[c], red);
        if (threadIdx.x == 0) B.partA[(size_t)tile * NPA + c] = t;
    }
}

__global__ void __launch_bounds__(NE_TILE) k_init_v_center(DevBatch B, int fix_cm)
{
    __shared__ double red[NE_TILE];
    __shared__ double s_mean[3];
    const int tile = blockIdx.x;
    const RepDev& P = B.rep[B.tile_rep[tile]];
    if (threadIdx.x < 32)
        for (int c = 0; c < 3; ++c) {
            const double t = ne_warp_tile_sum(B.partA, NPA, c, P.tile0, P.ntile);
            if (threadIdx.x == 0) s_mean[c] = fix_cm ? (P.nsp ? t : t / P.n) : 0.0;
        }
    __syncthreads();
    const int a = (tile - P.tile0) * NE_TILE + threadIdx.x;
    double ke = 0.0;
    if (a < P.n)
        for (int c = 0; c < 3; ++c) {
            double* vv = &B.v[3 * (P.off + a) + c];
            *vv -= s_mean[c];
            ke += 0.5 * init_mass(P, a) * (*vv) * (*vv);
        }
    const double t = tile_sum64(ke, red);
    if (threadIdx.x == 0) B.partA[(size_t)tile * NPA + 3] = t;
}

__global__ void __launch_bounds__(NE_TILE) k_init_v_scale(DevBatch B)
{
    __shared__ double s_sc;
    const int tile = blockIdx.x;
    const RepDev& P = B.rep[B.tile_rep[tile]];
    if (threadIdx.x < 32) {
        const double ke = ne_warp_tile_sum(B.partA, NPA, 3, P.tile0, P.ntile);
        const double kB = 8.617333262e-5;
        if (threadIdx.x == 0) s_sc = sqrt((P.kT / kB) / (2.0 * ke / (P.dof * kB)));
    }
    __syncthreads();
    const int a = (tile - P.tile0) * NE_TILE + threadIdx.x;
    if (a < P.n)
        for (int c = 0; c < 3; ++c) B.v[3 * (P.off + a) + c] *= s_sc;
}

// ------------------------------------------------------------ spring
// Einstein crystal (eq. einstein): U_E = sum k/2 |r - r0|^2, F_E = -k (r - r0).
__global__ void __launch_bounds__(1024) k_spring(const double* __restrict__ x, const double* __restrict__ x0,
                                                 int n, double k, double* f, double* e)
{
    __shared__ double red[1024];
    double acc = 0.0;
    for (int q = threadIdx.x; q < 3 * n; q += blockDim.x) {
        double u = x[q] - x0[q];
        acc += 0.5 * k * u * u;
        if (f) f[q] = -k * u;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0 && e) *e = red[0];
}

// EAM forces and energy of replica 0 to caller buffers.
template <bool MIXED>
__global__ void k_export(DevBatch B, double* f, double* e)
{
    const RepDev& P = B.rep[0];
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < P.n; a += gridDim.x * blockDim.x) {
        const int i = P.off + a;
        if (f) {
            if constexpr (MIXED) {
                float4 g = B.f32[i];
                f[3 * a] = g.x;
                f[3 * a + 1] = g.y;
                f[3 * a + 2] = g.z;
            } else {
                f[3 * a] = B.f64[3 * i];
                f[3 * a + 1] = B.f64[3 * i + 1];
                f[3 * a + 2] = B.f64[3 * i + 2];
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && e) *e = B.tot[TOT_UEMB] + B.tot[TOT_UPAIR];
}

// One msd sample per replica from the step-kernel partials:
// (1/n) sum |u_i - mean u|^2 = (1/n) sum |u|^2 - |mean u|^2.
__global__ void k_msd_sample(DevBatch B, double* acc)
{
    const int rep = blockIdx.x;
    const RepDev& P = B.rep[rep];
    double s[4];
    s[0] = ne_warp_tile_sum(B.partB, NPB, PB_UX, P.tile0, P.ntile);
    s[1] = ne_warp_tile_sum(B.partB, NPB, PB_UY, P.tile0, P.ntile);
    s[2] = ne_warp_tile_sum(B.partB, NPB, PB_UZ, P.tile0, P.ntile);
    s[3] = ne_warp_tile_sum(B.partB, NPB, PB_U2, P.tile0, P.ntile);
    if (threadIdx.x != 0) return;
    const double invN = 1.0 / P.n;
    acc[rep] += s[3] * invN - (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]) * invN * invN;
}

// One msd sample per species of each replica with species tables (Sec. V):
// displacements u_i = x_i - x0_i taken about the mass-weighted centre,
// dR = sum_i m_i u_i / M; acc[rep * NE_MAX_SPECIES + s] += (1/N_s) sum over
// the atoms of species s of |u_i - dR|^2.  One block per replica, FP64,
// fixed-order block sums.
__global__ void __launch_bounds__(256) k_msd_sample_species(DevBatch B, double* acc)
{
    __shared__ double red[3 + 2 * NE_MAX_SPECIES_DEV][256];
    const int rep = blockIdx.x;
    const RepDev& P = B.rep[rep];
    double s[3] = {0, 0, 0};
    for (int a = threadIdx.x; a < P.n; a += blockDim.x) {
        const double w = P.ms[P.sp[a]] / P.M;
        for (int c = 0; c < 3; ++c) s[c] += w * (B.x[3 * (P.off + a) + c] - B.x0[3 * (P.off + a) + c]);
    }
    for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    const double dR[3] = {red[0][0], red[1][0], red[2][0]};
    __syncthreads();
    double d2[NE_MAX_SPECIES_DEV] = {}, cnt[NE_MAX_SPECIES_DEV] = {};
    for (int a = threadIdx.x; a < P.n; a += blockDim.x) {
        const int q = P.sp[a];
        for (int c = 0; c < 3; ++c) {
            const double d = (B.x[3 * (P.off + a) + c] - B.x0[3 * (P.off + a) + c]) - dR[c];
            d2[q] += d * d;
        }
        cnt[q] += 1.0;
    }
    for (int q = 0; q < NE_MAX_SPECIES_DEV; ++q) {
        red[3 + q][threadIdx.x] = d2[q];
        red[3 + NE_MAX_SPECIES_DEV + q][threadIdx.x] = cnt[q];
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 3; q < 3 + 2 * NE_MAX_SPECIES_DEV; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < P.nsp && red[3 + NE_MAX_SPECIES_DEV + threadIdx.x][0] > 0)
        acc[rep * NE_MAX_SPECIES_DEV + threadIdx.x] +=
            red[3 + threadIdx.x][0] / red[3 + NE_MAX_SPECIES_DEV + threadIdx.x][0];
}

}  // namespace

namespace ne {

void launch_nl_build(const DevBatch& B, int force, int from_sites, cudaStream_t st)
{
    k_nl_prep<<<B.n_tiles, NE_TILE, 0, st>>>(B, force, from_sites);
    k_nl_bin<<<B.n_rep, 512, 0, st>>>(B, force, from_sites);
    k_nl_list<<<B.n_tiles, NE_TILE, 0, st>>>(B);
}

void launch_step(const DevBatch& B, const Sched& S, bool mixed, const long long* step_base, int j,
                 int do_close, int do_open, cudaStream_t st)
{
    if (mixed)
        k_step_mixed<<<B.n_tiles, NE_TILE, 0, st>>>(B, S, step_base, j, do_close, do_open);
    else
        k_step<false><<<B.n_tiles, NE_TILE, 0, st>>>(B, S, step_base, j, do_close, do_open);
    if (B.trace) k_trace_T<<<1, 32, 0, st>>>(B, step_base, j);
}

void launch_prep(const DevBatch& B, const Sched& S, bool mixed, const long long* step_base,
                 cudaStream_t st)
{
    if (mixed)
        k_step_mixed<<<B.n_tiles, NE_TILE, 0, st>>>(B, S, step_base, 0, 0, 0);
    else
        k_step<false><<<B.n_tiles, NE_TILE, 0, st>>>(B, S, step_base, 0, 0, 0);
}

void launch_npt_box(const DevBatch& B, const Sched& S, const long long* step_base, int j, cudaStream_t st)
{
    k_npt_box<<<B.n_rep, 32, 0, st>>>(B, S, step_base, j);
}

void launch_wrap32(const DevBatch& B, cudaStream_t st)
{
    k_wrap32<<<B.n_tiles, NE_TILE, 0, st>>>(B);
}

void launch_noise(unsigned long long seed, unsigned replica, int stream, long long step, int n, int mixed,
                  double* z, cudaStream_t st)
{
    k_noise<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, st>>>(seed, replica, stream, step, n,
                                                                            mixed, z);
}

void launch_advance(long long* step_base, long long by, cudaStream_t st)
{
    k_advance<<<1, 1, 0, st>>>(step_base, by);
}

void launch_init_velocities(const DevBatch& B, int fix_cm, cudaStream_t st)
{
    k_init_v_draw<<<B.n_tiles, NE_TILE, 0, st>>>(B);
    k_init_v_center<<<B.n_tiles, NE_TILE, 0, st>>>(B, fix_cm);
    k_init_v_scale<<<B.n_tiles, NE_TILE, 0, st>>>(B);
}

void launch_spring(const double* x, const double* x0, int n, double k, double* f, double* e,
                   double*, cudaStream_t st)
{
    k_spring<<<1, 1024, 0, st>>>(x, x0, n, k, f, e);
}

void launch_export(const DevBatch& B, bool mixed, double* f_out, double* e_out, cudaStream_t st)
{
    if (mixed)
        k_export<true><<<64, 256, 0, st>>>(B, f_out, e_out);
    else
        k_export<false><<<64, 256, 0, st>>>(B, f_out, e_out);
}

void launch_msd_sample(const DevBatch& B, double* acc, cudaStream_t st)
{
    if (B.species_any)
        k_msd_sample_species<<<B.n_rep, 256, 0, st>>>(B, acc);
    else
        k_msd_sample<<<B.n_rep, 32, 0, st>>>(B, acc);
}

}  // namespace ne
