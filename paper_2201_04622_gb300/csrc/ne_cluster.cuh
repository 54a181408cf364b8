// ne_cluster.cuh -- replica description and launcher of the persistent
// cluster-per-replica runner for crystals (ne_cluster.cu).
#pragma once
#include <cuda_runtime.h>

#include "ne_internal.cuh"

#define NE_STENCIL_MAX 512  // stencil entries per basis site
#define NE_STENCIL_PAD 16   // far entries ending each basis site's stencil (outside any cutoff)

struct XRep {
    double cell[3];       // cell edges (a, a, a; hcp: a, sqrt(3) a, c)
    double basis[4][3];   // basis positions as fractions of the cell edges
    double k;             // spring constant (FP64 for the mean spring force)
    float kf, mf, hdt_mf, c1f, c2f;
    float D;              // largest displacement from a site the stencil covers
    int n, off, nb, nx, ny, nz;
    int st_off, st_cnt;   // stencil of basis b: entries [st_off + b * st_cnt, + st_cnt)
    int st_margin;        // M: cell offsets of the stencil lie in [-M, M]
    unsigned long long seed;
    unsigned replica;
    int widx;             // index of the replica in the caller's arrays (work W)
    // several species (Sec. V): nsp >= 2 -- atom a has species sp[a]
    // (validated on the host) with spring kfs, half-step factor hdts, noise
    // amplitude c2fs and mass mfs of its species; invM = 1 / total mass
    int nsp;
    const unsigned char* sp;
    float invM;
    float kfs[NE_MAX_SPECIES_DEV], hdts[NE_MAX_SPECIES_DEV], c2fs[NE_MAX_SPECIES_DEV], mfs[NE_MAX_SPECIES_DEV];
    int cta0, ncta;       // brick runner: the replica's first CTA in the grid and its CTA count
    // barostat (reversible-scaling path; reading A23): 0 none, 1 isotropic,
    // 2 one equation per box edge; target pressure, mobility beta_T / tau_p,
    // k_B T, degrees of freedom and the box at the call's start
    int npt, dof;
    double P0, mp, kT;
    double box0[3];
};

// Tensor memory as per-thread scratch (both crystal runners): a CTA that is
// alone on its SM takes all NE_TM_COLS columns; a warp reads and writes
// NE_TM_BATCH columns of its own lanes at a time.
#define NE_TM_COLS 512
#define NE_TM_BATCH 8

// N (4 or 8) consecutive TMEM columns of this thread's lane (32x32b shape:
// thread i of the warp is lane i of the warp's quarter).  The load waits for
// its data; the registers pass through the wait so no use moves above it.
template <int N>
__device__ __forceinline__ void ne_tm_st(unsigned taddr, const float (&v)[N])
{
    static_assert(N == 4 || N == 8, "TMEM batches of 4 or 8 columns");
    if constexpr (N == 8)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                     :
                     : "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                       "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])),
                       "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                     : "memory");
    else
        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};"
                     :
                     : "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                       "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3]))
                     : "memory");
}

template <int N>
__device__ __forceinline__ void ne_tm_ld(unsigned taddr, float (&v)[N])
{
    static_assert(N == 4 || N == 8, "TMEM batches of 4 or 8 columns");
    unsigned r[8];
    if constexpr (N == 8) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7])
                     : "r"(taddr)
                     : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                       "+r"(r[7])
                     :
                     : "memory");
    } else {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                     : "r"(taddr)
                     : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]) : : "memory");
    }
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = __uint_as_float(r[q]);
}

// Four columns of 32-bit words (packed integers) of this thread's lane.
__device__ __forceinline__ void ne_tm_st_u4(unsigned taddr, const unsigned (&v)[4])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};"
                 :
                 : "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
                 : "memory");
}

__device__ __forceinline__ void ne_tm_ld_u4(unsigned taddr, unsigned (&v)[4])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]) : : "memory");
}

// Eight float columns at taddr_f and four word columns at taddr_w, both
// loads in flight before the one wait.
__device__ __forceinline__ void ne_tm_ld_f8u4(unsigned taddr_f, unsigned taddr_w, float (&f)[8], unsigned (&w)[4])
{
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr_f)
                 : "memory");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                 : "r"(taddr_w)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3])
                 :
                 : "memory");
#pragma unroll
    for (int q = 0; q < 8; ++q) f[q] = __uint_as_float(r[q]);
}

// Warp 0 of the CTA takes all NE_TM_COLS columns (the base address goes to
// *s_slot in shared memory); the caller then makes it visible with
// tcgen05.fence::before_thread_sync, a CTA barrier and
// tcgen05.fence::after_thread_sync.
__device__ __forceinline__ void ne_tm_alloc(unsigned* s_slot)
{
    if (threadIdx.x < 32) {
        __syncwarp();
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :
                     : "r"((unsigned)__cvta_generic_to_shared(s_slot)), "r"(NE_TM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
}

// Every thread of the CTA calls this once it is past its last TMEM access:
// warp 0 returns the columns.
__device__ __forceinline__ void ne_tm_free(unsigned base)
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(NE_TM_COLS) : "memory");
    }
}

namespace ne {
size_t cluster_smem_bytes(int n_max, int nb_nst_max, int lut_max, bool npt = false);
int cluster_atoms_per_cta();
int cluster_threads_per_atom();
int cluster_size_for(int n, int nb);           // smallest CTAs per cluster for an n-atom replica
int cluster_atoms_for(int n, int C, int nb);    // atoms per CTA of an n-atom replica on C CTAs
int cluster_max_active(int C, size_t smem);     // co-resident clusters of C CTAs (0 if none or on error)
cudaError_t launch_lambda_table(const Sched& S, long long s_begin, long long count, double* out, cudaStream_t st);
cudaError_t launch_cluster(const XRep* reps, int n_rep, int C, size_t smem, const float4* st_vec,
                           const float* st_dist, double* x, double* v, double* W, int* status, const Sched& S,
                           long long s_begin, long long n_steps, const Tables& tab, unsigned long long* work,
                           int k_lo, double* lam_tab, double* wcum, cudaStream_t st, bool npt = false,
                           double* boxes_out = nullptr);
// Brick runner (ne_brick.cu): replicas larger than a cluster holds, one
// cooperative launch over CTAs that own blocks of cells and exchange u and
// F' through global memory between grid barriers; with the barostat (npt)
// a third grid barrier a step carries the CTAs' virial sums.
size_t brick_smem_bytes(int tpa, int nb_nst_max, int lut_max, bool npt = false);
int brick_atoms_per_cta(int tpa);
int brick_max_ctas(int tpa, size_t smem, bool npt = false);  // co-resident CTAs of the launch (0 on error)
struct BrickBufs {
    float4* u4;      // [2][N] (u, 0) of every atom, by step parity
    float* fp;       // [N] F'(rho)
    float* part;     // [2][n_cta][NPART] per-CTA partial sums, by step parity
    float* vir;      // [n_cta][6] per-CTA diagonal virial (hi, lo per axis; barostat only)
    unsigned* bar;   // [2] grid barrier: arrivals, generation
    int* abortf;     // a bounded wait gave up: every CTA leaves
};
cudaError_t launch_brick(int tpa, const XRep* reps, const int* cta_rep, int n_cta, size_t smem, const float4* st_vec,
                         const float* st_dist, double* x, double* v, double* W, int* status, const Sched& S,
                         long long s_begin, long long n_steps, const Tables& tab, unsigned long long* work,
                         int k_lo, const double* lam_tab, double* wcum, const BrickBufs& bb, long long n_tot,
                         cudaStream_t st, bool npt = false, double* boxes_out = nullptr);
}  // namespace ne
