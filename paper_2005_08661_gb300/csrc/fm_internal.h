// fm_internal.h -- device-side building blocks shared by the CUDA translation units of
// the field-map library (not part of the public ABI; see include/fm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fm.h"

namespace fm {

constexpr int kMaxPairs = FM_MAX_ECHO * (FM_MAX_ECHO - 1) / 2;

// Neighbour-bit byte stored per voxel: bit 0 = voxel is an unknown (inside the mask);
// bits 1..6 = its (-x, +x, -y, +y, -z, +z) neighbour exists and is an unknown too;
// bit 7 = x + y + z is odd (the black colour of the red-black ordering; mask voxels only).
enum : uint8_t { NB_IN = 1, NB_XM = 2, NB_XP = 4, NB_YM = 8, NB_YP = 16, NB_ZM = 32, NB_ZP = 64, NB_ODD = 128 };

// Device scalar slots (double) kept per context.
enum Scal {
    S_ALPHA = 0,   // current step alpha (line search state; applied by the next gradient pass)
    S_GP,          // g_i' p_i
    S_GPREVP,      // g_{i-1}' p_i
    S_GP_PREV,     // g_{i-1}' p_{i-1}
    S_MU,          // mu_i
    S_CZ2,         // ||C z||^2
    S_CZW,         // (C z)'(C w)
    S_ZG,          // z' g
    S_ZZD,         // sum z^2 d
    S_COST,        // Psi(w)
    S_K,           // omega-independent part of Phi (Eq. 2 terms with m = n, and the coil-combination remainder)
    S_CG_RZPREV,   // adjoint CG: r'z of the previous iteration
    S_CG_PQ,       // adjoint CG: p' H p
    S_CG_ALPHA,    // adjoint CG: step r'z / p'Hp
    S_CG_RR,       // adjoint CG: ||r||^2 after the last update
    S_CG_BB,       // adjoint CG: ||b||^2
    S_ADJ_DOT,     // lambda' C'C w (implicit derivative with respect to beta)
    S_ICT_TAU,     // drop-tolerance IC: this factorisation's tolerance droptol * H_max
    S_NSCAL
};

// Integer device state.
enum IState {
    I_ERR = 0, I_ITER, I_DONE0, I_DONE1, I_BAR_COUNT, I_BAR_GEN, I_NMASK, I_CG_IT, I_CG_DONE,
    I_ICT_BAD,  // drop-tolerance IC: a pivot <= 0 on the held pattern (reported after the fill check)
    I_NISTATE
};

// Setup works on chunks of 1024 consecutive voxels (mask compaction keeps voxel order).
constexpr int kChunk = 1024;

struct Pairs {
    int P;                  // number of echo pairs m < n
    int m[kMaxPairs], n[kMaxPairs];
    double dt[kMaxPairs];   // t_m - t_n
    double gmag[kMaxPairs]; // L |Gamma_mn| (1 in the field-map case)
    double gph[kMaxPairs];  // angle Gamma_mn (0 in the field-map case)
    float dtt[kMaxPairs];   // (t_m - t_n) 2^32 / (2 pi): a field value's fixed-point phase per unit
};

template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

// ------------------------------------------------------------------ reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum of Q doubles (fixed shuffle tree); result valid in thread 0.
template <int Q>
__device__ __forceinline__ void block_sum(double (&v)[Q], double* sbuf /* >= 32*Q */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = warp_sum(v[q]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < Q; ++q) sbuf[q * 32 + wid] = v[q];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            double x = lane < nw ? sbuf[q * 32 + lane] : 0.0;
            v[q] = warp_sum(x);
        }
    }
    __syncthreads();
}

// Sum partials[q * n + i] over i in a fixed order with the whole block; result in thread 0.
template <int Q>
__device__ __forceinline__ void sum_partials(const double* partials, int n, double (&out)[Q],
                                             double* sbuf) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        double a = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) a += __ldcg(partials + (size_t)q * n + i);
        out[q] = a;
    }
    block_sum<Q>(out, sbuf);
}

// Each block stores its Q partial sums; the last block to finish reduces all of them in
// block order and returns true in every thread of that block (out valid in thread 0).
template <int Q>
__device__ __forceinline__ bool last_block_reduce(double (&v)[Q], double* partials, unsigned* done,
                                                  double (&out)[Q], double* sbuf) {
    __shared__ bool s_last;
    block_sum<Q>(v, sbuf);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < Q; ++q) partials[(size_t)q * gridDim.x + blockIdx.x] = v[q];
        __threadfence();
        unsigned prev = atomicAdd(done, 1u);
        s_last = (prev == gridDim.x - 1);
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (!s_last) return false;
    sum_partials<Q>(partials, gridDim.x, out, sbuf);
    if (threadIdx.x == 0) *done = 0u;
    return true;
}

// ------------------------------------------------------------------ memory ordering

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Spin until *flag == want, at most `limit` polls.  Returns false on timeout.
__device__ __forceinline__ bool spin_until(const int* flag, int want, long long limit) {
    long long n = 0;
    unsigned ns = 32;
    while (ld_acquire(flag) != want) {
        if (++n > limit) return false;
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;  // backoff capped at 256 ns per poll
    }
    return true;
}

// Grid-wide barrier for a launch whose blocks are all co-resident (grids sized by
// occupancy).  Bounded: on timeout it records FM_ERR_TIMEOUT and returns false (the caller
// then exits).  Generation counting: thread 0 of each block reads the generation, then
// arrives with one acquire-release atomic (releasing the block's writes, which the block
// barrier has ordered before it); the last to arrive resets the count and publishes the next
// generation with a release store; the others poll it with acquire loads -- tightly at
// first, since most waits last a few microseconds, then with backoff.
__device__ __forceinline__ int atom_add_acq_rel(int* p, int v) {
    int old;
    asm volatile("atom.add.acq_rel.gpu.global.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// nblocks: the blocks that take part (every block of the grid by default; blocks beyond it
// must have left the kernel before the first barrier).
__device__ __forceinline__ bool grid_barrier(int* istate, long long limit, int nblocks = -1) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int* count = istate + I_BAR_COUNT;
        int* gen = istate + I_BAR_GEN;
        const int g0 = ld_acquire(gen);
        const int arrived = atom_add_acq_rel(count, 1);
        int ok = 1;
        if (arrived == (nblocks > 0 ? nblocks : (int)gridDim.x) - 1) {
            atomicExch(count, 0);
            st_release(gen, g0 + 1);
        } else {
            long long n = 0;
            while (ld_acquire(gen) == g0) {
                if (++n > limit) { ok = 0; break; }
                if (n > 64) __nanosleep(n > 4096 ? 256 : 32);
            }
        }
        if (!ok) atomicCAS(istate + I_ERR, 0, FM_ERR_TIMEOUT);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void set_err(int* istate, int code) { atomicCAS(istate + I_ERR, 0, code); }

// ------------------------------------------------------------------ launch wrappers

struct Geo {
    int nx, ny, nz;
    long long nv;
};

struct SetupArgs {
    Geo geo;
    int nc, L;
    Pairs pr;
    const void* y;      // complex [L][nc][nv]
    const void* smap;   // complex [nc][nv] or null
    const uint8_t* mask;// [nv] or null
    double te0, te1;    // first two echo times (Eq. 6)
    int wf;             // water-fat model: R_mn = L Gamma_mn conj(Z_m) Z_n with lgam below
    double lgam[2 * FM_MAX_ECHO * FM_MAX_ECHO];  // L Gamma_mn, complex, row m, column n
    void* rho;          // T [nv] compact order: sum |r_cdmn| (Eq. w0_wf weights), or null
    void* pairs;        // T2 [P][nv]: (|R_mn|, angle R_mn)
    void* coils;        // T2 [L][nc][nv]: (|W_cm|, angle W_cm), or null
    uint8_t* nb;        // [nv]
    void* w0;           // T [nv] initial field map (Eq. 6)
    int* vlist;         // [nv] voxel index of each mask voxel, ascending (compact order)
    int* chunk_off;     // [nchunks] mask voxels before each chunk (exclusive scan)
    double* partials;   // [nchunks]
    double* scal;
    int* istate;
};

struct DataArgs {
    Geo geo;
    int nc, L;
    Pairs pr;
    double beta;
    int literal;           // literal curvature over coils (nc > 1 and FM_CURV_LITERAL)
    int wf;                // water-fat Gamma: the literal curvature takes the runtime-coil path
    const void* pairs;     // compact order: [P][cap]
    const void* coils;     // compact order: [L][nc][cap]
    const uint8_t* nb;
    const int* vlist;      // [cap] voxel index of compact entry k
    // gradient pass
    const void* w_in;      // T [nv]
    const void* z;         // T [nv] direction applied with scal[S_ALPHA] (update fused), or null
    void* w_out;           // T [nv]
    void* g;               // T [nv]
    void* d;               // T [nv]
    // direction pass
    const void* p;         // T [nv]
    const void* z_old;     // T [nv]
    void* z_new;           // T [nv]
    const void* g_prev;    // T [nv]
    const void* ip_in;     // T [nv] stored inverse pivots (red-black apply) or null
    void* ip_out;          // T [nv] inverse pivots out (red-black factor) or null
    double* scal;
    double* partials;      // [4][grid] (+ [2][2][grid] for the line search)
    double* cost_hist;     // device [niter+1] or null
    double* alpha_hist;
    double* mu_hist;
    int* istate;
    int nls;
    long long spin_limit;
    int first_iter;        // direction pass: 1 -> mu = 0
};

struct IcArgs {
    Geo geo;
    int ntx, nty, ntz, ntiles;
    const int* order;      // [ntiles] tiles in a dependency-respecting order
    int* ticket;           // claim counter
    int* done;             // finished-tile counter
    double beta;
    const uint8_t* nb;
    // forward
    const void* d;         // T [nv] (compute pivots) or null
    const void* ip_in;     // T [nv] stored inverse pivots (apply only) or null
    const void* g;         // T [nv] right-hand side
    void* v;               // T [nv] forward result
    void* ip_out;          // T [nv] inverse pivots (compute mode)
    float* ip_lo_out;      // FP32 mode, nullable: low float of each inverse pivot (1/pi = hi + lo)
    void* face;            // per-tile face buffer (pivots, v, p)
    // backward
    const void* vin;       // T [nv]
    const void* ipb;       // T [nv]
    void* p;               // T [nv]
    const void* gdot;      // T [nv] or null: g for g'p
    const void* gpdot;     // T [nv] or null: g_prev for g_prev'p
    double* tile_part;     // [2][ntiles]
    double* scal;
    int* istate;
    long long spin_limit;
};

// IC with a drop tolerance (k_ict.cu).  The factor is held on a set of nh grid offsets o
// (each pointing to an earlier voxel in natural order): factor planes, each [nv] double:
// plane 0 = 1 / L_ii, plane 1 + h = L_{i,i+o_h}, plane 1 + nh = the substitution vector.
// The first six offsets are always IC(0)'s (-1,0,0), (0,-1,0), (0,0,-1) and the level-1 fill
// offsets (1,-1,0), (1,0,-1), (0,1,-1); with exactly those the sweeps take the unrolled
// kernels, with more (fill the tolerance keeps beyond level 1) the table-driven ones.
constexpr int kIctBaseOffsets = 6;
constexpr int kIctPlanes = kIctBaseOffsets + 2;
constexpr int kIctMaxOffsets = 64;  // largest held pattern; beyond it the call reports FM_ERR_FILL
constexpr int kIctMaxCand = 4096;   // largest set of candidate fill offsets the check examines
constexpr int kIctThreads = 1024;   // most threads per block of the level sweeps (one per (y, z) column)

// Tables of a held pattern (device, int): off[3 nh] (dx, dy, dz by plane), ord[nh] (planes in
// increasing column order), hs[nh] (1: a stencil offset, H_{i,i+o} = -beta), the correction
// pairs of each held offset in CSR form pp[nh + 1] / pr[2 np] (plane pairs (p1, p2) with
// o_p1 - o_p2 = o_h), and the candidate fill offsets outside the pattern with their pairs,
// qoff[3 nq], qp[nq + 1], qpr[2 nqp].
struct IctTables {
    int nh, nq;
    int B, C;             // level of voxel (x, y, z): x + B y + C z
    const int *off, *ord, *hs, *pp, *pr, *qoff, *qp, *qpr;
    unsigned* qflags;     // [ceil(nq / 32)] bit q set: candidate q reached the tolerance somewhere
};
struct IctArgs {
    Geo geo;
    double beta;
    const uint8_t* nb;
    const int* vlist;
    const void* d;         // T [nv]: factor (forward sweep), or null: apply the stored factor
    const void* g;         // T [nv] right-hand side
    double* L;             // [nh + 2][nv] factor planes
    IctTables tb;          // held pattern (table-driven kernels and the fill check)
    void* ip_out;          // T [nv] or null: 1/L_ii^2 (the pivots' inverses), factor mode
    void* p;               // T [nv] result (back substitution)
    const void* gdot;      // T [nv] or null: g for g'p
    const void* gpdot;     // T [nv] or null: g_prev for g_prev'p
    double* scal;
    double* partials;
    int* istate;
    long long spin_limit;
};

// Implicit differentiation of the converged field map: true curvature, the adjoint CG on
// H_true = diag(h) + beta C'C, and the derivatives with respect to beta and the images.
struct AdjArgs {
    Geo geo;
    int nc, L;
    Pairs pr;
    double beta;
    double te[FM_MAX_ECHO];
    const void* pairs;     // compact order: [P][nv] (|R_mn|, angle R_mn)
    const uint8_t* nb;
    const int* vlist;
    const void* w;         // T [nv] field map at which everything is evaluated
    const void* rhs;       // T [nv] right-hand side b
    void* h;               // T [nv] true curvature
    void* x;               // T [nv] CG iterate (lambda)
    void* r;               // T [nv] residual
    const void* z;         // T [nv] preconditioned residual
    const void* p_old;     // T [nv]
    void* p_new;           // T [nv]
    void* q;               // T [nv] H_true p
    double tol2;           // stop when ||r||^2 <= tol2 ||b||^2
    int maxiter;
    int identity_pc;       // 1: no preconditioner (z = r; the update pass supplies r'r as r'z)
    const void* rho;       // T compact [nv]: PWLS weights (Eq. w0_wf)
    const void* x0;        // T [nv]: PWLS start (the sweep's map)
    double fat_re[FM_MAX_ECHO], fat_im[FM_MAX_ECHO];  // second basis column of Eq. gamma
    double ginv[8];        // (gamma^H gamma)^{-1}, complex 2 x 2 row-major
    void* water;           // complex [nv]
    void* fat;             // complex [nv]
    const void* y;         // complex [L][nc][nv] images
    const void* smap;      // complex [nc][nv] or null
    const void* lam;       // T [nv]
    void* dldy;            // complex [L][nc][nv]
    double* scal;
    double* partials;
    int* istate;
};

template <typename T> cudaError_t launch_setup(const SetupArgs& a, cudaStream_t s);
template <typename T> cudaError_t launch_masked_copy(const void* in, void* out, const uint8_t* nb, long long nv,
                                                     int grid, cudaStream_t s);
template <typename T> cudaError_t launch_grad(const DataArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_ls(const DataArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_pdiag(const DataArgs& a, int mode, int grid, cudaStream_t s);
template <typename T> int ls_max_blocks_per_sm(const DataArgs& a);
template <typename T> cudaError_t launch_rb_black(const DataArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_rb_red(const DataArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_ic_fwd(const IcArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_ic_bwd(const IcArgs& a, int grid, cudaStream_t s);
cudaError_t launch_inv_pivot64(const float* hi, const float* lo, double* out, long long nv, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_true_curv(const AdjArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_cg_init(const AdjArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_cg_dir(const AdjArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_cg_upd(const AdjArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_lap_dot(const AdjArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_dldy(const AdjArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_pwls_init(const AdjArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_wf_sweep(const AdjArgs& a, int nsweep, double wlo, double whi, int grid,
                                                  cudaStream_t s);
template <typename T> cudaError_t launch_wf_amp(const AdjArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_ict_tau(const DataArgs& a, double droptol, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_ict_fwd(const IctArgs& a, int grid, int block, cudaStream_t s);
template <typename T> cudaError_t launch_ict_bwd(const IctArgs& a, int grid, int block, cudaStream_t s);
template <typename T> cudaError_t launch_ict_check(const IctArgs& a, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_ictg_fwd(const IctArgs& a, int grid, int block, cudaStream_t s);
template <typename T> cudaError_t launch_ictg_bwd(const IctArgs& a, int grid, int block, cudaStream_t s);
template <typename T> int ict_max_blocks_per_sm(int block);
template <typename T> int ictg_max_blocks_per_sm(int block);
template <typename T> int ic_tz();
template <typename T> size_t ic_face_bytes_per_tile();
template <typename T> int ic_max_blocks_per_sm(bool bwd);  // resident IC sweep blocks per SM

constexpr int kThreads = 256;     // data-term / stencil kernels
constexpr int kTileX = 32, kTileY = 32;

}  // namespace fm
