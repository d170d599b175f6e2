// k_ic.cu -- IC(0) factorisation and triangular solves in the natural (x fastest, then y,
// then z) order, as tile wavefronts (Sec. III-B, Eq. 12; the "precondition" step of the
// Algorithm box).
//
// H = diag(d) + beta C'C on the mask voxels has, in natural order, the strictly lower
// entries E_jk = -beta for the in-mask neighbours k in {j-1, j-nx, j-nx*ny}.  The 6-neighbour
// grid graph has no triangles, so IC(0) (zero fill-in) only changes the diagonal:
//   pi_j = H_jj - sum_{k lower nbr} E_jk^2 / pi_k = d_j + beta n_j - beta^2 sum_k 1/pi_k,
//   L = (Pi + E) Pi^{-1/2},   L L' = H on H's nonzero set.
// Forward (fused with the pivots): (Pi + E) v = g  ->  v_j = (g_j + beta sum_{k lower} v_k) / pi_j.
// Back:                           (Pi + E') p = Pi v  ->  p_j = v_j + beta/pi_j sum_{k upper} p_k.
// Voxels outside the mask are identity rows with 1/pi = v = p = 0, so every sum may run over
// all grid neighbours: an outside neighbour contributes exactly 0.
//
// Parallel schedule: voxel (x, y, z) depends on (x-1, y, z), (x, y-1, z), (x, y, z-1), so
// every hyperplane x + y + z = const is independent.  The grid is cut into 32 x 32 x 8
// tiles; a CTA claims tiles through an atomic ticket in a dependency-respecting order (a
// tile's predecessors always hold smaller tickets, so no co-residency is assumed), starts
// the asynchronous copy of the tile's inputs into shared memory, waits on the predecessors'
// ready flags (bounded spin), and sweeps the tile's 70 local hyperplanes: lane = y,
// warp = z, and each thread walks its x row one step per hyperplane, taking the -y value
// from the neighbouring lane by shuffle, the -z value from the warp below through shared
// memory and the -x value from its own register.  Outputs are written back row-coalesced
// and the tile's flag is released before the back sweep's dot products.
//
// Pivot arithmetic: FP64 mode uses IEEE double.  FP32 mode carries the pivot recurrence
// in double-float (an unevaluated sum hi + lo of two floats, about 46 significant bits)
// on the FP32 pipes, because the GB300 FP64 pipe issues at about 1/64 of the FP32 rate and
// sits on the sweep's critical path; the solves themselves run in float.
#include "fm_internal.h"

namespace fm {

constexpr int kTZ = 8;
constexpr int kRows = kTZ * 32;  // rows of 32 x-values per tile (== threads per CTA)
constexpr int kFaceN = 32 * kTZ + 32 * kTZ + 32 * 32;  // pivot values per tile: +x, +y, +z faces

// ------------------------------------------------------------------ double-float

struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ DF df_quick(float a, float b) {  // requires |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
    const DF s = df_two_sum(x.hi, y.hi);
    const DF t = df_two_sum(x.lo, y.lo);
    DF u = df_quick(s.hi, __fadd_rn(s.lo, t.hi));
    return df_quick(u.hi, __fadd_rn(u.lo, t.lo));
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return df_quick(p, e);
}
__device__ __forceinline__ DF df_from(double v) {
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}
__device__ __forceinline__ DF df_neg(DF x) { return {-x.hi, -x.lo}; }
// 1/x by one Newton step on the float reciprocal, carried in double-float
__device__ __forceinline__ DF df_recip(DF x) {
    const float r = __frcp_rn(x.hi);
    // e = 1 - x r exactly enough: x.hi r + x.lo r in double-float
    const float p = __fmul_rn(x.hi, r);
    float pe = __fmaf_rn(x.hi, r, -p);
    pe = __fmaf_rn(x.lo, r, pe);
    const DF xr = df_quick(p, pe);
    const DF e = df_add({1.0f, 0.0f}, df_neg(xr));
    return df_add({r, 0.0f}, df_mul({r, 0.0f}, e));
}

// Pivot arithmetic per precision mode: P is the carried type (double or DF, 8 bytes).
template <typename T> struct PivOps;
template <> struct PivOps<double> {
    using P = double;
    static __device__ __forceinline__ P zero() { return 0.0; }
    static __device__ __forceinline__ P add(P a, P b) { return a + b; }
    // H_jj - beta^2 s with H_jj = d + beta n; returns 1/pi and whether pi > 0
    static __device__ __forceinline__ P inv_pivot(double d, int n, double beta, P s, bool& ok) {
        const double piv = d + beta * (double)n - beta * beta * s;
        ok = piv > 0.0;
        return ok ? 1.0 / piv : 0.0;
    }
    static __device__ __forceinline__ double to_T(P x) { return x; }
};
template <> struct PivOps<float> {
    using P = DF;
    static __device__ __forceinline__ P zero() { return {0.0f, 0.0f}; }
    static __device__ __forceinline__ P add(P a, P b) { return df_add(a, b); }
    static __device__ __forceinline__ P inv_pivot(float d, int n, double beta, P s, bool& ok) {
        const DF b = df_from(beta), b2 = df_from(beta * beta);
        const DF h = df_add({d, 0.0f}, df_mul(b, {(float)n, 0.0f}));
        const DF piv = df_add(h, df_neg(df_mul(b2, s)));
        ok = piv.hi > 0.0f;
        return ok ? df_recip(piv) : DF{0.0f, 0.0f};
    }
    static __device__ __forceinline__ float to_T(P x) { return x.hi; }
};

// Pivot faces are written by other CTAs of the same launch: read them through L2.
__device__ __forceinline__ double ld_face(const double* p) { return __ldcg(p); }
__device__ __forceinline__ DF ld_face(const DF* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}

// ------------------------------------------------------------------ asynchronous staging

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp4(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp8(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp16(void* s, const void* g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Start copying this thread's row (ly, lz) = (r & 31, r >> 5) of a T tile into s[r * 32 ..];
// elements outside the grid are filled with `fill`.
template <typename T>
__device__ __forceinline__ void stage_row(T* s, const T* g, int r, int x0, int y0, int z0, const Geo& geo,
                                          T fill) {
    T* srow = s + r * 32;
    const int y = y0 + (r & 31), z = z0 + (r >> 5);
    if (y >= geo.ny || z >= geo.nz) {
#pragma unroll
        for (int i = 0; i < 32; ++i) srow[i] = fill;
        return;
    }
    const T* grow = g + ((long long)z * geo.ny + y) * geo.nx + x0;
    const int nvalid = min(32, geo.nx - x0);
    if (nvalid == 32 && ((reinterpret_cast<uintptr_t>(grow) & 15) == 0)) {
        constexpr int per = 16 / sizeof(T);
#pragma unroll
        for (int i = 0; i < 32; i += per) cp16(srow + i, grow + i);
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            if (i < nvalid) {
                if (sizeof(T) == 4) cp4(srow + i, grow + i);
                else cp8(srow + i, grow + i);
            } else {
                srow[i] = fill;
            }
        }
    }
}

__device__ __forceinline__ void stage_row_u8(uint8_t* s, const uint8_t* g, int r, int x0, int y0, int z0,
                                             const Geo& geo) {
    uint8_t* srow = s + r * 32;
    const int y = y0 + (r & 31), z = z0 + (r >> 5);
    if (y >= geo.ny || z >= geo.nz) {
#pragma unroll
        for (int i = 0; i < 32; ++i) srow[i] = 0;
        return;
    }
    const uint8_t* grow = g + ((long long)z * geo.ny + y) * geo.nx + x0;
    const int nvalid = min(32, geo.nx - x0);
    if (nvalid == 32 && ((reinterpret_cast<uintptr_t>(grow) & 15) == 0)) {
        cp16(srow, grow);
        cp16(srow + 16, grow + 16);
    } else {
        uint8_t v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = i < nvalid ? grow[i] : (uint8_t)0;
#pragma unroll
        for (int i = 0; i < 32; ++i) srow[i] = v[i];
    }
}

template <typename T>
struct FwdSmem {
    using P = typename PivOps<T>::P;
    static constexpr size_t bytes = 2 * kRows * 32 * sizeof(T) + (kTZ * 32 * 2 + 1024 + 2 * kTZ * 32) * sizeof(P) +
                                    (kTZ * 32 * 2 + 1024 + 2 * kTZ * 32) * sizeof(T) + kRows * 32;
};
template <typename T>
struct BwdSmem {
    static constexpr size_t bytes = 2 * kRows * 32 * sizeof(T) + (kTZ * 32 * 2 + 1024 + 2 * kTZ * 32) * sizeof(T);
};

// mode 0: pivots from d (factor + forward); mode 1: stored 1/pi (forward only)
template <typename T>
__global__ void __launch_bounds__(32 * kTZ) k_ic_fwd(IcArgs a, int mode) {
    using Ops = PivOps<T>;
    using P = typename Ops::P;
    extern __shared__ __align__(16) unsigned char smem[];
    T* sg = (T*)smem;                              // [kTZ][32][32]: g, then v
    T* sd = sg + kRows * 32;                       // d (or stored 1/pi), then 1/pi
    P* fx_ip = (P*)(sd + kRows * 32);              // [kTZ][32] (lz, ly)
    P* fy_ip = fx_ip + kTZ * 32;                   // [kTZ][32] (lz, lx)
    P* fz_ip = fy_ip + kTZ * 32;                   // [32][32]  (ly, lx)
    P* zb_ip = fz_ip + 1024;                       // [2][kTZ][32]
    T* fx_v = (T*)(zb_ip + 2 * kTZ * 32);
    T* fy_v = fx_v + kTZ * 32;
    T* fz_v = fy_v + kTZ * 32;
    T* zb_v = fz_v + 1024;
    uint8_t* snb = (uint8_t*)(zb_v + 2 * kTZ * 32);  // [kTZ][32][32]
    __shared__ int s_tile;

    const Geo geo = a.geo;
    const int nx = geo.nx, ny = geo.ny, nz = geo.nz;
    const long long nxy = (long long)nx * ny;
    const int tid = threadIdx.x, lane = tid & 31, wz = tid >> 5;
    const T* g = (const T*)a.g;
    const T* d = (const T*)a.d;
    const T* ipin = (const T*)a.ip_in;
    T* v = (T*)a.v;
    T* ipo = (T*)a.ip_out;
    P* face = (P*)a.face;
    const T betaT = (T)a.beta;

    for (;;) {
        if (tid == 0) {
            const int t = atomicAdd(a.ticket, 1);
            s_tile = t < a.ntiles ? a.order[t] : -1;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0) break;
        const int X = tile % a.ntx, Y = (tile / a.ntx) % a.nty, Z = tile / (a.ntx * a.nty);
        const int x0 = X * 32, y0 = Y * 32, z0 = Z * kTZ;

        // start the copies of this tile's inputs (they do not depend on other tiles)
        stage_row<T>(sg, g, tid, x0, y0, z0, geo, T(0));
        stage_row<T>(sd, mode == 0 ? d : ipin, tid, x0, y0, z0, geo, T(0));
        if (mode == 0) stage_row_u8(snb, a.nb, tid, x0, y0, z0, geo);
        // wait for the -x, -y, -z neighbour tiles
        if (tid == 0) {
            bool ok = true;
            if (X > 0) ok = spin_until(a.flags + tile - 1, 1, a.spin_limit) && ok;
            if (Y > 0) ok = spin_until(a.flags + tile - a.ntx, 1, a.spin_limit) && ok;
            if (Z > 0) ok = spin_until(a.flags + tile - a.ntx * a.nty, 1, a.spin_limit) && ok;
            if (!ok) set_err(a.istate, FM_ERR_TIMEOUT);
            __threadfence();
        }
        __syncthreads();
        // faces produced by the neighbour tiles in this launch (read through L2): thread tid
        // owns x-face and y-face entry tid and z-face entries tid + 256 q
        {
            const int hi = tid >> 5, lo = tid & 31;
            P ipx = Ops::zero(), ipy = Ops::zero(), ipz[4];
            T vx = 0, vy = 0, vz[4];
            if (X > 0 && y0 + lo < ny && z0 + hi < nz) {
                vx = __ldcg(v + (long long)(z0 + hi) * nxy + (long long)(y0 + lo) * nx + (x0 - 1));
                if (mode == 0) ipx = ld_face(face + (size_t)(tile - 1) * kFaceN + tid);
            }
            if (Y > 0 && x0 + lo < nx && z0 + hi < nz) {
                vy = __ldcg(v + (long long)(z0 + hi) * nxy + (long long)(y0 - 1) * nx + (x0 + lo));
                if (mode == 0) ipy = ld_face(face + (size_t)(tile - a.ntx) * kFaceN + 32 * kTZ + tid);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = tid + 256 * q, ly = i >> 5, lx = i & 31;
                ipz[q] = Ops::zero();
                vz[q] = 0;
                if (Z > 0 && x0 + lx < nx && y0 + ly < ny) {
                    vz[q] = __ldcg(v + (long long)(z0 - 1) * nxy + (long long)(y0 + ly) * nx + (x0 + lx));
                    if (mode == 0) ipz[q] = ld_face(face + (size_t)(tile - a.ntx * a.nty) * kFaceN + 64 * kTZ + i);
                }
            }
            fx_ip[tid] = ipx;
            fx_v[tid] = vx;
            fy_ip[tid] = ipy;
            fy_v[tid] = vy;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                fz_ip[tid + 256 * q] = ipz[q];
                fz_v[tid + 256 * q] = vz[q];
            }
        }
        cp_wait_all();
        __syncthreads();

        // sweep the local hyperplanes s = lx + ly + lz
        const int ly = lane, lz = wz;
        P out_ip = Ops::zero();
        T out_v = 0;
        bool bad = false;
        P* myface = face + (size_t)tile * kFaceN;
        for (int s = 0; s < 64 + kTZ - 2; ++s) {
            P up_ip;
            if constexpr (sizeof(P) == 8 && sizeof(T) == 8) {
                up_ip = __shfl_up_sync(0xffffffffu, out_ip, 1);
            } else {
                DF o = *reinterpret_cast<DF*>(&out_ip);
                DF u{__shfl_up_sync(0xffffffffu, o.hi, 1), __shfl_up_sync(0xffffffffu, o.lo, 1)};
                up_ip = *reinterpret_cast<P*>(&u);
            }
            const T up_v = __shfl_up_sync(0xffffffffu, out_v, 1);
            const int lx = s - ly - lz;
            if (lx >= 0 && lx < 32) {
                const int i = (lz * 32 + ly) * 32 + lx;
                P ipj = Ops::zero();
                T vj = 0;
                const P xip = lx == 0 ? fx_ip[lz * 32 + ly] : out_ip;
                const T xv = lx == 0 ? fx_v[lz * 32 + ly] : out_v;
                const P yip = ly == 0 ? fy_ip[lz * 32 + lx] : up_ip;
                const T yv = ly == 0 ? fy_v[lz * 32 + lx] : up_v;
                const int q = ((s - 1) & 1) * kTZ * 32 + (lz - 1) * 32 + ly;
                const P zip = lz == 0 ? fz_ip[ly * 32 + lx] : zb_ip[q];
                const T zv = lz == 0 ? fz_v[ly * 32 + lx] : zb_v[q];
                if (mode == 0) {
                    const uint8_t b = snb[i];
                    if (b & NB_IN) {
                        bool ok;
                        ipj = Ops::inv_pivot(sd[i], __popc((unsigned)(b >> 1) & 0x3fu), a.beta,
                                             Ops::add(Ops::add(xip, yip), zip), ok);
                        bad |= !ok;
                        vj = (sg[i] + betaT * ((xv + yv) + zv)) * (T)Ops::to_T(ipj);
                    }
                    sd[i] = (T)Ops::to_T(ipj);
                } else {
                    const T ipt = sd[i];
                    vj = (sg[i] + betaT * ((xv + yv) + zv)) * ipt;
                }
                sg[i] = vj;
                out_ip = ipj;
                out_v = vj;
                zb_ip[(s & 1) * kTZ * 32 + lz * 32 + ly] = ipj;
                zb_v[(s & 1) * kTZ * 32 + lz * 32 + ly] = vj;
                if (mode == 0) {
                    if (lx == 31) myface[lz * 32 + ly] = ipj;
                    if (ly == 31) myface[32 * kTZ + lz * 32 + lx] = ipj;
                    if (lz == kTZ - 1) myface[64 * kTZ + ly * 32 + lx] = ipj;
                }
            }
            __syncthreads();
        }
        if (bad) set_err(a.istate, FM_ERR_NOT_PD);

        // write back row-coalesced (warp lz writes its 32 rows, lane = x), then publish
        {
            const int nvalid = min(32, nx - x0);
            const int z = z0 + wz;
            if (z < nz && lane < nvalid) {
                for (int ly2 = 0; ly2 < 32 && y0 + ly2 < ny; ++ly2) {
                    const long long j = (long long)z * nxy + (long long)(y0 + ly2) * nx + x0 + lane;
                    const int i = (wz * 32 + ly2) * 32 + lane;
                    v[j] = sg[i];
                    if (mode == 0 && ipo) ipo[j] = sd[i];
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            st_release(a.flags + tile, 1);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(32 * kTZ) k_ic_bwd(IcArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    T* sv = (T*)smem;                 // [kTZ][32][32]: v, then p
    T* sip = sv + kRows * 32;         // 1/pi
    T* fx = sip + kRows * 32;         // [kTZ][32] (lz, ly) p at x0 + 32
    T* fy = fx + kTZ * 32;            // [kTZ][32] (lz, lx) p at y0 + 32
    T* fz = fy + kTZ * 32;            // [32][32] (ly, lx) p at z0 + kTZ
    T* zb = fz + 1024;                // [2][kTZ][32]
    __shared__ int s_tile;
    __shared__ bool s_last;
    __shared__ double sbuf[2 * 32];

    const Geo geo = a.geo;
    const int nx = geo.nx, ny = geo.ny, nz = geo.nz;
    const long long nxy = (long long)nx * ny;
    const int tid = threadIdx.x, lane = tid & 31, wz = tid >> 5;
    const T* vin = (const T*)a.vin;
    const T* ipb = (const T*)a.ipb;
    T* p = (T*)a.p;
    const T* gd = (const T*)a.gdot;
    const T* gpd = (const T*)a.gpdot;
    const T beta = (T)a.beta;

    for (;;) {
        if (tid == 0) {
            const int t = atomicAdd(a.ticket, 1);
            s_tile = t < a.ntiles ? a.order[a.ntiles - 1 - t] : -1;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0) break;
        const int X = tile % a.ntx, Y = (tile / a.ntx) % a.nty, Z = tile / (a.ntx * a.nty);
        const int x0 = X * 32, y0 = Y * 32, z0 = Z * kTZ;

        stage_row<T>(sv, vin, tid, x0, y0, z0, geo, T(0));
        stage_row<T>(sip, ipb, tid, x0, y0, z0, geo, T(0));
        if (tid == 0) {
            bool ok = true;
            if (X + 1 < a.ntx) ok = spin_until(a.flags + tile + 1, 1, a.spin_limit) && ok;
            if (Y + 1 < a.nty) ok = spin_until(a.flags + tile + a.ntx, 1, a.spin_limit) && ok;
            if (Z + 1 < a.ntz) ok = spin_until(a.flags + tile + a.ntx * a.nty, 1, a.spin_limit) && ok;
            if (!ok) set_err(a.istate, FM_ERR_TIMEOUT);
            __threadfence();
        }
        __syncthreads();
        {
            const int hi = tid >> 5, lo = tid & 31;
            T qx = 0, qy = 0, qz[4];
            if (X + 1 < a.ntx && y0 + lo < ny && z0 + hi < nz)
                qx = __ldcg(p + (long long)(z0 + hi) * nxy + (long long)(y0 + lo) * nx + (x0 + 32));
            if (Y + 1 < a.nty && x0 + lo < nx && z0 + hi < nz)
                qy = __ldcg(p + (long long)(z0 + hi) * nxy + (long long)(y0 + 32) * nx + (x0 + lo));
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = tid + 256 * q, ly = i >> 5, lx = i & 31;
                qz[q] = 0;
                if (Z + 1 < a.ntz && x0 + lx < nx && y0 + ly < ny)
                    qz[q] = __ldcg(p + (long long)(z0 + kTZ) * nxy + (long long)(y0 + ly) * nx + (x0 + lx));
            }
            fx[tid] = qx;
            fy[tid] = qy;
#pragma unroll
            for (int q = 0; q < 4; ++q) fz[tid + 256 * q] = qz[q];
        }
        cp_wait_all();
        __syncthreads();

        const int ly = lane, lz = wz;
        T out = 0;
        for (int s = 64 + kTZ - 3; s >= 0; --s) {
            const T dn = __shfl_down_sync(0xffffffffu, out, 1);
            const int lx = s - ly - lz;
            if (lx >= 0 && lx < 32) {
                const int i = (lz * 32 + ly) * 32 + lx;
                const T px = lx == 31 ? fx[lz * 32 + ly] : out;
                const T py = ly == 31 ? fy[lz * 32 + lx] : dn;
                const T pz = lz == kTZ - 1 ? fz[ly * 32 + lx] : zb[((s + 1) & 1) * kTZ * 32 + (lz + 1) * 32 + ly];
                const T pj = sv[i] + beta * sip[i] * ((px + py) + pz);
                sv[i] = pj;
                out = pj;
                zb[(s & 1) * kTZ * 32 + lz * 32 + ly] = pj;
            }
            __syncthreads();
        }

        // write back, publish, then the dot products (off the wavefront's critical path)
        const int nvalid = min(32, nx - x0);
        const int z = z0 + wz;
        const bool zin = z < nz && lane < nvalid;
        if (zin) {
            for (int ly2 = 0; ly2 < 32 && y0 + ly2 < ny; ++ly2)
                p[(long long)z * nxy + (long long)(y0 + ly2) * nx + x0 + lane] = sv[(wz * 32 + ly2) * 32 + lane];
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            st_release(a.flags + tile, 1);
        }
        if (a.tile_part) {
            double acc[2] = {0.0, 0.0};
            if (zin) {
                for (int ly2 = 0; ly2 < 32 && y0 + ly2 < ny; ++ly2) {
                    const long long j = (long long)z * nxy + (long long)(y0 + ly2) * nx + x0 + lane;
                    const T pj = sv[(wz * 32 + ly2) * 32 + lane];
                    if (gd) acc[0] += (double)(gd[j] * pj);
                    if (gpd) acc[1] += (double)(gpd[j] * pj);
                }
            }
            block_sum<2>(acc, sbuf);
            if (tid == 0) {
                a.tile_part[tile] = acc[0];
                a.tile_part[a.ntiles + tile] = acc[1];
                __threadfence();
                const int prev = atomicAdd(a.done, 1);
                s_last = (prev == a.ntiles - 1);
                if (s_last) __threadfence();
            }
            __syncthreads();
            if (s_last) {
                double tot[2];
                sum_partials<2>(a.tile_part, a.ntiles, tot, sbuf);
                if (tid == 0) {
                    a.scal[S_GP] = tot[0];
                    a.scal[S_GPREVP] = tot[1];
                    if (!isfinite(tot[0]) || !isfinite(tot[1])) set_err(a.istate, FM_ERR_NONFINITE);
                }
            }
        }
        __syncthreads();
    }
}

template <typename T> int ic_tz() { return kTZ; }
template <typename T> size_t ic_smem_bytes() {
    return FwdSmem<T>::bytes > BwdSmem<T>::bytes ? FwdSmem<T>::bytes : BwdSmem<T>::bytes;
}

template <typename T>
static cudaError_t prep() {
    static bool done = false;  // attributes are per function, set once per process
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_ic_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)FwdSmem<T>::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_ic_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BwdSmem<T>::bytes);
    if (e == cudaSuccess) done = true;
    return e;
}

template <typename T>
int ic_max_blocks_per_sm() {
    if (prep<T>() != cudaSuccess) return 0;
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_ic_fwd<T>, 32 * kTZ, FwdSmem<T>::bytes) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ic_bwd<T>, 32 * kTZ, BwdSmem<T>::bytes) != cudaSuccess)
        return 0;
    return a < b ? a : b;
}

template <typename T>
cudaError_t launch_ic_fwd(const IcArgs& a, int grid, cudaStream_t s) {
    cudaError_t e = prep<T>();
    if (e != cudaSuccess) return e;
    k_ic_fwd<T><<<grid, 32 * kTZ, FwdSmem<T>::bytes, s>>>(a, a.d ? 0 : 1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ic_bwd(const IcArgs& a, int grid, cudaStream_t s) {
    cudaError_t e = prep<T>();
    if (e != cudaSuccess) return e;
    k_ic_bwd<T><<<grid, 32 * kTZ, BwdSmem<T>::bytes, s>>>(a);
    return cudaGetLastError();
}

#define FM_INST(T)                                                            \
    template cudaError_t launch_ic_fwd<T>(const IcArgs&, int, cudaStream_t);  \
    template cudaError_t launch_ic_bwd<T>(const IcArgs&, int, cudaStream_t);  \
    template int ic_tz<T>();                                                  \
    template size_t ic_smem_bytes<T>();                                       \
    template int ic_max_blocks_per_sm<T>();
FM_INST(float)
FM_INST(double)

}  // namespace fm
