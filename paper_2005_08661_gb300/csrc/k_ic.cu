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
// the asynchronous copy of the tile's inputs into shared memory, forms H_jj and sweeps the
// tile's 70 local hyperplanes: lane = y, warp = z, and each thread walks its x row one step
// per hyperplane, taking the -y value from the neighbouring lane by shuffle, the -z value
// from the warp below through shared memory and the -x value from its own register.  The
// step body is branch-free (divergent branches cost more per step than the idle lanes'
// arithmetic).  In both sweeps faces stream between tiles while they sweep (see "streamed
// faces" below): a tile runs a fixed number of hyperplanes behind its predecessors instead
// of waiting for them to finish.  The row-coalesced write-back of the whole tile follows the
// sweep.
//
// Pivot arithmetic.  FP64 mode uses IEEE double.  FP32 mode carries each inverse pivot as
// an unevaluated pair a + b of floats (about 46 significant bits, like double-float), but
// arranged so that the hi part a is exactly the float recurrence a_j = 1/fl(H - beta^2 sum a_k)
// -- a short dependency chain -- while b, the first-order correction, is formed from
// error-free residuals (two-sum / two-product) of that chain and the neighbours' b:
//   pi = pi_f + dpi,  dpi = (rounding residuals of pi_f) + H_lo - beta^2 (sum b_k + sum errors),
//   1/pi = a (1 + e_r - dpi a) + O(eps^2),  e_r = 1 - pi_f a  (exact by FMA),
// so b = a (e_r - dpi a) with a relative truncation of order (dpi/pi)^2 ~ 1e-14.  The GB300
// FP64 pipe issues at about 1/64 of the FP32 rate and would sit on the sweep's critical path.
#include "fm_internal.h"

namespace fm {

// ------------------------------------------------------------------ split pivot (FP32 mode)

struct PF {
    float a, b;  // inverse pivot = a + b
};

__device__ __forceinline__ void two_sum(float x, float y, float& s, float& e) {
    s = __fadd_rn(x, y);
    const float bb = __fsub_rn(s, x);
    e = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bb)), __fsub_rn(y, bb));
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct PivScal {     // beta-derived constants of the pivot recurrence
    float bh, bl;    // beta = bh + bl
    float b2h, b2l;  // beta^2 = b2h + b2l
};

// Per precision: H_jj = d_j + beta n_j is formed once per voxel while the tile is staged
// (stored as hi in the d slot, -1 outside the mask, and, in FP32 mode, its low part in a
// second array); the sweep then only needs 1/pi_j = 1/(H_jj - beta^2 sum_k 1/pi_k).
template <typename T> struct PivOps;
template <> struct PivOps<double> {
    using P = double;
    static constexpr bool kLo = false;
    static __device__ __forceinline__ P zero() { return 0.0; }
    static __device__ __forceinline__ double hi(P x) { return x; }
    static __device__ __forceinline__ double lo(P) { return 0.0; }
    static __device__ __forceinline__ P make(double a, double) { return a; }
    static __device__ __forceinline__ void form_h(double d, int n, double beta, const PivScal&, double& hH,
                                                  double&) {
        hH = d + beta * (double)n;
    }
    static __device__ __forceinline__ P inv_pivot(double hH, double, double beta, const PivScal&, P x, P y, P z,
                                                  bool& ok) {
        const double piv = hH - beta * beta * ((x + y) + z);
        ok = piv > 0.0;
        return ok ? 1.0 / piv : 0.0;
    }
};
template <> struct PivOps<float> {
    using P = PF;
    static constexpr bool kLo = true;
    static __device__ __forceinline__ P zero() { return {0.0f, 0.0f}; }
    static __device__ __forceinline__ float hi(P x) { return x.a; }
    static __device__ __forceinline__ float lo(P x) { return x.b; }
    static __device__ __forceinline__ P make(float a, float b) { return {a, b}; }
    // H = d + beta n as hH + hL (n <= 6, so bh * n has one rounding, recovered by FMA)
    static __device__ __forceinline__ void form_h(float d, int n, double, const PivScal& c, float& hH, float& hL) {
        const float fn = (float)n;
        const float bn = __fmul_rn(c.bh, fn);
        const float bn_e = __fmaf_rn(c.bh, fn, -bn);
        float hE;
        two_sum(d, bn, hH, hE);
        hL = __fadd_rn(hE, __fmaf_rn(c.bl, fn, bn_e));
    }
    static __device__ __forceinline__ P inv_pivot(float hH, float hL, double, const PivScal& c, P x, P y, P z,
                                                  bool& ok) {
        // hi chain: S = (a_x + a_y) + a_z, pi_f = hH - b2h S, a ~ 1/pi_f
        float s1, e1, S, e2;
        two_sum(x.a, y.a, s1, e1);
        two_sum(s1, z.a, S, e2);
        const float th = __fmul_rn(c.b2h, S);
        const float tl = __fmaf_rn(c.b2h, S, -th);
        float pf, pe;
        two_sum(hH, -th, pf, pe);
        ok = pf > 0.0f;
        const float a = rcp_approx(pf);
        const float er = __fmaf_rn(-pf, a, 1.0f);  // exact residual of the reciprocal
        // lo: dpi = pe + hL - tl - b2l S - b2h (e1 + e2 + sum b)
        const float base = __fsub_rn(__fadd_rn(pe, hL), __fmaf_rn(c.b2l, S, tl));
        const float sb = __fadd_rn(__fadd_rn(__fadd_rn(x.b, y.b), z.b), __fadd_rn(e1, e2));
        const float dpi = __fmaf_rn(-c.b2h, sb, base);
        const float b = __fmul_rn(a, __fmaf_rn(-dpi, a, er));
        return ok ? P{a, b} : P{0.0f, 0.0f};
    }
};


// Faces are written by other CTAs of the same launch: read them through L2.
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ PF ld_cg(const PF* p) {
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

// Start copying row r = (ly, lz) = (r & 31, r >> 5) of a T tile into s[r * 32 ..]; elements
// outside the grid are filled with `fill`.
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

// ------------------------------------------------------------------ tile geometry

#ifndef FM_IC_CSF
#define FM_IC_CSF 4
#endif
#ifndef FM_IC_CSB
#define FM_IC_CSB 8
#endif
constexpr int kTZ = 8;              // tile = 32 x 32 x 8 voxels, 8 compute warps
constexpr int kSteps = 62 + kTZ;    // local hyperplanes lx + ly + lz of a tile
// Steps per chunk (the unit of the face hand-off): forward 4, back substitution 8.  With 8
// the back substitution's per-chunk face flush lines up with what its successors' chunks
// need (x / y faces 31 steps later, z faces 7); at most kTZ, one z diagonal per warp.
constexpr int kCSF = FM_IC_CSF, kCSB = FM_IC_CSB;
static_assert(kCSB <= kTZ, "the back substitution's face flush takes one z diagonal per warp");
constexpr int kCompute = 32 * kTZ;  // compute threads
// Warps that fetch incoming faces, taking alternate chunks, so that the polls for consecutive
// chunks are in flight together (one poll round trip is longer than a chunk of the back
// substitution's steps)
constexpr int kFetchF = 2, kFetchB = 2;
constexpr int kThreadsIC = kCompute + 32 * kFetchF;
constexpr int kThreadsB = kCompute + 32 * kFetchB;

// Face layout per tile (counts of values): x face [TZ][32] (lz, ly), y face [TZ][32]
// (lz, lx), z face [32][32].  In shared memory the z face is (ly, lx); in the forward
// sweep's global face buffer it is stored by diagonals t = lx + ly (see zdiag), so the
// entries produced at one step, and fetched for one step, are contiguous.
struct FN {
    static constexpr int x = 0, y = kTZ * 32, z = 2 * kTZ * 32, n = 2 * kTZ * 32 + 1024;
};

template <typename T>
struct FwdSmem {
    using P = typename PivOps<T>::P;
    static constexpr int nface = FN::n + 2 * kTZ * 32;  // incoming faces + z exchange
    static constexpr size_t bytes = (PivOps<T>::kLo ? 3 : 2) * kTZ * 1024 * sizeof(T) +
                                    nface * (sizeof(P) + sizeof(T)) + kTZ * 1024;
};
template <typename T>
struct BwdSmem {
    static constexpr size_t bytes = 2 * kTZ * 1024 * sizeof(T) + (FN::n + 2 * kTZ * 32) * sizeof(T);
};

__device__ __forceinline__ double shfl_up(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ PF shfl_up(PF v) {
    return {__shfl_up_sync(0xffffffffu, v.a, 1), __shfl_up_sync(0xffffffffu, v.b, 1)};
}

// Per-tile face buffer (device): forward pivots [P][n], forward v [T][n], backward p [T][n].
template <typename T>
__host__ __device__ constexpr size_t face_bytes_per_tile() {
    return (size_t)FN::n * (sizeof(typename PivOps<T>::P) + 2 * sizeof(T));
}

// smem index of voxel (lx, ly, lz) and of each outgoing face entry i
__device__ __forceinline__ int vox(int lx, int ly, int lz) { return (lz * 32 + ly) * 32 + lx; }
__device__ __forceinline__ int out_face_vox(int i, bool fwd) {
    // forward: the +x (lx = 31), +y (ly = 31) and +z (lz = TZ-1) faces; backward: lx = 0, ly = 0, lz = 0
    if (i < FN::y) return vox(fwd ? 31 : 0, i & 31, i >> 5);
    if (i < FN::z) { const int k = i - FN::y; return vox(k & 31, fwd ? 31 : 0, k >> 5); }
    const int k = i - FN::z;
    return vox(k & 31, k >> 5, fwd ? kTZ - 1 : 0);
}

// ------------------------------------------------------------------ streamed faces
//
// A forward tile's sweep does not wait for its predecessor tiles to finish: every voxel of a
// tile's three outgoing faces is written to the face buffer as soon as it is computed.  A
// successor's step s needs, from its -x and -y neighbours, face values those tiles produce
// at their step s + 31, and from its -z neighbour values produced at step s + kTZ - 1.  So a
// successor runs about 32 steps behind its x / y predecessors and kTZ behind its z
// predecessor instead of a whole tile (70 steps) behind; the chain through the grid shrinks
// from (tile levels) x 70 steps towards the nx + ny + nz hyperplanes of the global wavefront,
// plus one hand-off latency per tile hop.
//
// The face entries are their own ready signal.  Between launches every forward face entry
// holds an all-ones bit pattern -- a NaN that no FP32 / FP64 operation produces (arithmetic
// returns the canonical NaN) and that a producer never writes (canon).  A successor polls the
// entries themselves with relaxed loads: an entry that no longer holds the pattern has its
// final value for this launch (each entry is written once, element by element, with relaxed
// stores).  This spares the producer a release fence and the consumer a flag round trip
// before the data round trip: the hand-off is one store's propagation plus the poll.  Each
// entry has exactly one reader (the neighbour across that face), which writes the pattern
// back after reading it, so the buffer is ready for the next launch; the host fills it with
// the pattern when the context is created and after a device error.
//
// Extra warps per CTA fetch the faces: chunk by chunk (a few steps each), they poll the
// entries the chunk needs (bounded, with a short sleep), copies them into shared memory and
// signals the compute warps through a shared-memory counter.  The compute warps synchronise
// among themselves with a named barrier and never poll global memory.

__device__ __forceinline__ void bar_compute() { asm volatile("bar.sync 1, %0;" ::"n"(kCompute) : "memory"); }

// the unset pattern of a face entry, and values kept clear of it
__device__ __forceinline__ bool unset(float x) { return __float_as_uint(x) == 0xffffffffu; }
__device__ __forceinline__ bool unset(double x) { return __double_as_longlong(x) == -1LL; }
__device__ __forceinline__ bool unset(PF x) { return unset(x.a) || unset(x.b); }
__device__ __forceinline__ float canon(float x) { return unset(x) ? __uint_as_float(0x7fffffffu) : x; }
__device__ __forceinline__ double canon(double x) {
    return unset(x) ? __longlong_as_double(0x7fffffffffffffffLL) : x;
}
__device__ __forceinline__ PF canon(PF x) { return {canon(x.a), canon(x.b)}; }

// relaxed (gpu scope) loads and stores of face entries
__device__ __forceinline__ float ld_rlx(const float* p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_rlx(const double* p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ PF ld_rlx(const PF* p) {
    PF v;
    asm volatile("ld.relaxed.gpu.global.v2.f32 {%0, %1}, [%2];" : "=f"(v.a), "=f"(v.b) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_unset(float* p) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(-1) : "memory");
}
__device__ __forceinline__ void st_unset(double* p) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(-1LL) : "memory");
}
__device__ __forceinline__ void st_unset(PF* p) {
    asm volatile("st.relaxed.gpu.global.v2.b32 [%0], {%1, %1};" ::"l"(p), "r"(-1) : "memory");
}

// Offset of diagonal t = lx + ly (0 <= t <= 62) in the diagonal-major z face: diagonal t holds
// min(t + 1, 63 - t) entries, ordered by lx.
__device__ __forceinline__ int zdiag(int t) { return t <= 32 ? t * (t + 1) / 2 : 528 + (t - 32) * (95 - t) / 2; }

// Face entries used at local step s of the forward sweep: x face (ly, lz) with ly + lz = s,
// y face (lx, lz) with lx + lz = s, z face (lx, ly) with lx + ly = s.  Each lane takes at most
// one z-face entry and one x- or y-face entry per step; -1 = none.  z_entry returns the shared
// memory index; lane k of a z diagonal reads global entry FN::z + zdiag(s) + k.
__device__ __forceinline__ int z_entry(int s, int lane) {
    const int lx = max(0, s - 31) + lane;
    return (s >= 0 && lx <= min(31, s)) ? FN::z + (s - lx) * 32 + lx : -1;
}
__device__ __forceinline__ int xy_entry(int s, int lane, int& which) {
    if (lane < kTZ) {  // x face: lanes 0..TZ-1 take lz = lane
        const int ly = s - lane;
        which = 0;
        return (ly >= 0 && ly < 32) ? FN::x + lane * 32 + ly : -1;
    }
    if (lane >= 16 && lane < 16 + kTZ) {  // y face: lanes 16.. take lz = lane - 16
        const int lz = lane - 16, lx = s - lz;
        which = 1;
        return (lx >= 0 && lx < 32) ? FN::y + lz * 32 + lx : -1;
    }
    return -1;
}

// Predicated relaxed stores of outgoing face entries: written by the one lane that produces
// the entry at a step, without a divergent branch in the step body.  No compiler memory
// clobber: the stored value is an operand, nothing in the kernel reads the entry back, and
// volatile asm keeps its order relative to the barriers.  The caller keeps the
// value clear of the unset pattern: an inverse pivot is finite by construction (0 where the
// pivot is not positive or outside the mask), and v passes through canon.
__device__ __forceinline__ void st_if(bool p, double* a, double v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.relaxed.gpu.global.f64 [%1], %2;\n\t}"
                 ::"r"((int)p), "l"(a), "d"(v));
}
__device__ __forceinline__ void st_if(bool p, float* a, float v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.relaxed.gpu.global.f32 [%1], %2;\n\t}"
                 ::"r"((int)p), "l"(a), "f"(v));
}
__device__ __forceinline__ void st_if(bool p, PF* a, PF v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.relaxed.gpu.global.v2.f32 [%1], {%2, %3};\n\t}"
                 ::"r"((int)p), "l"(a), "f"(v.a), "f"(v.b));
}

// After a tile's sweep every entry of its incoming faces has been read (the compute warps
// waited for every chunk), so the compute warps return them to the unset pattern for the
// next launch: the -x (or +x) neighbour's x face, the y neighbour's y face and the z
// neighbour's z face are contiguous ranges of those tiles' face buffers.
template <typename T>
__device__ __forceinline__ void unset_faces(T* fx, T* fy, T* fz) {
    for (int i = threadIdx.x; i < FN::n; i += kCompute) {
        T* f = i < FN::y ? fx : i < FN::z ? fy : fz;
        if (f) st_unset(f + i);
    }
}

// Chunk hand-off from the fetch warp to the compute warps: one mbarrier per chunk with an
// arrival count of 1, completing one phase per tile (the wait parity is the CTA's tile count
// & 1).  The fetch warp's lane 0 arrives (release) once the chunk's faces are in shared
// memory; the compute warps wait with try_wait (acquire), which suspends the warp instead of
// spinning and, unlike an acquire load, does not wait for the warp's own outstanding global
// stores to drain.
__device__ __forceinline__ void mbar_init(unsigned long long* m, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* m) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}"
                 ::"r"(smem_u32(m)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* m, unsigned parity) {
    unsigned ok;
    // suspend hint 1000 ns: each call returns within about a microsecond, so spin_limit calls
    // bound the wait
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, 1000;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(m)), "r"(parity) : "memory");
    return ok != 0;
}
// Compute warps: wait until a chunk of the incoming faces is in shared memory (bounded).
__device__ __forceinline__ void wait_chunk(unsigned long long* m, unsigned parity, long long limit, int* istate) {
    long long n = 0;
    while (!mbar_try_wait(m, parity)) {
        if (++n > limit) {
            set_err(istate, FM_ERR_TIMEOUT);
            break;
        }
    }
}

// MODE 0: pivots from d (factor + forward); MODE 1: stored 1/pi (forward only)
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreadsIC) k_ic_fwd(IcArgs a, PivScal pc) {
    constexpr int mode = MODE;
    using Ops = PivOps<T>;
    using P = typename Ops::P;
    extern __shared__ __align__(16) unsigned char smem[];
    T* sg = (T*)smem;                              // [TZ][32][32]: g, then v
    T* sd = sg + kTZ * 1024;                       // d -> H_hi (-1 outside) -> 1/pi hi; or stored 1/pi
    T* sl = sd + kTZ * 1024;                       // FP32: H_lo -> 1/pi lo
    P* f_ip = (P*)(sd + (Ops::kLo ? 2 : 1) * kTZ * 1024);  // incoming faces: x, y, z
    P* zb_ip = f_ip + FN::n;                       // [2][TZ][32]
    T* f_v = (T*)(zb_ip + 2 * kTZ * 32);
    T* zb_v = f_v + FN::n;
    uint8_t* snb = (uint8_t*)(zb_v + 2 * kTZ * 32);  // [TZ][32][32]
    __shared__ int s_tile;
    constexpr int kCS = kCSF, kNch = (kSteps + kCS - 1) / kCS;
    __shared__ __align__(8) unsigned long long s_mbar[kNch];

    const Geo geo = a.geo;
    const int nx = geo.nx, ny = geo.ny, nz = geo.nz;
    const long long nxy = (long long)nx * ny;
    const int tid = threadIdx.x, lane = tid & 31, wz = tid >> 5;
    const T* g = (const T*)a.g;
    const T* d = (const T*)a.d;
    const T* ipin = (const T*)a.ip_in;
    T* v = (T*)a.v;
    T* ipo = (T*)a.ip_out;
    unsigned char* faceb = (unsigned char*)a.face;
    const T betaT = (T)a.beta;
    auto face_ip = [&](int t) { return (P*)(faceb + (size_t)t * face_bytes_per_tile<T>()); };
    auto face_v = [&](int t) { return (T*)(face_ip(t) + FN::n); };

    if (tid == 0)
        for (int c = 0; c < kNch; ++c) mbar_init(&s_mbar[c], 1);
    unsigned par = 0;  // phase parity of this CTA's current tile
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

        if (wz >= kTZ) {
            // fetch warps: the -x, -y, -z neighbours' outgoing +x, +y, +z faces, alternate chunks each
            const int sx = X > 0 ? tile - 1 : -1, sy = Y > 0 ? tile - a.ntx : -1;
            const int sz = Z > 0 ? tile - a.ntx * a.nty : -1;
            bool ok = true;
            for (int c = wz - kTZ; c < kNch; c += kFetchF) {
                P zp[kCS], qp[kCS];
                T zv[kCS], qv[kCS];
                int zi[kCS], zg[kCS], qi[kCS], qsrc[kCS];
                unsigned want = 0;  // bit q: z entry of step q; bit kCS + q: x / y entry
#pragma unroll
                for (int q = 0; q < kCS; ++q) {
                    const int s = c * kCS + q;
                    int which = 0;
                    zi[q] = s < kSteps ? z_entry(s, lane) : -1;
                    zg[q] = FN::z + zdiag(min(s, 62)) + lane;
                    qi[q] = s < kSteps ? xy_entry(s, lane, which) : -1;
                    qsrc[q] = which ? sy : sx;
                    zp[q] = Ops::zero();
                    qp[q] = Ops::zero();
                    zv[q] = T(0);
                    qv[q] = T(0);
                    if (zi[q] >= 0 && sz >= 0) want |= 1u << q;
                    if (qi[q] >= 0 && qsrc[q] >= 0) want |= 1u << (kCS + q);
                }
                // poll until every wanted entry is set (all of a round's loads are in flight
                // together); a wait that gives up leaves zeros and reports the timeout
                unsigned todo = ok ? want : 0u;
                long long tries = 0;
                while (__any_sync(0xffffffffu, todo != 0u)) {
#pragma unroll
                    for (int q = 0; q < kCS; ++q) {
                        if (todo & (1u << q)) {
                            if (mode == 0) zp[q] = ld_rlx(face_ip(sz) + zg[q]);
                            zv[q] = ld_rlx(face_v(sz) + zg[q]);
                        }
                        if (todo & (1u << (kCS + q))) {
                            if (mode == 0) qp[q] = ld_rlx(face_ip(qsrc[q]) + qi[q]);
                            qv[q] = ld_rlx(face_v(qsrc[q]) + qi[q]);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < kCS; ++q) {
                        if ((todo & (1u << q)) && !unset(zv[q]) && (mode != 0 || !unset(zp[q])))
                            todo &= ~(1u << q);
                        if ((todo & (1u << (kCS + q))) && !unset(qv[q]) && (mode != 0 || !unset(qp[q])))
                            todo &= ~(1u << (kCS + q));
                    }
                    if (++tries > a.spin_limit && __any_sync(0xffffffffu, todo != 0u)) {
                        ok = false;
#pragma unroll
                        for (int q = 0; q < kCS; ++q) {
                            if (todo & (1u << q)) { zp[q] = Ops::zero(); zv[q] = T(0); }
                            if (todo & (1u << (kCS + q))) { qp[q] = Ops::zero(); qv[q] = T(0); }
                        }
                        want &= ~todo;
                        todo = 0u;
                    } else if (todo != 0u) {
                        __nanosleep(20);
                    }
                }
#pragma unroll
                for (int q = 0; q < kCS; ++q) {
                    if (zi[q] >= 0) { f_ip[zi[q]] = zp[q]; f_v[zi[q]] = zv[q]; }
                    if (qi[q] >= 0) { f_ip[qi[q]] = qp[q]; f_v[qi[q]] = qv[q]; }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_mbar[c]);
            }
            if (!ok) set_err(a.istate, FM_ERR_TIMEOUT);  // the host resets the faces with the error
        } else {
            // stage this tile's inputs and form H while the predecessors are still running
            stage_row<T>(sg, g, tid, x0, y0, z0, geo, T(0));
            stage_row<T>(sd, mode == 0 ? d : ipin, tid, x0, y0, z0, geo, T(0));
            if (mode == 0) stage_row_u8(snb, a.nb, tid, x0, y0, z0, geo);
            cp_wait_all();
            if (mode == 0) {
                T* dr = sd + tid * 32;
                T* lr = sl + tid * 32;
                const uint8_t* br = snb + tid * 32;
                // each thread walks its own row; starting at column `lane` keeps the 32 lanes
                // of a warp on 32 different banks (rows are 32 elements apart)
#pragma unroll 4
                for (int k = 0; k < 32; ++k) {
                    const int i = (k + lane) & 31;
                    const uint8_t b = br[i];
                    T hH = T(-1), hL = T(0);
                    if (b & NB_IN) Ops::form_h(dr[i], __popc((unsigned)(b >> 1) & 0x3fu), a.beta, pc, hH, hL);
                    dr[i] = hH;
                    if (Ops::kLo) lr[i] = hL;
                }
            }
            bar_compute();

            // sweep the local hyperplanes s = lx + ly + lz.  The body is branch-free: a lane
            // outside its row (lx not in [0, 32)) computes on the wrapped index lx & 31 -- every
            // lane keeps its own shared-memory bank -- and only active lanes store.
            const int ly = lane, lz = wz, l0 = ly + lz;
            const int row = (lz * 32 + ly) * 32;
            const P* fy_ip = f_ip + FN::y + lz * 32;
            const T* fy_v = f_v + FN::y + lz * 32;
            const P* fz_ip = f_ip + FN::z + ly * 32;
            const T* fz_v = f_v + FN::z + ly * 32;
            const int fxi = FN::x + lz * 32 + ly;
            const int zr = (lz > 0 ? lz - 1 : 0) * 32 + ly, zw = lz * 32 + ly;
            P* oip = face_ip(tile);
            T* ov = face_v(tile);
            P out_ip = Ops::zero();
            T out_v = 0;
            bool bad = false;
            // zdiag(t) - max(0, t - 31) for this warp's current diagonal t = s - lz (0 while t < 0):
            // the z-face entry of lane ly at step s is FN::z + zbase + lx
            int zbase = 0;
            for (int c = 0; c < kNch; ++c) {
              wait_chunk(&s_mbar[c], par, a.spin_limit, a.istate);
#pragma unroll
              for (int q = 0; q < kCS; ++q) {
                const int s = c * kCS + q;
                if (kSteps % kCS != 0 && s >= kSteps) break;
                const P up_ip = shfl_up(out_ip);
                const T up_v = __shfl_up_sync(0xffffffffu, out_v, 1);
                const int lx = s - l0;
                const bool act = (unsigned)lx < 32u;
                const int lw = lx & 31;
                const int i = row + lw;
                const int par = (s & 1) * kTZ * 32;
                const T fyq = fy_v[lw], fzq = fz_v[lw], zbq = zb_v[(kTZ * 32 - par) + zr];
                const T fxq = f_v[fxi];
                const T xv = lx == 0 ? fxq : out_v;
                const T yv = ly == 0 ? fyq : up_v;
                const T zv = lz == 0 ? fzq : zbq;
                const T hH = sd[i];
                const T gi = sg[i];
                const T rhs = gi + betaT * ((xv + yv) + zv);
                P ipj = Ops::zero();
                T vj;
                if constexpr (MODE == 0) {
                    const P fyp = fy_ip[lw], fzp = fz_ip[lw], zbp = zb_ip[(kTZ * 32 - par) + zr];
                    const P fxp = f_ip[fxi];
                    const P xip = lx == 0 ? fxp : out_ip;
                    const P yip = ly == 0 ? fyp : up_ip;
                    const P zip = lz == 0 ? fzp : zbp;
                    const T hL = Ops::kLo ? sl[i] : T(0);
                    const bool inm = hH >= T(0);  // H_jj, or -1 outside the mask
                    bool ok = true;
                    ipj = Ops::inv_pivot(hH, hL, a.beta, pc, xip, yip, zip, ok);
                    if (!inm) ipj = Ops::zero();
                    bad |= act & !(ok || !inm);
                    vj = rhs * (T)Ops::hi(ipj);
                    // every lane stores: an inactive lane writes back what it read
                    sd[i] = act ? (T)Ops::hi(ipj) : hH;
                    if (Ops::kLo) sl[i] = act ? (T)Ops::lo(ipj) : hL;
                    zb_ip[par + zw] = ipj;
                } else {
                    vj = rhs * hH;  // stored 1/pi
                }
                sg[i] = act ? vj : gi;
                // an inactive lane's outputs are read by no active lane at the next step
                out_ip = ipj;
                out_v = vj;
                zb_v[par + zw] = vj;
                // outgoing faces go out as they are produced
                const bool fx_out = act & (lx == 31), fy_out = act & (ly == 31), fz_out = act & (lz == kTZ - 1);
                const int zo = FN::z + zbase + lw;
                if constexpr (MODE == 0) {
                    st_if(fx_out, oip + FN::x + zw, ipj);
                    st_if(fy_out, oip + FN::y + lz * 32 + lw, ipj);
                    st_if(fz_out, oip + zo, ipj);
                }
                const T vc = canon(vj);
                st_if(fx_out, ov + FN::x + zw, vc);
                st_if(fy_out, ov + FN::y + lz * 32 + lw, vc);
                st_if(fz_out, ov + zo, vc);
                {  // next step's diagonal t + 1 = s + 1 - lz: zbase(t + 1) = zbase(t) + max(0, min(t + 1, 62 - t))
                    const int t = s - lz;
                    zbase += max(0, min(t + 1, 62 - t));
                }
                bar_compute();
              }
            }
            if (bad) set_err(a.istate, FM_ERR_NOT_PD);
            {
                const int sx = X > 0 ? tile - 1 : -1, sy = Y > 0 ? tile - a.ntx : -1;
                const int sz = Z > 0 ? tile - a.ntx * a.nty : -1;
                if (mode == 0)
                    unset_faces<P>(sx >= 0 ? face_ip(sx) : nullptr, sy >= 0 ? face_ip(sy) : nullptr,
                                   sz >= 0 ? face_ip(sz) : nullptr);
                unset_faces<T>(sx >= 0 ? face_v(sx) : nullptr, sy >= 0 ? face_v(sy) : nullptr,
                               sz >= 0 ? face_v(sz) : nullptr);
            }
            // write back row-coalesced (warp lz writes its 32 rows, lane = x)
            const int nvalid = min(32, nx - x0);
            const int z = z0 + wz;
            if (z < nz && lane < nvalid) {
                for (int ly2 = 0; ly2 < 32 && y0 + ly2 < ny; ++ly2) {
                    const long long j = (long long)z * nxy + (long long)(y0 + ly2) * nx + x0 + lane;
                    const int i = (wz * 32 + ly2) * 32 + lane;
                    v[j] = sg[i];
                    if (mode == 0 && ipo) ipo[j] = sd[i];
                    if (Ops::kLo && mode == 0 && a.ip_lo_out) a.ip_lo_out[j] = (float)sl[i];
                }
            }
        }
        __syncthreads();
        par ^= 1u;
    }
}

// Deterministic sum of Q doubles over the compute warps (named barrier, the same tree as
// block_sum over 8 warps); result valid in thread 0.
template <int Q>
__device__ __forceinline__ void block_sum_compute(double (&v)[Q], double* sbuf /* >= 32*Q */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = warp_sum(v[q]);
    bar_compute();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < Q; ++q) sbuf[q * 32 + wid] = v[q];
    bar_compute();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const double x = lane < kTZ ? sbuf[q * 32 + lane] : 0.0;
            v[q] = warp_sum(x);
        }
    }
    bar_compute();
}

// Back substitution, streamed like the forward sweep: the reverse sweep of a tile needs, at
// its local hyperplane s, the +x / +y neighbours' low-face values those tiles produce 31
// steps earlier in their own reverse sweeps, and the +z neighbour's 7 (kTZ - 1) steps
// earlier.  Every low-face voxel (lx = 0, ly = 0, lz = 0) goes to the face buffer as it is
// computed (the z face by diagonals, as in the forward sweep), and a fetch warp polls the
// entries each chunk of kCS reverse steps needs, with the same unset-pattern hand-off.
template <typename T>
__global__ void __launch_bounds__(kThreadsB, 2) k_ic_bwd(IcArgs a) {
    using P = typename PivOps<T>::P;
    extern __shared__ __align__(16) unsigned char smem[];
    T* sv = (T*)smem;                 // [TZ][32][32]: v, then p
    T* sip = sv + kTZ * 1024;         // 1/pi
    T* f_p = sip + kTZ * 1024;        // incoming faces (the successors' -x, -y, -z faces)
    T* zb = f_p + FN::n;              // [2][TZ][32]
    __shared__ int s_tile;
    constexpr int kCS = kCSB, kNch = (kSteps + kCS - 1) / kCS;
    __shared__ __align__(8) unsigned long long s_mbar[kNch];
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
    unsigned char* faceb = (unsigned char*)a.face;
    // backward faces live after the forward pivot and v faces of each tile
    auto face_p = [&](int t) {
        return (T*)(faceb + (size_t)t * face_bytes_per_tile<T>() + (size_t)FN::n * (sizeof(P) + sizeof(T)));
    };

    if (tid == 0) {
        s_last = false;
        for (int c = 0; c < kNch; ++c) mbar_init(&s_mbar[c], 1);
    }
    unsigned par = 0;  // phase parity of this CTA's current tile
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

        if (wz >= kTZ) {
            // fetch warps: the +x, +y, +z neighbours' outgoing low faces, alternate chunks each
            const int sx = X + 1 < a.ntx ? tile + 1 : -1, sy = Y + 1 < a.nty ? tile + a.ntx : -1;
            const int sz = Z + 1 < a.ntz ? tile + a.ntx * a.nty : -1;
            bool ok = true;
            for (int c = wz - kTZ; c < kNch; c += kFetchB) {
                T zv[kCS], qv[kCS];
                int zi[kCS], zg[kCS], qi[kCS], qsrc[kCS];
                unsigned want = 0;
#pragma unroll
                for (int q = 0; q < kCS; ++q) {
                    // reverse step c * kCS + q is local hyperplane s; the +z face entry (lx, ly) is
                    // used at s = lx + ly + kTZ - 1, the +x / +y entries at s = 31 + ly + lz / lx + lz
                    const int s = kSteps - 1 - (c * kCS + q);
                    int which = 0;
                    const bool in = s >= 0;
                    zi[q] = in ? z_entry(s - (kTZ - 1), lane) : -1;
                    zg[q] = FN::z + zdiag(min(max(s - (kTZ - 1), 0), 62)) + lane;
                    qi[q] = in ? xy_entry(s - 31, lane, which) : -1;
                    qsrc[q] = which ? sy : sx;
                    zv[q] = T(0);
                    qv[q] = T(0);
                    if (zi[q] >= 0 && sz >= 0) want |= 1u << q;
                    if (qi[q] >= 0 && qsrc[q] >= 0) want |= 1u << (kCS + q);
                }
                unsigned todo = ok ? want : 0u;
                long long tries = 0;
                while (__any_sync(0xffffffffu, todo != 0u)) {
#pragma unroll
                    for (int q = 0; q < kCS; ++q) {
                        if (todo & (1u << q)) zv[q] = ld_rlx(face_p(sz) + zg[q]);
                        if (todo & (1u << (kCS + q))) qv[q] = ld_rlx(face_p(qsrc[q]) + qi[q]);
                    }
#pragma unroll
                    for (int q = 0; q < kCS; ++q) {
                        if ((todo & (1u << q)) && !unset(zv[q])) todo &= ~(1u << q);
                        if ((todo & (1u << (kCS + q))) && !unset(qv[q])) todo &= ~(1u << (kCS + q));
                    }
                    if (++tries > a.spin_limit && __any_sync(0xffffffffu, todo != 0u)) {
                        ok = false;
#pragma unroll
                        for (int q = 0; q < kCS; ++q) {
                            if (todo & (1u << q)) zv[q] = T(0);
                            if (todo & (1u << (kCS + q))) qv[q] = T(0);
                        }
                        want &= ~todo;
                        todo = 0u;
                    } else if (todo != 0u) {
                        __nanosleep(20);
                    }
                }
#pragma unroll
                for (int q = 0; q < kCS; ++q) {
                    if (zi[q] >= 0) f_p[zi[q]] = zv[q];
                    if (qi[q] >= 0) f_p[qi[q]] = qv[q];
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_mbar[c]);
            }
            if (!ok) set_err(a.istate, FM_ERR_TIMEOUT);  // the host resets the faces with the error
        } else {
            stage_row<T>(sv, vin, tid, x0, y0, z0, geo, T(0));
            stage_row<T>(sip, ipb, tid, x0, y0, z0, geo, T(0));
            cp_wait_all();
            bar_compute();

            // sweep in reverse, branch-free as in the forward kernel; the low-face entries a chunk
            // produces go out after the chunk, read back from shared memory by every warp
            const int ly = lane, lz = wz, l0 = ly + lz;
            const int row = (lz * 32 + ly) * 32;
            const int fxi = FN::x + lz * 32 + ly;
            const T* fy = f_p + FN::y + lz * 32;
            const T* fz = f_p + FN::z + ly * 32;
            const int zr = (lz < kTZ - 1 ? lz + 1 : lz) * 32 + ly, zw = lz * 32 + ly;
            T* op = face_p(tile);
            T out = 0;
            for (int c = 0; c < kNch; ++c) {
                wait_chunk(&s_mbar[c], par, a.spin_limit, a.istate);
                const T fxv = f_p[fxi];  // used at s = 31 + l0, in the chunk whose fetch brought it
#pragma unroll
                for (int q = 0; q < kCS; ++q) {
                    const int s = kSteps - 1 - (c * kCS + q);
                    if (kSteps % kCS != 0 && s < 0) break;
                    const T dn = __shfl_down_sync(0xffffffffu, out, 1);
                    const int lx = s - l0;
                    const bool act = (unsigned)lx < 32u;
                    const int lw = lx & 31;
                    const int i = row + lw;
                    const int par = (s & 1) * kTZ * 32;
                    const T fyv = fy[lw], fzv = fz[lw], zbv = zb[(kTZ * 32 - par) + zr];
                    const T px = lx == 31 ? fxv : out;
                    const T py = ly == 31 ? fyv : dn;
                    const T pz = lz == kTZ - 1 ? fzv : zbv;
                    const T vi = sv[i];
                    const T pj = vi + beta * sip[i] * ((px + py) + pz);
                    // every lane stores (an inactive lane writes back what it read); an inactive
                    // lane's outputs are read by no active lane at the next step
                    sv[i] = act ? pj : vi;
                    out = pj;
                    zb[par + zw] = pj;
                    bar_compute();
                }
                // low faces produced at local hyperplanes s0..s1 of this chunk: x face (ly, lz) is
                // this thread's lx = 0 voxel, produced at s = l0; y face (lx, lz) was produced by
                // lane 0 of warp lz, one per step, and lane q stores step s1 - q; z face diagonal
                // s1 - wz (warps 0..kCS-1) holds entries (lx, ly) of the lz = 0 plane
                const int s1 = kSteps - 1 - c * kCS, s0 = max(s1 - kCS + 1, 0);
                const int sy_ = s1 - lane, lxy = sy_ - lz;
                const int sz_ = s1 - wz, lxz = sz_ - ly;
                const T vx = sv[row], vy = sv[lz * 1024 + (lxy & 31)], vz = sv[ly * 32 + (lxz & 31)];
                const int zo = FN::z + zdiag(min(max(sz_, 0), 62)) - max(0, sz_ - 31) + (lxz & 31);
                st_if(l0 >= s0 && l0 <= s1, op + FN::x + zw, canon(vx));
                st_if(lane < kCS && sy_ >= s0 && (unsigned)lxy < 32u, op + FN::y + lz * 32 + (lxy & 31), canon(vy));
                st_if(wz < kCS && sz_ >= s0 && (unsigned)lxz < 32u, op + zo, canon(vz));
            }

            {
                const int sx = X + 1 < a.ntx ? tile + 1 : -1, sy = Y + 1 < a.nty ? tile + a.ntx : -1;
                const int sz = Z + 1 < a.ntz ? tile + a.ntx * a.nty : -1;
                unset_faces<T>(sx >= 0 ? face_p(sx) : nullptr, sy >= 0 ? face_p(sy) : nullptr,
                               sz >= 0 ? face_p(sz) : nullptr);
            }
            // write back, then the dot products (off the wavefront's critical path).  The loads of
            // g and g_prev go out kWb rows at a time, so that a tile pays a few memory round
            // trips here, not one per row (the CTA claims its next tile only after this).  A
            // thread's 32 products are summed in T with Kahan compensation and converted to
            // double once: per-product FP64 additions would queue on GB300's narrow FP64 pipe
            // (about 1/64 of the FP32 rate) behind every other CTA on the SM.
            const int nvalid = min(32, nx - x0);
            const int z = z0 + wz;
            const bool zin = z < nz && lane < nvalid;
            const int nrow = min(32, ny - y0);
            double acc[2] = {0.0, 0.0};
            if (zin) {
                constexpr int kWb = 16;
                T s0 = 0, c0 = 0, s1 = 0, c1 = 0;  // Kahan sums of g p and g_prev p
                for (int r0 = 0; r0 < 32; r0 += kWb) {
                    T pv[kWb], gv[kWb], gpv[kWb];
#pragma unroll
                    for (int k = 0; k < kWb; ++k) {
                        const int ly2 = r0 + k;
                        const bool in = ly2 < nrow;
                        const long long j = (long long)z * nxy + (long long)(y0 + (in ? ly2 : 0)) * nx + x0 + lane;
                        pv[k] = in ? sv[(wz * 32 + ly2) * 32 + lane] : T(0);
                        gv[k] = (gd && in) ? gd[j] : T(0);
                        gpv[k] = (gpd && in) ? gpd[j] : T(0);
                        if (in) p[j] = pv[k];
                    }
#pragma unroll
                    for (int k = 0; k < kWb; ++k) {
                        const T y0k = gv[k] * pv[k] - c0, t0 = s0 + y0k;
                        c0 = (t0 - s0) - y0k;
                        s0 = t0;
                        const T y1k = gpv[k] * pv[k] - c1, t1 = s1 + y1k;
                        c1 = (t1 - s1) - y1k;
                        s1 = t1;
                    }
                }
                acc[0] = (double)s0 - (double)c0;
                acc[1] = (double)s1 - (double)c1;
            }
            if (a.tile_part) {
                block_sum_compute(acc, sbuf);
                if (tid == 0) {
                    a.tile_part[tile] = acc[0];
                    a.tile_part[a.ntiles + tile] = acc[1];
                    __threadfence();
                    const int prev = atomicAdd(a.done, 1);
                    s_last = (prev == a.ntiles - 1);
                    if (s_last) __threadfence();
                }
            }
        }
        __syncthreads();
        if (a.tile_part && s_last) {
            double tot[2];
            sum_partials<2>(a.tile_part, a.ntiles, tot, sbuf);
            if (tid == 0) {
                a.scal[S_GP] = tot[0];
                a.scal[S_GPREVP] = tot[1];
                if (!isfinite(tot[0]) || !isfinite(tot[1])) set_err(a.istate, FM_ERR_NONFINITE);
            }
            __syncthreads();
            if (tid == 0) s_last = false;
        }
        par ^= 1u;
    }
}

template <typename T> int ic_tz() { return kTZ; }
template <typename T> size_t ic_face_bytes_per_tile() { return face_bytes_per_tile<T>(); }

template <typename T>
static cudaError_t prep() {
    static bool done = false;  // attributes are per function, set once per process
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_ic_fwd<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)FwdSmem<T>::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_ic_fwd<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FwdSmem<T>::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_ic_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BwdSmem<T>::bytes);
    if (e == cudaSuccess) done = true;
    return e;
}

template <typename T>
int ic_max_blocks_per_sm(bool bwd) {
    if (prep<T>() != cudaSuccess) return 0;
    int n = 0;
    const cudaError_t e =
        bwd ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ic_bwd<T>, kThreadsB, BwdSmem<T>::bytes)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ic_fwd<T, 0>, kThreadsIC, FwdSmem<T>::bytes);
    return e == cudaSuccess ? n : 0;
}

static PivScal piv_scal(double beta) {
    PivScal c;
    c.bh = (float)beta;
    c.bl = (float)(beta - (double)c.bh);
    const double b2 = beta * beta;
    c.b2h = (float)b2;
    c.b2l = (float)(b2 - (double)c.b2h);
    return c;
}

template <typename T>
cudaError_t launch_ic_fwd(const IcArgs& a, int grid, cudaStream_t s) {
    cudaError_t e = prep<T>();
    if (e != cudaSuccess) return e;
    if (a.d)
        k_ic_fwd<T, 0><<<grid, kThreadsIC, FwdSmem<T>::bytes, s>>>(a, piv_scal(a.beta));
    else
        k_ic_fwd<T, 1><<<grid, kThreadsIC, FwdSmem<T>::bytes, s>>>(a, piv_scal(a.beta));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ic_bwd(const IcArgs& a, int grid, cudaStream_t s) {
    cudaError_t e = prep<T>();
    if (e != cudaSuccess) return e;
    k_ic_bwd<T><<<grid, kThreadsB, BwdSmem<T>::bytes, s>>>(a);
    return cudaGetLastError();
}

// 1/pi = hi + lo as one double (FP32 mode's pivot pair, for inspection)
__global__ void k_inv_pivot64(const float* hi, const float* lo, double* out, long long nv) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nv; j += (long long)gridDim.x * blockDim.x)
        out[j] = (double)hi[j] + (double)lo[j];
}

cudaError_t launch_inv_pivot64(const float* hi, const float* lo, double* out, long long nv, int grid, cudaStream_t s) {
    k_inv_pivot64<<<grid, kThreads, 0, s>>>(hi, lo, out, nv);
    return cudaGetLastError();
}

#define FM_INST(T)                                                            \
    template cudaError_t launch_ic_fwd<T>(const IcArgs&, int, cudaStream_t);  \
    template cudaError_t launch_ic_bwd<T>(const IcArgs&, int, cudaStream_t);  \
    template int ic_tz<T>();                                                  \
    template size_t ic_face_bytes_per_tile<T>();                              \
    template int ic_max_blocks_per_sm<T>(bool);
FM_INST(float)
FM_INST(double)

}  // namespace fm
