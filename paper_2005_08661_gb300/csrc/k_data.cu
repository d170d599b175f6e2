// k_data.cu -- the per-voxel data term (cost, gradient, Huber curvature), fused with the
// regulariser stencil, the NCG direction update and the monotonic line search.
//
// Per voxel j at field value w (Sec. II-III; see k_setup.cu for the pair factorisation):
//   Phi_j  = K_j + 4 sum_{m<n} |R_mn| sin^2(theta_mn / 2),  theta_mn = angle R_mn + w (t_m - t_n)
//   dPhi_j = 2 sum_{m<n} (t_m - t_n) |R_mn| sin(theta_mn)                         (Eq. 8)
//   d_j    = 2 sum_{m<n} (t_m - t_n)^2 sum_{c,d} |W_cm||W_dn| sinc(wrap(angle W_dn - angle W_cm
//                                                              + w (t_m - t_n)))  (Eq. 10-11)
// (the (n, m, d, c) term of every sum equals its (m, n, c, d) mirror, hence the factor 2),
// or, in the labelled FM_CURV_COMBINED variant and always for one coil,
//   d_j    = 2 sum_{m<n} (t_m - t_n)^2 |R_mn| sinc(wrap(theta_mn)).
// wrap() removes the nearest multiple of 2 pi ("mod pi" of Eq. 11 read as the wrap into
// [-pi, pi], Huber's optimal curvature for 1 - cos).
//
// FP32 mode evaluates the voxel arithmetic in float and sums in double; FP64 mode is double
// throughout.  Global sums are block partials reduced in a fixed order (bitwise
// reproducible).
#include <cooperative_groups.h>

#include "fm_internal.h"

namespace fm {

// ------------------------------------------------------------------ scalar helpers

__device__ __forceinline__ float wrap_angle(float t) {
    // nearest integer of t / (2 pi) by the 1.5 * 2^23 rounding constant (|t| < 2^21 here)
    const float k = fmaf(t, 0.159154943091895336f, 12582912.0f) - 12582912.0f;
    return fmaf(k, -6.28318530717958648f, t);
}
__device__ __forceinline__ double wrap_angle(double t) {
    return t - 6.283185307179586476925286766559 * rint(t * 0.15915494309189533576888376337251);
}

// sin(u)/u on the wrapped interval [-pi, pi] as a degree-5 polynomial in v = u^2: the
// discrete minimax fit derived by csrc/sinc_poly.py (truncation error 6.4e-8, 2.3e-7 overall
// in float Horner form, the level of float rounding of the weights).
__device__ __forceinline__ float sinc_wrapped(float u) {
    const float v = u * u;
    float p = -2.0676877099390367e-08f;
    p = fmaf(p, v, 2.708367901504971e-06f);
    p = fmaf(p, v, -0.00019817284191958606f);
    p = fmaf(p, v, 0.008332781493663788f);
    p = fmaf(p, v, -0.1666661947965622f);
    return fmaf(p, v, 0.9999999403953552f);
}
__device__ __forceinline__ double sinc_wrapped(double u) { return u == 0.0 ? 1.0 : sin(u) / u; }

// ------------------------------------------------------------------ FP32 literal curvature

// In FP32 mode (field-map model) the setup stores each coil weight's angle as a fixed-point
// fraction of a turn in the bits of the float slot: 2^32 is one turn, so a difference of two
// angles wraps into [-1/2, 1/2) turn by the integer subtraction's own wrap-around (Eq. 11's
// "mod pi" of the half angle).  The water-fat model and FP64 mode store radians.
__device__ __forceinline__ float fixed_to_radians(float bits) {
    return (float)__float_as_int(bits) * 1.4629180792671596e-09f;  // 2 pi / 2^32
}
template <typename T>
__device__ __forceinline__ T coil_angle(const DataArgs& a, T y) {
    if constexpr (sizeof(T) == 4) return a.wf ? y : fixed_to_radians(y);
    else return y;
}

// w (t_m - t_n) as a fixed-point angle (mod one turn) from dtt = (t_m - t_n) 2^32 / (2 pi):
// the float product split exactly into hi + lo, each rounded to an integer.
__device__ __forceinline__ unsigned phase_fixed(float w, float dtt) {
    const float hi = w * dtt, lo = fmaf(w, dtt, -hi);
    return (unsigned)(unsigned long long)__float2ll_rn(hi) + (unsigned)__float2int_rn(lo);
}

// sin(2 pi x)/(2 pi x) for x in [-1/2, 1/2] turns as a degree-5 polynomial in x^2: the
// discrete minimax fit derived by csrc/sinc_poly.py (truncation error 6.1e-8, 2.1e-7 in
// float Horner form).
constexpr float kSincT0 = 0.9999999403953552f;
constexpr float kSincT1 = -6.579718589782715f;
constexpr float kSincT2 = 12.987038612365723f;
constexpr float kSincT3 = -12.193624496459961f;
constexpr float kSincT4 = 6.580165386199951f;
constexpr float kSincT5 = -1.9852460622787476f;

// The wrapped angle in turns from the difference t of two fixed-point angles that carry the
// offset 2^31 + 2^8: one funnel shift makes the float 1 + (x + 1/2) in [1, 2) with 23
// fraction bits (the 2^8 rounds the 9 bits the shift drops), and subtracting 1.5 is exact.
__device__ __forceinline__ float turns_of(unsigned t) {
    return __uint_as_float(__funnelshift_r(t, 0x7Fu, 9)) - 1.5f;
}
__device__ __forceinline__ float sinc_turns(float x) {
    const float v = x * x;
    float p = fmaf(kSincT5, v, kSincT4);
    p = fmaf(p, v, kSincT3);
    p = fmaf(p, v, kSincT2);
    p = fmaf(p, v, kSincT1);
    return fmaf(p, v, kSincT0);
}

// The inner coil sum of Eq. 10 for one echo pair (m, n) in FP32, two coils d per
// instruction (the f32x2 forms of add, multiply and fused multiply-add, rounding each
// component as the scalar operation does):
//   sum_c |W_cm| sum_d |W_dn| sinc(wrap(angle W_dn + w (t_m - t_n) - angle W_cm)).
// Per term: the integer difference of the fixed-point angles (offset by half a turn, plus
// half of the 2^9 the shift drops, to round), one funnel shift that makes the float
// 1 + (difference + 1/2) in [1, 2) with 23 fraction bits, an exact subtraction of 1.5 that
// leaves the wrapped angle x in turns, and the degree-5 polynomial of sinc(2 pi x) in x^2
// (csrc/sinc_poly.py).  Even and odd d are summed apart, then added.
template <int NC>
__device__ __forceinline__ float coil_pair_sum_x2(const float2 (&Wm)[NC], const float2 (&Wn)[NC], unsigned ph) {
    static_assert(NC % 2 == 0, "two coils per instruction");
    constexpr int H = NC / 2;
    unsigned an[NC];
    float2 ad[H];
#pragma unroll
    for (int dd = 0; dd < NC; ++dd) an[dd] = (unsigned)__float_as_int(Wn[dd].y) + ph + 0x80000100u;
#pragma unroll
    for (int h = 0; h < H; ++h) ad[h] = make_float2(Wn[2 * h].x, Wn[2 * h + 1].x);
    const float2 c5 = make_float2(kSincT5, kSincT5), c4 = make_float2(kSincT4, kSincT4);
    const float2 c3 = make_float2(kSincT3, kSincT3), c2 = make_float2(kSincT2, kSincT2);
    const float2 c1 = make_float2(kSincT1, kSincT1), c0 = make_float2(kSincT0, kSincT0);
    const float2 mid = make_float2(-1.5f, -1.5f);
    float inner = 0;
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
        const unsigned bm = (unsigned)__float_as_int(Wm[cc].y);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const float2 f = make_float2(__uint_as_float(__funnelshift_r(an[2 * h] - bm, 0x7Fu, 9)),
                                         __uint_as_float(__funnelshift_r(an[2 * h + 1] - bm, 0x7Fu, 9)));
            const float2 x = __fadd2_rn(f, mid);
            const float2 v = __fmul2_rn(x, x);
            float2 p = __ffma2_rn(c5, v, c4);
            p = __ffma2_rn(p, v, c3);
            p = __ffma2_rn(p, v, c2);
            p = __ffma2_rn(p, v, c1);
            p = __ffma2_rn(p, v, c0);
            acc = __ffma2_rn(ad[h], p, acc);
        }
        inner = fmaf(Wm[cc].x, acc.x + acc.y, inner);
    }
    return inner;
}

__device__ __forceinline__ void sin_cos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sin_cos(double x, double* s, double* c) { sincos(x, s, c); }

// ------------------------------------------------------------------ per-voxel data term

// Adds the data-term pieces of voxel j at field value w.  NC > 0: literal curvature over
// NC coils held in registers; NC == 0: literal curvature, runtime coil count; NC == 1:
// coil-combined curvature (exact for one coil).
template <typename T, int NC, bool COST, bool CURV>
__device__ __forceinline__ void eval_voxel(const DataArgs& a, long long j /* compact index */, T w, T& cost,
                                           T& grad, T& curv) {
    using T2 = typename V2<T>::t;
    const long long nv = a.geo.nv;
    const T2* pairs = (const T2*)a.pairs;
    const T2* coils = (const T2*)a.coils;
    T c_acc = 0, g_acc = 0, d_acc = 0;
    for (int p = 0; p < a.pr.P; ++p) {
        const T dt = (T)a.pr.dt[p];
        const T2 R = pairs[(size_t)p * nv + j];
        const T th = R.y + w * dt;
        T s, c;
        sin_cos(th * T(0.5), &s, &c);
        if (COST) c_acc += R.x * (s * s);
        g_acc += dt * R.x * (s * c);
        if (CURV) {
            if (NC == 1) {
                d_acc += dt * dt * R.x * sinc_wrapped(wrap_angle(th));
            } else if (NC > 1) {
                const int m = a.pr.m[p], n = a.pr.n[p];
                T psi[NC > 1 ? NC : 1], ad[NC > 1 ? NC : 1];
#pragma unroll
                for (int dd = 0; dd < NC; ++dd) {
                    const T2 q = coils[((size_t)n * NC + dd) * nv + j];
                    ad[dd] = q.x;
                    psi[dd] = coil_angle(a, q.y) + w * dt;
                }
                T inner = 0;
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const T2 q = coils[((size_t)m * NC + cc) * nv + j];
                    T acc = 0;
#pragma unroll
                    for (int dd = 0; dd < NC; ++dd) acc += ad[dd] * sinc_wrapped(wrap_angle(psi[dd] - coil_angle(a, q.y)));
                    inner += q.x * acc;
                }
                d_acc += dt * dt * inner;
            } else {
                // runtime coil count; also the water-fat model, whose angle r_cdmn carries the
                // phase of Gamma_mn and |r_cdmn| the factor L |Gamma_mn| (0 and 1 otherwise)
                const int m = a.pr.m[p], n = a.pr.n[p], nc = a.nc;
                if constexpr (sizeof(T) == 4) {
                    if (!a.wf) {
                        // field-map model in FP32: fixed-point angles (as in coil_pair_sum_x2)
                        const unsigned ph = phase_fixed(w, a.pr.dtt[p]) + 0x80000100u;
                        float inner = 0;
                        for (int cc = 0; cc < nc; ++cc) {
                            const float2 q = coils[((size_t)m * nc + cc) * nv + j];
                            const unsigned bm = (unsigned)__float_as_int(q.y) - ph;
                            float acc = 0;
                            for (int dd = 0; dd < nc; ++dd) {
                                const float2 r = coils[((size_t)n * nc + dd) * nv + j];
                                acc += r.x * sinc_turns(turns_of((unsigned)__float_as_int(r.y) - bm));
                            }
                            inner += q.x * acc;
                        }
                        d_acc += dt * dt * inner;
                        continue;  // the curvature is the last piece of the pair's work
                    }
                }
                const T gph = (T)a.pr.gph[p];
                T inner = 0;
                for (int cc = 0; cc < nc; ++cc) {
                    const T2 q = coils[((size_t)m * nc + cc) * nv + j];
                    T acc = 0;
                    for (int dd = 0; dd < nc; ++dd) {
                        const T2 r = coils[((size_t)n * nc + dd) * nv + j];
                        acc += r.x * sinc_wrapped(wrap_angle(coil_angle(a, r.y) + w * dt + gph - coil_angle(a, q.y)));
                    }
                    inner += q.x * acc;
                }
                d_acc += dt * dt * (T)a.pr.gmag[p] * inner;
            }
        }
    }
    cost = T(4) * c_acc;
    grad = T(4) * g_acc;
    curv = T(2) * d_acc;
}

// Same as eval_voxel for a compile-time echo count L: the pair loop is unrolled and every
// pair and coil value of the voxel is loaded before the arithmetic starts.
template <typename T, int NC, int L, bool COST, bool CURV>
__device__ __forceinline__ void eval_voxel_fixed(const DataArgs& a, long long j /* compact index */, T w,
                                                 T& cost, T& grad, T& curv) {
    using T2 = typename V2<T>::t;
    constexpr int P = L * (L - 1) / 2;
    constexpr int NCL = (CURV && NC > 1) ? NC : 1;
    const long long nv = a.geo.nv;
    const T2* pairs = (const T2*)a.pairs;
    const T2* coils = (const T2*)a.coils;
    T2 R[P];
#pragma unroll
    for (int p = 0; p < P; ++p) R[p] = pairs[(size_t)p * nv + j];
    T2 W[L][NCL];
    if (CURV && NC > 1) {
#pragma unroll
        for (int m = 0; m < L; ++m)
#pragma unroll
            for (int c = 0; c < NCL; ++c) W[m][c] = coils[((size_t)m * NC + c) * nv + j];
    }
    T c_acc = 0, g_acc = 0, d_acc = 0;
    int p = 0;
#pragma unroll
    for (int m = 0; m < L; ++m) {
#pragma unroll
        for (int n = m + 1; n < L; ++n, ++p) {
            const T dt = (T)a.pr.dt[p];
            const T th = R[p].y + w * dt;
            T s, c;
            sin_cos(th * T(0.5), &s, &c);
            if (COST) c_acc += R[p].x * (s * s);
            g_acc += dt * R[p].x * (s * c);
            if (CURV) {
                if constexpr (NC == 1) {
                    d_acc += dt * dt * R[p].x * sinc_wrapped(wrap_angle(th));
                } else if constexpr (sizeof(T) == 4 && NCL % 2 == 0) {
                    d_acc += dt * dt * coil_pair_sum_x2<NCL>(W[m], W[n], phase_fixed(w, a.pr.dtt[p]));
                } else {
                    T psi[NCL];
#pragma unroll
                    for (int dd = 0; dd < NCL; ++dd) psi[dd] = coil_angle(a, W[n][dd].y) + w * dt;
                    T inner = 0;
#pragma unroll
                    for (int cc = 0; cc < NCL; ++cc) {
                        T acc = 0;
#pragma unroll
                        for (int dd = 0; dd < NCL; ++dd)
                            acc += W[n][dd].x * sinc_wrapped(wrap_angle(psi[dd] - coil_angle(a, W[m][cc].y)));
                        inner += W[m][cc].x * acc;
                    }
                    d_acc += dt * dt * inner;
                }
            }
        }
    }
    cost = T(4) * c_acc;
    grad = T(4) * g_acc;
    curv = T(2) * d_acc;
}

// Dispatch to the unrolled three-echo path when it applies.
template <typename T, int NC, bool COST, bool CURV>
__device__ __forceinline__ void eval_any(const DataArgs& a, long long j, T w, T& cost, T& grad, T& curv) {
    if (NC != 0 && a.L == 3) eval_voxel_fixed<T, (NC == 0 ? 1 : NC), 3, COST, CURV>(a, j, w, cost, grad, curv);
    else eval_voxel<T, NC, COST, CURV>(a, j, w, cost, grad, curv);
}

// ------------------------------------------------------------------ gradient pass

// w_out = w_in + alpha z (the previous iteration's update, Algorithm box), then at w_out:
// g = grad Psi (Eq. 8), d (Eq. 10), and Psi (Eq. 5) reduced to scal[S_COST] / cost_hist.
// Runs over the compact list of mask voxels; entries outside the mask are never written
// (the host zeroes them once).
template <typename T, int NC>
__global__ void __launch_bounds__(kThreads, 2) k_grad(DataArgs a) {
    __shared__ double sbuf[32];
    const int nx = a.geo.nx;
    const long long nxy = (long long)nx * a.geo.ny;
    const T* w_in = (const T*)a.w_in;
    const T* z = (const T*)a.z;
    T* w_out = (T*)a.w_out;
    T* g = (T*)a.g;
    T* d = (T*)a.d;
    const T alpha = z ? (T)a.scal[S_ALPHA] : T(0);
    const T beta = (T)a.beta;
    auto upd = [&](long long k) -> T { return z ? w_in[k] + alpha * z[k] : w_in[k]; };
    const long long nm = a.istate[I_NMASK];
    // the thread's cost and penalty sums in T with Kahan compensation, converted to double
    // once (per-voxel FP64 additions would queue on GB300's narrow FP64 pipe)
    T cs = 0, cc = 0, rs = 0, rc = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
         k += (long long)gridDim.x * blockDim.x) {
        const long long j = a.vlist[k];
        const uint8_t b = a.nb[j];
        const T wj = upd(j);
        w_out[j] = wj;
        T lap = 0, reg = 0;
        if (b & NB_XM) lap += wj - upd(j - 1);
        if (b & NB_YM) lap += wj - upd(j - nx);
        if (b & NB_ZM) lap += wj - upd(j - nxy);
        if (b & NB_XP) { const T e = wj - upd(j + 1); lap += e; reg += e * e; }
        if (b & NB_YP) { const T e = wj - upd(j + nx); lap += e; reg += e * e; }
        if (b & NB_ZP) { const T e = wj - upd(j + nxy); lap += e; reg += e * e; }
        T cst, gr, cu;
        eval_any<T, NC, true, true>(a, k, wj, cst, gr, cu);
        if (g) g[j] = gr + beta * lap;
        if (d) d[j] = cu;
        {
            const T y1 = cst - cc, t1 = cs + y1;
            cc = (t1 - cs) - y1;
            cs = t1;
            const T y2 = reg - rc, t2 = rs + y2;
            rc = (t2 - rs) - y2;
            rs = t2;
        }
    }
    double v[1] = {((double)cs - (double)cc) + 0.5 * a.beta * ((double)rs - (double)rc)}, out[1];
    if (last_block_reduce<1>(v, a.partials, (unsigned*)(a.istate + I_DONE0), out, sbuf)) {
        if (threadIdx.x == 0) {
            const double total = a.scal[S_K] + out[0];
            a.scal[S_COST] = total;
            if (a.cost_hist) a.cost_hist[a.istate[I_ITER]] = total;
            if (!isfinite(total)) set_err(a.istate, FM_ERR_NONFINITE);
        }
    }
}

// ------------------------------------------------------------------ line search

// The search direction and the monotonic line search (Algorithm box, Sec. III-C, Eq. 16) as
// one persistent cooperative kernel.
//
// Direction: mu (Polak-Ribiere with the preconditioned gradients; 0 at the first iteration),
// z = -p + mu z, and the sums the line search needs: ||C z||^2, (C z)'(C w), z'g and
// sum z^2 d (each thread sums its voxels in the voxel type, blocks and the grid in FP64, in a
// fixed order, so every block computes the same totals after one grid barrier).  The first
// step alpha_1 = -z'g / (sum z^2 d + beta ||C z||^2) reuses the gradient pass's g and d.
//
// Steps k = 1 .. nls-1: each re-evaluates the data term at w + alpha_k z, reduces
// sum z_j dPhi_j and sum z_j^2 d_j the same way, and updates alpha without leaving the device.
// Every thread visits the same voxels in both phases (one grid-stride mapping), so it reads
// back only the z values it wrote itself.
//
// The grid is sized for the whole voxel grid, but a small mask does not need all of it: only
// the first nb blocks take part -- one mask voxel per thread at most (fewer threads with
// several voxels each measured slower: each voxel is a chain of dependent gathers) -- and the
// rest leave before the first grid barrier, which then counts the nb participants only.
template <typename T, int NC>
__global__ void __launch_bounds__(kThreads) k_ls(DataArgs a) {
    __shared__ double sbuf[4 * 32];
    __shared__ double s_tot[4];
    const T* w = (const T*)a.w_out;
    const T* z = (const T*)a.z_new;
    const int it = a.istate[I_ITER];
    const long long nm = a.istate[I_NMASK];
    const int nb = (int)max(1LL, min((long long)gridDim.x, (nm + kThreads - 1) / kThreads));
    if ((int)blockIdx.x >= nb) return;
    const int nx = a.geo.nx;
    const long long nxy = (long long)nx * a.geo.ny;
    double mu = 0.0;
    if (it > 0) {
        const double den = a.scal[S_GP_PREV];
        mu = den != 0.0 ? (a.scal[S_GP] - a.scal[S_GPREVP]) / den : 0.0;
    }
    {
        const T muT = (T)mu;
        const T* p = (const T*)a.p;
        const T* zo = (const T*)a.z_old;
        T* zn = (T*)a.z_new;
        const T* g = (const T*)a.g;
        const T* d = (const T*)a.d;
        auto zval = [&](long long k) -> T { return -p[k] + muT * zo[k]; };
        T s_cz2 = 0, s_czw = 0, s_zg = 0, s_zzd = 0;
        // one voxel's direction entry and its terms of the four sums (the +x, +y, +z edges)
        auto dir_voxel = [&](long long j, uint8_t b, T pj, T zoj, T wj, T gj, T dj) {
            const T zj = -pj + muT * zoj;
            zn[j] = zj;
            if (b & NB_XP) { const T e = zj - zval(j + 1), f = wj - w[j + 1]; s_cz2 += e * e; s_czw += e * f; }
            if (b & NB_YP) { const T e = zj - zval(j + nx), f = wj - w[j + nx]; s_cz2 += e * e; s_czw += e * f; }
            if (b & NB_ZP) { const T e = zj - zval(j + nxy), f = wj - w[j + nxy]; s_cz2 += e * e; s_czw += e * f; }
            s_zg += zj * gj;
            s_zzd += zj * zj * dj;
        };
        // four voxels per pass with their own loads issued first (the gathers of a voxel
        // depend on its list entry), then the rest one by one, in the same voxel order
        constexpr int U = 4;
        const long long stride = (long long)nb * blockDim.x;
        long long k0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        for (; k0 + (U - 1) * stride < nm; k0 += U * stride) {
            long long jj[U];
            uint8_t bb[U];
            T pp[U], zz[U], ww[U], gg[U], dd[U];
#pragma unroll
            for (int u = 0; u < U; ++u) jj[u] = a.vlist[k0 + u * stride];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                bb[u] = a.nb[jj[u]];
                pp[u] = p[jj[u]];
                zz[u] = zo[jj[u]];
                ww[u] = w[jj[u]];
                gg[u] = g[jj[u]];
                dd[u] = d[jj[u]];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) dir_voxel(jj[u], bb[u], pp[u], zz[u], ww[u], gg[u], dd[u]);
        }
        for (long long k = k0; k < nm; k += stride) {
            const long long j = a.vlist[k];
            dir_voxel(j, a.nb[j], p[j], zo[j], w[j], g[j], d[j]);
        }
        double v[4] = {(double)s_cz2, (double)s_czw, (double)s_zg, (double)s_zzd};
        block_sum<4>(v, sbuf);
        if (threadIdx.x == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) a.partials[(size_t)q * nb + blockIdx.x] = v[q];
        if (!grid_barrier(a.istate, a.spin_limit, nb)) return;
        double tot[4];
        sum_partials<4>(a.partials, nb, tot, sbuf);
        if (threadIdx.x == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) s_tot[q] = tot[q];
        __syncthreads();
    }
    const double cz2 = s_tot[0], czw = s_tot[1];
    double alpha;
    {
        const double den = s_tot[3] + a.beta * cz2;
        alpha = den != 0.0 ? -s_tot[2] / den : 0.0;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.scal[S_CZ2] = cz2;
            a.scal[S_CZW] = czw;
            a.scal[S_ZG] = s_tot[2];
            a.scal[S_ZZD] = s_tot[3];
            a.scal[S_MU] = mu;
            a.scal[S_GP_PREV] = a.scal[S_GP];  // every block read the old value before the barrier
            if (a.mu_hist) a.mu_hist[it] = mu;
            if (!isfinite(alpha) || !isfinite(mu) || !isfinite(den)) set_err(a.istate, FM_ERR_NONFINITE);
        }
        __syncthreads();  // s_tot is reused by the steps below
    }
    for (int step = 1; step < a.nls; ++step) {
        const T aT = (T)alpha;
        // each thread sums its few voxels in the voxel type, then the block and the grid in FP64
        T t1 = 0, t2 = 0;
        if (NC == 1) {
            // HBM-bound form (one coil, or the combined curvature): four voxels per pass with
            // every load issued before the arithmetic, while all four exist; the rest one by
            // one.  The voxels are visited in the same order as below, and a voxel with z = 0
            // adds exactly 0 whether or not it is evaluated, so the sums are unchanged.
            constexpr int U = 4;
            const long long stride = (long long)nb * blockDim.x;
            long long k0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
            for (; k0 + (U - 1) * stride < nm; k0 += U * stride) {
                long long jj[U];
                T zz[U], ww[U];
#pragma unroll
                for (int u = 0; u < U; ++u) jj[u] = a.vlist[k0 + u * stride];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    zz[u] = z[jj[u]];
                    ww[u] = w[jj[u]];
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    T cst, gr, cu;
                    eval_any<T, NC, false, true>(a, k0 + u * stride, ww[u] + aT * zz[u], cst, gr, cu);
                    t1 += zz[u] * gr;
                    t2 += zz[u] * zz[u] * cu;
                }
            }
            for (long long k = k0; k < nm; k += stride) {
                const long long j = a.vlist[k];
                const T zj = z[j];
                if (zj == T(0)) continue;
                T cst, gr, cu;
                eval_any<T, NC, false, true>(a, k, w[j] + aT * zj, cst, gr, cu);
                t1 += zj * gr;
                t2 += zj * zj * cu;
            }
        } else {
            for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
                 k += (long long)nb * blockDim.x) {
                const long long j = a.vlist[k];
                const T zj = z[j];
                if (zj == T(0)) continue;
                T cst, gr, cu;
                eval_any<T, NC, false, true>(a, k, w[j] + aT * zj, cst, gr, cu);
                t1 += zj * gr;
                t2 += zj * zj * cu;
            }
        }
        double v[2] = {(double)t1, (double)t2};
        block_sum<2>(v, sbuf);
        double* part = a.partials + 4 * (size_t)nb + (size_t)(step & 1) * 2 * nb;
        if (threadIdx.x == 0) {
            part[blockIdx.x] = v[0];
            part[nb + blockIdx.x] = v[1];
        }
        if (!grid_barrier(a.istate, a.spin_limit, nb)) return;
        double tot[2];
        sum_partials<2>(part, nb, tot, sbuf);
        if (threadIdx.x == 0) { s_tot[0] = tot[0]; s_tot[1] = tot[1]; }
        __syncthreads();
        const double fp = s_tot[0] + a.beta * (czw + alpha * cz2);
        const double den = s_tot[1] + a.beta * cz2;
        __syncthreads();
        if (den == 0.0) { alpha = 0.0; break; }
        alpha = alpha - fp / den;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.scal[S_ALPHA] = alpha;
        if (a.alpha_hist) a.alpha_hist[it] = alpha;
        if (!isfinite(alpha)) set_err(a.istate, FM_ERR_NONFINITE);
        a.istate[I_ITER] = it + 1;
    }
}

// ------------------------------------------------------------------ diagonal / no preconditioner

// p = g / H_jj (mode 1, the NCG-MLS-D comparison) or p = g (mode 2), with g'p and g_prev'p.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_pdiag(DataArgs a, int mode) {
    __shared__ double sbuf[2 * 32];
    const T* g = (const T*)a.g;
    const T* gp = (const T*)a.g_prev;
    const T* d = (const T*)a.d;
    T* p = (T*)a.z_new;  // output slot
    double s_gp = 0.0, s_gpp = 0.0;
    const long long nm = a.istate[I_NMASK];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
         k += (long long)gridDim.x * blockDim.x) {
        const long long j = a.vlist[k];
        const uint8_t b = a.nb[j];
        T pj = g[j];
        if (mode == 1) {
            const int cnt = __popc((unsigned)(b >> 1) & 0x3fu);
            const T h = d[j] + (T)a.beta * (T)cnt;
            if (!(h > T(0))) set_err(a.istate, FM_ERR_NOT_PD);
            pj = h > T(0) ? pj / h : T(0);
        }
        p[j] = pj;
        s_gp += (double)(g[j] * pj);
        s_gpp += (double)(gp[j] * pj);
    }
    double v[2] = {s_gp, s_gpp}, out[2];
    if (last_block_reduce<2>(v, a.partials, (unsigned*)(a.istate + I_DONE0), out, sbuf)) {
        if (threadIdx.x == 0) {
            a.scal[S_GP] = out[0];
            a.scal[S_GPREVP] = out[1];
        }
    }
}

// ------------------------------------------------------------------ launchers

template <typename T, int NC>
static cudaError_t grad_nc(const DataArgs& a, int grid, cudaStream_t s) {
    k_grad<T, NC><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grad(const DataArgs& a, int grid, cudaStream_t s) {
    if (!a.literal) return grad_nc<T, 1>(a, grid, s);
    if (a.wf) return grad_nc<T, 0>(a, grid, s);
    switch (a.nc) {
        case 2: return grad_nc<T, 2>(a, grid, s);
        case 4: return grad_nc<T, 4>(a, grid, s);
        case 8: return grad_nc<T, 8>(a, grid, s);
        default: return grad_nc<T, 0>(a, grid, s);
    }
}

template <typename T, int NC>
static cudaError_t ls_nc(const DataArgs& a, int grid, cudaStream_t s) {
    DataArgs copy = a;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void*)k_ls<T, NC>, dim3(grid), dim3(kThreads), args, 0, s);
}

template <typename T>
cudaError_t launch_ls(const DataArgs& a, int grid, cudaStream_t s) {
    if (!a.literal) return ls_nc<T, 1>(a, grid, s);
    if (a.wf) return ls_nc<T, 0>(a, grid, s);
    switch (a.nc) {
        case 2: return ls_nc<T, 2>(a, grid, s);
        case 4: return ls_nc<T, 4>(a, grid, s);
        case 8: return ls_nc<T, 8>(a, grid, s);
        default: return ls_nc<T, 0>(a, grid, s);
    }
}

template <typename T, int NC>
static int ls_occ() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ls<T, NC>, kThreads, 0) != cudaSuccess) return 0;
    return n;
}

template <typename T>
int ls_max_blocks_per_sm(const DataArgs& a) {
    if (!a.literal) return ls_occ<T, 1>();
    if (a.wf) return ls_occ<T, 0>();
    switch (a.nc) {
        case 2: return ls_occ<T, 2>();
        case 4: return ls_occ<T, 4>();
        case 8: return ls_occ<T, 8>();
        default: return ls_occ<T, 0>();
    }
}

template <typename T>
cudaError_t launch_pdiag(const DataArgs& a, int mode, int grid, cudaStream_t s) {
    k_pdiag<T><<<grid, kThreads, 0, s>>>(a, mode);
    return cudaGetLastError();
}

#define FM_INST(T)                                                                  \
    template cudaError_t launch_grad<T>(const DataArgs&, int, cudaStream_t);        \
    template cudaError_t launch_ls<T>(const DataArgs&, int, cudaStream_t);          \
    template cudaError_t launch_pdiag<T>(const DataArgs&, int, int, cudaStream_t);  \
    template int ls_max_blocks_per_sm<T>(const DataArgs&);
FM_INST(float)
FM_INST(double)

}  // namespace fm
