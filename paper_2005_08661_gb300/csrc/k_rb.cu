// k_rb.cu -- red-black IC(0): the labelled multicolour variant of the IC(0) preconditioner
// (Sec. III-B, Eq. 12), in place of the natural order the paper uses.
//
// Unknowns with x + y + z even (red) come before those with x + y + z odd (black).  The
// 6-neighbour grid is bipartite, so no two reds and no two blacks are coupled, and IC(0) of
// P H P' (H = diag(d) + beta C'C, zero fill-in) has
//   red pivots    pi_r = H_rr = d_r + beta deg_r           (a red has no earlier neighbour)
//   black pivots  pi_b = H_bb - beta^2 sum_{r ~ b} 1 / pi_r  (its earlier neighbours are reds)
// and with L = (Pi + E) Pi^{-1/2} as in the natural order, p = (L L')^{-1} g is
//   forward  v_r = g_r / pi_r,   v_b = (g_b + beta sum_{r ~ b} v_r) / pi_b
//   back     p_b = v_b,          p_r = (g_r + beta sum_{b ~ r} p_b) / pi_r.
// Both halves are single stencil passes with no recurrence: one kernel for the blacks
// (recomputing the reds' v on the fly) and one for the reds, which also forms g'p and
// g_prev'p over every mask voxel.
#include "fm_internal.h"

namespace fm {

template <typename T>
__device__ __forceinline__ T h_diag(const T* d, long long j, uint8_t b, T beta) {
    return d[j] + beta * (T)__popc((unsigned)(b >> 1) & 0x3fu);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_rb_black(DataArgs a) {
    const int nx = a.geo.nx;
    const long long nxy = (long long)nx * a.geo.ny;
    const T* d = (const T*)a.d;
    const T* ipin = (const T*)a.ip_in;
    T* ipout = (T*)a.ip_out;
    const T* g = (const T*)a.g;
    T* p = (T*)a.z_new;
    const T beta = (T)a.beta;
    const long long nm = a.istate[I_NMASK];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
         k += (long long)gridDim.x * blockDim.x) {
        const long long j = a.vlist[k];
        const uint8_t b = a.nb[j];
        if (!(b & NB_ODD)) {  // red: only its stored pivot, when factoring
            if (ipout) ipout[j] = T(1) / h_diag(d, j, b, beta);
            continue;
        }
        T s1 = 0, s2 = 0;
        auto red = [&](long long r) {
            const T ir = ipin ? ipin[r] : T(1) / h_diag(d, r, a.nb[r], beta);
            s1 += ir;
            s2 += g[r] * ir;
        };
        if (b & NB_XM) red(j - 1);
        if (b & NB_XP) red(j + 1);
        if (b & NB_YM) red(j - nx);
        if (b & NB_YP) red(j + nx);
        if (b & NB_ZM) red(j - nxy);
        if (b & NB_ZP) red(j + nxy);
        T ipb;
        if (ipin) {
            ipb = ipin[j];
        } else {
            const T pib = h_diag(d, j, b, beta) - beta * beta * s1;
            if (!(pib > T(0))) set_err(a.istate, FM_ERR_NOT_PD);
            ipb = T(1) / pib;
            if (ipout) ipout[j] = ipb;
        }
        p[j] = (g[j] + beta * s2) * ipb;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_rb_red(DataArgs a) {
    __shared__ double sbuf[2 * 32];
    const int nx = a.geo.nx;
    const long long nxy = (long long)nx * a.geo.ny;
    const T* d = (const T*)a.d;
    const T* ipin = (const T*)a.ip_in;
    const T* g = (const T*)a.g;
    const T* gp = (const T*)a.g_prev;  // nullable
    T* p = (T*)a.z_new;
    const T beta = (T)a.beta;
    const long long nm = a.istate[I_NMASK];
    T t0 = 0, t1 = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
         k += (long long)gridDim.x * blockDim.x) {
        const long long j = a.vlist[k];
        const uint8_t b = a.nb[j];
        T pj;
        if (b & NB_ODD) {
            pj = p[j];  // black, final after k_rb_black
        } else {
            T ir;
            if (ipin) {
                ir = ipin[j];
            } else {
                const T h = h_diag(d, j, b, beta);
                if (!(h > T(0))) set_err(a.istate, FM_ERR_NOT_PD);
                ir = T(1) / h;
            }
            T s = 0;
            if (b & NB_XM) s += p[j - 1];
            if (b & NB_XP) s += p[j + 1];
            if (b & NB_YM) s += p[j - nx];
            if (b & NB_YP) s += p[j + nx];
            if (b & NB_ZM) s += p[j - nxy];
            if (b & NB_ZP) s += p[j + nxy];
            pj = (g[j] + beta * s) * ir;
            p[j] = pj;
        }
        t0 += g[j] * pj;
        if (gp) t1 += gp[j] * pj;
    }
    double v[2] = {(double)t0, (double)t1}, out[2];
    if (last_block_reduce<2>(v, a.partials, (unsigned*)(a.istate + I_DONE0), out, sbuf)) {
        if (threadIdx.x == 0) {
            a.scal[S_GP] = out[0];
            a.scal[S_GPREVP] = out[1];
            if (!isfinite(out[0]) || !isfinite(out[1])) set_err(a.istate, FM_ERR_NONFINITE);
        }
    }
}

template <typename T>
cudaError_t launch_rb_black(const DataArgs& a, int grid, cudaStream_t s) {
    k_rb_black<T><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_rb_red(const DataArgs& a, int grid, cudaStream_t s) {
    k_rb_red<T><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

#define FM_RB_INST(T)                                                            \
    template cudaError_t launch_rb_black<T>(const DataArgs&, int, cudaStream_t); \
    template cudaError_t launch_rb_red<T>(const DataArgs&, int, cudaStream_t);
FM_RB_INST(float)
FM_RB_INST(double)

}  // namespace fm
