// k_adj.cu -- implicit differentiation of the converged field map.
//
// At a minimiser w^ of Psi (Eq. 5) the gradient vanishes: grad Phi(w^; y) + beta C'C w^ = 0.
// Differentiating that identity gives, for a scalar loss l(w^) with b = dl/dw^,
//   lambda = H_true^{-1} b,   H_true = diag(h) + beta C'C,
//   h_j    = d^2 Phi_j / dw_j^2 = sum_{c,d,m,n} |r| (t_m - t_n)^2 cos(angle r + w_j (t_m - t_n))
//          = 2 sum_{m<n} (t_m - t_n)^2 |R_mn| cos(theta_mn)       (r is linear in the pair sum R)
//   dl/dbeta = -lambda' C'C w^,    dl/dy = -(d grad Phi / dy)' lambda.
// h is the exact second derivative, not the Huber majoriser d of Eq. 10-11; the IC(0)
// factor of the majoriser's H (Eq. 9, 12) serves only as the CG preconditioner.
//
// The image derivative uses the coil combination Z_m = sum_c conj(s_c) y_cm / sqrt(L S)
// (S = sum_c |s_c|^2), for which grad Phi_j = sum_{m,n} (t_m - t_n) Im(conj(Z_m) Z_n
// e^{i w (t_m - t_n)}).  With Q_n = Z_n e^{-i w t_n}, U = sum_n t_n Q_n and V = sum_n Q_n,
//   d grad Phi_j / d conj(y_cm) = i s_c e^{i w t_m} (U - t_m V) / sqrt(L S),
// and the real-pair gradient (d/dRe + i d/dIm) is twice that.
#include "fm_internal.h"

namespace fm {

__device__ __forceinline__ float cos_(float x) { return cosf(x); }
__device__ __forceinline__ double cos_(double x) { return cos(x); }
__device__ __forceinline__ void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }

template <typename T>
__device__ __forceinline__ T true_curv_at(const AdjArgs& a, long long k /* compact index */, T w) {
    using T2 = typename V2<T>::t;
    const T2* pairs = (const T2*)a.pairs;
    T acc = 0;
    for (int p = 0; p < a.pr.P; ++p) {
        const T dt = (T)a.pr.dt[p];
        const T2 R = pairs[(size_t)p * a.geo.nv + k];
        acc += dt * dt * R.x * cos_(R.y + w * dt);
    }
    return T(2) * acc;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_true_curv(AdjArgs a) {
    const T* w = (const T*)a.w;
    T* h = (T*)a.h;
    const long long nm = a.istate[I_NMASK];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
         k += (long long)gridDim.x * blockDim.x) {
        const long long j = a.vlist[k];
        h[j] = true_curv_at<T>(a, k, w[j]);
    }
}

// h, r = b, ||b||^2; resets the iteration counter and the stop flag.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_init(AdjArgs a) {
    __shared__ double sbuf[32];
    const T* w = (const T*)a.w;
    const T* b = (const T*)a.rhs;
    T* h = (T*)a.h;
    T* r = (T*)a.r;
    const long long nm = a.istate[I_NMASK];
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
         k += (long long)gridDim.x * blockDim.x) {
        const long long j = a.vlist[k];
        h[j] = true_curv_at<T>(a, k, w[j]);
        const T bj = b[j];
        r[j] = bj;
        acc += (double)bj * (double)bj;
    }
    double v[1] = {acc}, out[1];
    if (last_block_reduce<1>(v, a.partials, (unsigned*)(a.istate + I_DONE0), out, sbuf)) {
        if (threadIdx.x == 0) {
            a.scal[S_CG_BB] = out[0];
            a.scal[S_CG_RR] = out[0];
            a.scal[S_CG_RZPREV] = 0.0;
            a.istate[I_CG_IT] = 0;
            a.istate[I_CG_DONE] = (out[0] == 0.0 || a.maxiter <= 0) ? 1 : 0;
            if (!isfinite(out[0])) { set_err(a.istate, FM_ERR_NONFINITE); a.istate[I_CG_DONE] = 1; }
        }
    }
}

// p = z + (r'z / r_prev'z_prev) p_old (recomputed at the six neighbours), q = H_true p, and
// p'q; the last block sets the step alpha = r'z / p'q.  r'z comes from the back
// substitution (scal[S_GP]).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_dir(AdjArgs a) {
    __shared__ double sbuf[32];
    if (a.istate[I_CG_DONE]) return;
    const int nx = a.geo.nx;
    const long long nxy = (long long)nx * a.geo.ny;
    const double rz = a.scal[S_GP];
    const double rzp = a.scal[S_CG_RZPREV];
    const T bc = (T)((a.istate[I_CG_IT] > 0 && rzp != 0.0) ? rz / rzp : 0.0);
    const T* z = (const T*)a.z;
    const T* po = (const T*)a.p_old;
    const T* h = (const T*)a.h;
    T* pn = (T*)a.p_new;
    T* q = (T*)a.q;
    const T beta = (T)a.beta;
    auto pv = [&](long long i) -> T { return z[i] + bc * po[i]; };
    const long long nm = a.istate[I_NMASK];
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
         k += (long long)gridDim.x * blockDim.x) {
        const long long j = a.vlist[k];
        const uint8_t b = a.nb[j];
        const T pj = pv(j);
        T lap = 0;
        if (b & NB_XM) lap += pj - pv(j - 1);
        if (b & NB_XP) lap += pj - pv(j + 1);
        if (b & NB_YM) lap += pj - pv(j - nx);
        if (b & NB_YP) lap += pj - pv(j + nx);
        if (b & NB_ZM) lap += pj - pv(j - nxy);
        if (b & NB_ZP) lap += pj - pv(j + nxy);
        const T qj = h[j] * pj + beta * lap;
        pn[j] = pj;
        q[j] = qj;
        acc += (double)pj * (double)qj;
    }
    double v[1] = {acc}, out[1];
    if (last_block_reduce<1>(v, a.partials, (unsigned*)(a.istate + I_DONE0), out, sbuf)) {
        if (threadIdx.x == 0) {
            a.scal[S_CG_PQ] = out[0];
            a.scal[S_CG_RZPREV] = rz;
            if (rz == 0.0) {
                a.scal[S_CG_ALPHA] = 0.0;
                a.istate[I_CG_DONE] = 1;  // exact solution
            } else if (!(out[0] > 0.0) || !isfinite(out[0]) || !isfinite(rz)) {
                set_err(a.istate, isfinite(out[0]) && isfinite(rz) ? FM_ERR_NOT_PD : FM_ERR_NONFINITE);
                a.scal[S_CG_ALPHA] = 0.0;
                a.istate[I_CG_DONE] = 1;
            } else {
                a.scal[S_CG_ALPHA] = rz / out[0];
            }
        }
    }
}

// x += alpha p, r -= alpha q, ||r||^2; the last block advances the counter and sets the stop
// flag (1: converged, 2: iteration limit).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_upd(AdjArgs a) {
    __shared__ double sbuf[32];
    if (a.istate[I_CG_DONE]) return;
    const T alpha = (T)a.scal[S_CG_ALPHA];
    const T* p = (const T*)a.p_new;
    const T* q = (const T*)a.q;
    T* x = (T*)a.x;
    T* r = (T*)a.r;
    const long long nm = a.istate[I_NMASK];
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
         k += (long long)gridDim.x * blockDim.x) {
        const long long j = a.vlist[k];
        x[j] += alpha * p[j];
        const T rj = r[j] - alpha * q[j];
        r[j] = rj;
        acc += (double)rj * (double)rj;
    }
    double v[1] = {acc}, out[1];
    if (last_block_reduce<1>(v, a.partials, (unsigned*)(a.istate + I_DONE0), out, sbuf)) {
        if (threadIdx.x == 0) {
            a.scal[S_CG_RR] = out[0];
            if (a.identity_pc) a.scal[S_GP] = out[0];  // r'z with z = r
            const int it = a.istate[I_CG_IT] + 1;
            a.istate[I_CG_IT] = it;
            if (!isfinite(out[0])) {
                set_err(a.istate, FM_ERR_NONFINITE);
                a.istate[I_CG_DONE] = 1;
            } else if (out[0] <= a.tol2 * a.scal[S_CG_BB]) {
                a.istate[I_CG_DONE] = 1;
            } else if (it >= a.maxiter) {
                a.istate[I_CG_DONE] = 2;
            }
        }
    }
}

// lambda' C'C w over the mask (scal[S_ADJ_DOT]).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_lap_dot(AdjArgs a) {
    __shared__ double sbuf[32];
    const int nx = a.geo.nx;
    const long long nxy = (long long)nx * a.geo.ny;
    const T* w = (const T*)a.w;
    const T* lam = (const T*)a.lam;
    const long long nm = a.istate[I_NMASK];
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
         k += (long long)gridDim.x * blockDim.x) {
        const long long j = a.vlist[k];
        const uint8_t b = a.nb[j];
        const T wj = w[j];
        T lap = 0;
        if (b & NB_XM) lap += wj - w[j - 1];
        if (b & NB_XP) lap += wj - w[j + 1];
        if (b & NB_YM) lap += wj - w[j - nx];
        if (b & NB_YP) lap += wj - w[j + nx];
        if (b & NB_ZM) lap += wj - w[j - nxy];
        if (b & NB_ZP) lap += wj - w[j + nxy];
        acc += (double)lam[j] * (double)lap;
    }
    double v[1] = {acc}, out[1];
    if (last_block_reduce<1>(v, a.partials, (unsigned*)(a.istate + I_DONE0), out, sbuf)) {
        if (threadIdx.x == 0) {
            a.scal[S_ADJ_DOT] = out[0];
            if (!isfinite(out[0])) set_err(a.istate, FM_ERR_NONFINITE);
        }
    }
}

// dl/dy_cm = -lambda_j 2 i s_c e^{i w t_m} (U - t_m V) / sqrt(L S) on every grid voxel (0
// outside the mask and where S = 0).  Echo times are taken relative to t_1, which leaves
// the result unchanged and keeps the phases small.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dldy(AdjArgs a) {
    using T2 = typename V2<T>::t;
    const long long nv = a.geo.nv;
    const int L = a.L, nc = a.nc;
    const T2* y = (const T2*)a.y;
    const T2* s = (const T2*)a.smap;
    const T* w = (const T*)a.w;
    const T* lam = (const T*)a.lam;
    T2* out = (T2*)a.dldy;
    T tt[FM_MAX_ECHO];
#pragma unroll
    for (int m = 0; m < FM_MAX_ECHO; ++m) tt[m] = (T)(a.te[m] - a.te[0]);
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nv;
         j += (long long)gridDim.x * blockDim.x) {
        T S = 0;
        const bool in = (a.nb[j] & NB_IN) != 0;
        if (in) {
            if (s) {
                for (int c = 0; c < nc; ++c) {
                    const T2 sc = s[(size_t)c * nv + j];
                    S += sc.x * sc.x + sc.y * sc.y;
                }
            } else {
                S = T(nc);
            }
        }
        if (!in || S == T(0)) {
            for (int i = 0; i < L * nc; ++i) out[(size_t)i * nv + j] = T2{T(0), T(0)};
            continue;
        }
        const T wj = w[j];
        const T inv = T(1) / sqrt(T(L) * S);
        // U = sum_m t_m Q_m, V = sum_m Q_m with Q_m = Z_m e^{-i w t_m}
        T Ur = 0, Ui = 0, Vr = 0, Vi = 0;
        T cs[FM_MAX_ECHO], sn[FM_MAX_ECHO];
#pragma unroll
        for (int m = 0; m < FM_MAX_ECHO; ++m) {
            if (m < L) {
                sincos_(wj * tt[m], &sn[m], &cs[m]);
                T zr = 0, zi = 0;
                for (int c = 0; c < nc; ++c) {
                    const T2 yc = y[((size_t)m * nc + c) * nv + j];
                    const T2 sc = s ? s[(size_t)c * nv + j] : T2{T(1), T(0)};
                    zr += sc.x * yc.x + sc.y * yc.y;  // conj(s) y
                    zi += sc.x * yc.y - sc.y * yc.x;
                }
                zr *= inv;
                zi *= inv;
                const T qr = zr * cs[m] + zi * sn[m];  // Z e^{-i w t}
                const T qi = zi * cs[m] - zr * sn[m];
                Vr += qr;
                Vi += qi;
                Ur += tt[m] * qr;
                Ui += tt[m] * qi;
            }
        }
        const T coef = T(-2) * lam[j] * inv;
#pragma unroll
        for (int m = 0; m < FM_MAX_ECHO; ++m) {
            if (m < L) {
                const T dr = Ur - tt[m] * Vr, di = Ui - tt[m] * Vi;
                // A = e^{i w t_m} (U - t_m V); out = coef * i * s_c * A
                const T Ar = dr * cs[m] - di * sn[m];
                const T Ai = dr * sn[m] + di * cs[m];
                for (int c = 0; c < nc; ++c) {
                    const T2 sc = s ? s[(size_t)c * nv + j] : T2{T(1), T(0)};
                    const T br = sc.x * Ar - sc.y * Ai, bi = sc.x * Ai + sc.y * Ar;  // s A
                    out[((size_t)m * nc + c) * nv + j] = T2{-coef * bi, coef * br};  // coef * i * (s A)
                }
            }
        }
    }
}

template <typename T>
cudaError_t launch_true_curv(const AdjArgs& a, int grid, cudaStream_t s) {
    k_true_curv<T><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cg_init(const AdjArgs& a, int grid, cudaStream_t s) {
    k_cg_init<T><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cg_dir(const AdjArgs& a, int grid, cudaStream_t s) {
    k_cg_dir<T><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cg_upd(const AdjArgs& a, int grid, cudaStream_t s) {
    k_cg_upd<T><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_lap_dot(const AdjArgs& a, int grid, cudaStream_t s) {
    k_lap_dot<T><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_dldy(const AdjArgs& a, int grid, cudaStream_t s) {
    k_dldy<T><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

#define FM_ADJ_INST(T)                                                             \
    template cudaError_t launch_true_curv<T>(const AdjArgs&, int, cudaStream_t);   \
    template cudaError_t launch_cg_init<T>(const AdjArgs&, int, cudaStream_t);     \
    template cudaError_t launch_cg_dir<T>(const AdjArgs&, int, cudaStream_t);      \
    template cudaError_t launch_cg_upd<T>(const AdjArgs&, int, cudaStream_t);      \
    template cudaError_t launch_lap_dot<T>(const AdjArgs&, int, cudaStream_t);     \
    template cudaError_t launch_dldy<T>(const AdjArgs&, int, cudaStream_t);
FM_ADJ_INST(float)
FM_ADJ_INST(double)

}  // namespace fm
