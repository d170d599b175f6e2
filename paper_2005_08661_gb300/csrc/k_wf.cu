// k_wf.cu -- the water-fat pieces around the solver (Sec. II-III):
//   * the voxel-wise initial sweep: Phi_j (Eq. 2) at nsweep equally spaced field values,
//     keeping the first smallest (Sec. III-A, following the paper's initialisation);
//   * the start of the PWLS initialisation (Eq. w0_wf): conjugate gradients on
//     (2 diag(rho) + beta C'C) w = 2 rho w~ from w = w~, with rho_j = sum |r_cdmnj| from the
//     setup; the iterations themselves are the adjoint CG's kernels (k_adj.cu) without a
//     preconditioner;
//   * the water and fat components by the closed form of Eq. wf: with the basis
//     gamma = [1, phi] (Eq. gamma), B = (gamma diag(e^{i w t})) kron s_j has
//     B^H B = S gamma^H gamma and B^H y_j = sum_l conj(gamma_lk) e^{-i w t_l} sum_c conj(s_c) y_cl,
//     so [m_w, m_f] = (gamma^H gamma)^{-1} B^H y_j / S.
#include "fm_internal.h"

namespace fm {

__device__ __forceinline__ void sincos_wf(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_wf(double x, double* s, double* c) { sincos(x, s, c); }

template <typename T>
__global__ void __launch_bounds__(kThreads) k_wf_sweep(AdjArgs a, int nsweep, double wlo, double whi) {
    using T2 = typename V2<T>::t;
    const T2* pairs = (const T2*)a.pairs;
    T* out = (T*)a.x;
    const int P = a.pr.P;
    const long long nm = a.istate[I_NMASK];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
         k += (long long)gridDim.x * blockDim.x) {
        T2 R[kMaxPairs];
#pragma unroll
        for (int p = 0; p < kMaxPairs; ++p)
            if (p < P) R[p] = pairs[(size_t)p * a.geo.nv + k];
        T best_w = 0, best_phi = 0;
        for (int q = 0; q < nsweep; ++q) {
            const T w = (T)(nsweep > 1 ? wlo + (whi - wlo) * (double)q / (double)(nsweep - 1) : wlo);
            T phi = 0;
#pragma unroll
            for (int p = 0; p < kMaxPairs; ++p) {
                if (p < P) {
                    T sn, cs;
                    sincos_wf((R[p].y + w * (T)a.pr.dt[p]) * T(0.5), &sn, &cs);
                    phi += R[p].x * (sn * sn);
                }
            }
            if (q == 0 || phi < best_phi) {
                best_phi = phi;
                best_w = w;
            }
        }
        out[a.vlist[k]] = best_w;
    }
}

// h = 2 rho, x = w~, r = 2 rho w~ - (h x + beta C'C x), ||b||^2 and ||r||^2 (= r'z without a
// preconditioner); resets the counter and the stop flag.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_pwls_init(AdjArgs a) {
    __shared__ double sbuf[2 * 32];
    const int nx = a.geo.nx;
    const long long nxy = (long long)nx * a.geo.ny;
    const T* rho = (const T*)a.rho;
    const T* x0 = (const T*)a.x0;
    T* h = (T*)a.h;
    T* x = (T*)a.x;
    T* r = (T*)a.r;
    const T beta = (T)a.beta;
    const long long nm = a.istate[I_NMASK];
    double bb = 0.0, rr = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
         k += (long long)gridDim.x * blockDim.x) {
        const long long j = a.vlist[k];
        const uint8_t b = a.nb[j];
        const T xj = x0[j];
        T lap = 0;
        if (b & NB_XM) lap += xj - x0[j - 1];
        if (b & NB_XP) lap += xj - x0[j + 1];
        if (b & NB_YM) lap += xj - x0[j - nx];
        if (b & NB_YP) lap += xj - x0[j + nx];
        if (b & NB_ZM) lap += xj - x0[j - nxy];
        if (b & NB_ZP) lap += xj - x0[j + nxy];
        const T hj = T(2) * rho[k];
        const T bj = hj * xj;
        const T rj = bj - (hj * xj + beta * lap);
        h[j] = hj;
        x[j] = xj;
        r[j] = rj;
        bb += (double)bj * (double)bj;
        rr += (double)rj * (double)rj;
    }
    double v[2] = {bb, rr}, out[2];
    if (last_block_reduce<2>(v, a.partials, (unsigned*)(a.istate + I_DONE0), out, sbuf)) {
        if (threadIdx.x == 0) {
            a.scal[S_CG_BB] = out[0];
            a.scal[S_CG_RR] = out[1];
            a.scal[S_GP] = out[1];
            a.scal[S_CG_RZPREV] = 0.0;
            a.istate[I_CG_IT] = 0;
            a.istate[I_CG_DONE] = (out[1] == 0.0 || a.maxiter <= 0) ? 1 : 0;
            if (!isfinite(out[0]) || !isfinite(out[1])) {
                set_err(a.istate, FM_ERR_NONFINITE);
                a.istate[I_CG_DONE] = 1;
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_wf_amp(AdjArgs a) {
    using T2 = typename V2<T>::t;
    const long long nv = a.geo.nv;
    const int L = a.L, nc = a.nc;
    const T2* y = (const T2*)a.y;
    const T2* s = (const T2*)a.smap;
    const T* w = (const T*)a.w;
    T2* water = (T2*)a.water;
    T2* fat = (T2*)a.fat;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nv;
         j += (long long)gridDim.x * blockDim.x) {
        T2 ow = T2{T(0), T(0)}, of = T2{T(0), T(0)};
        if (a.nb[j] & NB_IN) {
            T S = 0;
            if (s) {
                for (int c = 0; c < nc; ++c) {
                    const T2 sc = s[(size_t)c * nv + j];
                    S += sc.x * sc.x + sc.y * sc.y;
                }
            } else {
                S = T(nc);
            }
            if (S > T(0)) {
                const T wj = w[j];
                T p0r = 0, p0i = 0, p1r = 0, p1i = 0;  // B^H y
                for (int l = 0; l < L; ++l) {
                    T zr = 0, zi = 0;  // sum_c conj(s_c) y_cl
                    for (int c = 0; c < nc; ++c) {
                        const T2 yc = y[((size_t)l * nc + c) * nv + j];
                        const T2 sc = s ? s[(size_t)c * nv + j] : T2{T(1), T(0)};
                        zr += sc.x * yc.x + sc.y * yc.y;
                        zi += sc.x * yc.y - sc.y * yc.x;
                    }
                    T sn, cs;
                    sincos_wf(wj * (T)a.te[l], &sn, &cs);
                    const T er = zr * cs + zi * sn, ei = zi * cs - zr * sn;  // e^{-i w t} z
                    p0r += er;
                    p0i += ei;
                    const T fr = (T)a.fat_re[l], fi = (T)a.fat_im[l];  // conj(phi_l) * e
                    p1r += fr * er + fi * ei;
                    p1i += fr * ei - fi * er;
                }
                const T inv = T(1) / S;
                // u = Ginv [p0; p1] / S
                const T g00r = (T)a.ginv[0], g00i = (T)a.ginv[1], g01r = (T)a.ginv[2], g01i = (T)a.ginv[3];
                const T g10r = (T)a.ginv[4], g10i = (T)a.ginv[5], g11r = (T)a.ginv[6], g11i = (T)a.ginv[7];
                ow.x = (g00r * p0r - g00i * p0i + g01r * p1r - g01i * p1i) * inv;
                ow.y = (g00r * p0i + g00i * p0r + g01r * p1i + g01i * p1r) * inv;
                of.x = (g10r * p0r - g10i * p0i + g11r * p1r - g11i * p1i) * inv;
                of.y = (g10r * p0i + g10i * p0r + g11r * p1i + g11i * p1r) * inv;
            }
        }
        water[j] = ow;
        fat[j] = of;
    }
}

template <typename T>
cudaError_t launch_pwls_init(const AdjArgs& a, int grid, cudaStream_t s) {
    k_pwls_init<T><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_wf_sweep(const AdjArgs& a, int nsweep, double wlo, double whi, int grid, cudaStream_t s) {
    k_wf_sweep<T><<<grid, kThreads, 0, s>>>(a, nsweep, wlo, whi);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_wf_amp(const AdjArgs& a, int grid, cudaStream_t s) {
    k_wf_amp<T><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

#define FM_WF_INST(T)                                                                                  \
    template cudaError_t launch_pwls_init<T>(const AdjArgs&, int, cudaStream_t);                       \
    template cudaError_t launch_wf_sweep<T>(const AdjArgs&, int, double, double, int, cudaStream_t);   \
    template cudaError_t launch_wf_amp<T>(const AdjArgs&, int, cudaStream_t);
FM_WF_INST(float)
FM_WF_INST(double)

}  // namespace fm
