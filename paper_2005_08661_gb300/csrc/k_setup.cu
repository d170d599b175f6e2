// k_setup.cu -- once-per-acquisition precompute (Algorithm box: "precompute r_cdmnj by
// Eq. 3 and t_m - t_n"), neighbour bits of the support mask, the Eq. 6 initial map and
// the omega-independent part of the cost.
//
// With W_cm = conj(s_c) y_cm / sqrt(L S), S = sum_c |s_c|^2 (field-map case, Gamma = 1/L),
// Eq. 3 factors exactly as r_cdmn = conj(W_cm) W_dn.  Hence
//   sum_{c,d} r_cdmn = conj(Z_m) Z_n =: R_mn  with Z_m = sum_c W_cm,
//   sum_{c,d} |r_cdmn| = A_m A_n             with A_m = sum_c |W_cm|,
// and the literal Eq. 2 sum over all ordered (c, d, m, n) equals
//   Phi_j(w) = K_j + 4 sum_{m<n} |R_mn| sin^2((angle R_mn + w (t_m - t_n)) / 2),
//   K_j = (sum_m A_m)^2 - (sum_m |Z_m|)^2  (the m = n terms plus, for each pair, the
//   coil-combination remainder sum_cd |r| - |R|), which does not depend on w.
// Stored per voxel: (|R_mn|, angle R_mn) for each pair m < n, and (|W_cm|, angle W_cm)
// for the literal curvature sum of Eq. 10, which does not collapse over coils.
#include "fm_internal.h"

namespace fm {

template <typename T>
__global__ void __launch_bounds__(kThreads) k_setup(SetupArgs a) {
    using T2 = typename V2<T>::t;
    __shared__ double sbuf[32];
    const long long nv = a.geo.nv;
    const int nx = a.geo.nx, ny = a.geo.ny, nz = a.geo.nz, nc = a.nc, L = a.L;
    const T2* y = (const T2*)a.y;
    const T2* sm = (const T2*)a.smap;
    T2* pairs = (T2*)a.pairs;
    T2* coils = (T2*)a.coils;
    T* w0 = (T*)a.w0;
    double kacc = 0.0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nv;
         j += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(j % nx);
        const int yy = (int)((j / nx) % ny);
        const int z = (int)(j / ((long long)nx * ny));
        const bool in = a.mask ? a.mask[j] != 0 : true;
        uint8_t bits = 0;
        if (in) {
            const long long nxy = (long long)nx * ny;
            auto m = [&](long long k) { return a.mask ? a.mask[k] != 0 : true; };
            bits = NB_IN;
            if (x > 0 && m(j - 1)) bits |= NB_XM;
            if (x + 1 < nx && m(j + 1)) bits |= NB_XP;
            if (yy > 0 && m(j - nx)) bits |= NB_YM;
            if (yy + 1 < ny && m(j + nx)) bits |= NB_YP;
            if (z > 0 && m(j - nxy)) bits |= NB_ZM;
            if (z + 1 < nz && m(j + nxy)) bits |= NB_ZP;
        }
        a.nb[j] = bits;
        double S = 0.0;
        for (int c = 0; c < nc; ++c) {
            double sr = sm ? (double)sm[(size_t)c * nv + j].x : 1.0;
            double si = sm ? (double)sm[(size_t)c * nv + j].y : 0.0;
            S += sr * sr + si * si;
        }
        const bool live = in && S > 0.0;
        const double scale = live ? 1.0 / sqrt((double)L * S) : 0.0;
        double Zr[FM_MAX_ECHO], Zi[FM_MAX_ECHO], Am[FM_MAX_ECHO];
        for (int mm = 0; mm < L; ++mm) {
            double zr = 0.0, zi = 0.0, am = 0.0;
            for (int c = 0; c < nc; ++c) {
                double sr = sm ? (double)sm[(size_t)c * nv + j].x : 1.0;
                double si = sm ? (double)sm[(size_t)c * nv + j].y : 0.0;
                T2 yv = y[((size_t)mm * nc + c) * nv + j];
                double yr = (double)yv.x, yi = (double)yv.y;
                // conj(s) * y, scaled
                double wr = (sr * yr + si * yi) * scale;
                double wi = (sr * yi - si * yr) * scale;
                double amp = sqrt(wr * wr + wi * wi);
                zr += wr;
                zi += wi;
                am += amp;
                if (coils) {
                    T2 o;
                    o.x = (T)amp;
                    o.y = (T)(amp > 0.0 ? atan2(wi, wr) : 0.0);
                    coils[((size_t)mm * nc + c) * nv + j] = o;
                }
            }
            Zr[mm] = zr;
            Zi[mm] = zi;
            Am[mm] = am;
        }
        for (int p = 0; p < a.pr.P; ++p) {
            const int mm = a.pr.m[p], n = a.pr.n[p];
            // R = conj(Z_m) Z_n
            double rr = Zr[mm] * Zr[n] + Zi[mm] * Zi[n];
            double ri = Zr[mm] * Zi[n] - Zi[mm] * Zr[n];
            T2 o;
            o.x = (T)sqrt(rr * rr + ri * ri);
            o.y = (T)((rr == 0.0 && ri == 0.0) ? 0.0 : atan2(ri, rr));
            pairs[(size_t)p * nv + j] = o;
        }
        double sa = 0.0, sz = 0.0;
        for (int mm = 0; mm < L; ++mm) {
            sa += Am[mm];
            sz += sqrt(Zr[mm] * Zr[mm] + Zi[mm] * Zi[mm]);
        }
        if (live) kacc += (sa - sz) * (sa + sz);
        // Eq. 6: angle(conj(z_1) z_2) / (t_2 - t_1); z_m and Z_m differ by a positive scale
        double er = Zr[0] * Zr[1] + Zi[0] * Zi[1];
        double ei = Zr[0] * Zi[1] - Zi[0] * Zr[1];
        double w = (live && (er != 0.0 || ei != 0.0)) ? atan2(ei, er) / (a.te1 - a.te0) : 0.0;
        w0[j] = (T)w;
    }
    double v[1] = {kacc}, out[1];
    if (last_block_reduce<1>(v, a.partials, (unsigned*)(a.istate + I_DONE0), out, sbuf)) {
        if (threadIdx.x == 0) {
            a.scal[S_K] = out[0];
            if (!isfinite(out[0])) set_err(a.istate, FM_ERR_NONFINITE);
        }
    }
}

template <typename T>
cudaError_t launch_setup(const SetupArgs& a, int grid, cudaStream_t s) {
    k_setup<T><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_setup<float>(const SetupArgs&, int, cudaStream_t);
template cudaError_t launch_setup<double>(const SetupArgs&, int, cudaStream_t);

}  // namespace fm
