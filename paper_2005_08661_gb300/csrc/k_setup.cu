// k_setup.cu -- once-per-acquisition precompute (Algorithm box: "precompute r_cdmnj by
// Eq. 3 and t_m - t_n"), neighbour bits of the support mask, the compact list of mask
// voxels, the Eq. 6 initial map and the omega-independent part of the cost.
//
// With W_cm = conj(s_c) y_cm / sqrt(L S), S = sum_c |s_c|^2 (field-map case, Gamma = 1/L),
// Eq. 3 factors exactly as r_cdmn = conj(W_cm) W_dn.  Hence
//   sum_{c,d} r_cdmn = conj(Z_m) Z_n =: R_mn  with Z_m = sum_c W_cm,
//   sum_{c,d} |r_cdmn| = A_m A_n             with A_m = sum_c |W_cm|,
// and the literal Eq. 2 sum over all ordered (c, d, m, n) equals
//   Phi_j(w) = K_j + 4 sum_{m<n} |R_mn| sin^2((angle R_mn + w (t_m - t_n)) / 2),
//   K_j = (sum_m A_m)^2 - (sum_m |Z_m|)^2  (the m = n terms plus, for each pair, the
//   coil-combination remainder sum_cd |r| - |R|), which does not depend on w.
// Water-fat model (Eq. gamma): r_cdmn = L Gamma_mn conj(W_cm) W_dn with the complex projector
// Gamma, so R_mn = L Gamma_mn conj(Z_m) Z_n, sum_cd |r_cdmn| = L |Gamma_mn| A_m A_n and
//   K_j = sum_{m,n} L |Gamma_mn| (A_m A_n - |Z_m| |Z_n|)
// (the m = n terms of the varying part vanish: Gamma_mm is real and nonnegative).  The PWLS
// weights of the water-fat initialisation are rho_j = sum_{m,n} L |Gamma_mn| A_m A_n.
// Stored per mask voxel, in the compact (ascending voxel) order the data-term kernels
// iterate: (|R_mn|, angle R_mn) for each pair m < n, and (|W_cm|, angle W_cm) for the
// literal curvature sum of Eq. 10, which does not collapse over coils.
//
// Compaction: k_mask_count counts mask voxels per 1024-voxel chunk, k_chunk_scan turns the
// counts into exclusive offsets (single block, fixed order), and k_setup ranks each mask
// voxel inside its chunk with warp ballots, so the compact order is the voxel order.
#include "fm_internal.h"

namespace fm {

constexpr int kSetupThreads = 256;

__device__ __forceinline__ bool in_mask(const uint8_t* mask, long long j) { return mask ? mask[j] != 0 : true; }

__global__ void __launch_bounds__(kSetupThreads) k_mask_count(const uint8_t* mask, long long nv, int* counts) {
    __shared__ int warp_cnt[kSetupThreads / 32];
    const long long base = (long long)blockIdx.x * kChunk;
    int c = 0;
#pragma unroll
    for (int q = 0; q < kChunk / kSetupThreads; ++q) {
        const long long j = base + q * kSetupThreads + threadIdx.x;
        c += (j < nv && in_mask(mask, j)) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) warp_cnt[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kSetupThreads / 32; ++w) t += warp_cnt[w];
        counts[blockIdx.x] = t;
    }
}

// Exclusive scan of counts[0..n) in place (one block of 1024 threads, tiles of 1024);
// the total goes to *total.
__global__ void __launch_bounds__(1024) k_chunk_scan(int* counts, int n, int* total) {
    __shared__ int warp_sum[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        const int x = i < n ? counts[i] : 0;
        int incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int ws = warp_sum[lane];
            int wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            warp_sum[lane] = wi - ws;  // exclusive warp offsets
        }
        __syncthreads();
        const int carry = s_carry;
        if (i < n) counts[i] = carry + warp_sum[wid] + incl - x;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = carry + warp_sum[wid] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = s_carry;
}

// Polar form of a coil-combined echo value w (the literal curvature's per-coil weights) or of
// an echo-pair weight R_mn.
// FP64 mode: IEEE double.  FP32 mode stores float, and the line search forms its phases in
// float (|theta| up to about 16 rad, rounding near 1e-6 rad), so the angle comes from the
// float atan2f of the rounded components (within 3 ulp) instead of a double atan2 -- the
// FP64 pipe issues at about 1/64 of the FP32 rate and the double form dominated this
// kernel.  The amplitude also enters the cost constant K, so it stays double-accurate: a
// float square root refined by one Newton-Raphson step in double, f + (x - f^2) / (2 f).
template <typename T>
__device__ __forceinline__ double polar_amp(double wr, double wi) {
    const double x = wr * wr + wi * wi;
    if (sizeof(T) == 8) return sqrt(x);
    const float f = sqrtf((float)x);
    return f > 0.0f ? (double)f + fma(-(double)f, (double)f, x) * (double)(0.5f / f) : 0.0;
}
template <typename T>
__device__ __forceinline__ T polar_angle(double wr, double wi) {
    if (sizeof(T) == 8) return (T)((wr != 0.0 || wi != 0.0) ? atan2(wi, wr) : 0.0);
    const float fr = (float)wr, fi = (float)wi;
    return (T)((fr != 0.0f || fi != 0.0f) ? atan2f(fi, fr) : 0.0f);
}

// ------------------------------------------------------------------ float-float arithmetic
//
// FP32 field-map setup: the cost constant K_j = (sum_m A_m)^2 - (sum_m |Z_m|)^2 cancels
// heavily when the coil-combined echoes are in phase, so its inputs must be accurate far
// beyond float; GB300's FP64 pipe runs at about 1/64 of the FP32 rate, so they are carried as
// unevaluated float pairs hi + lo (about 48 significant bits) on the FP32 pipe instead:
// Knuth's two-sum, the FMA two-product, and Dekker's double-length add, multiply and square
// root built on them.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF ff_fast(float a, float b) {  // |a| >= |b| (or a == 0)
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ FF ff_prod(float a, float b) {  // exact product
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ FF ff_neg(FF x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ FF ff_add(FF x, FF y) {
    const FF s = ff_two_sum(x.hi, y.hi);
    const FF t = ff_two_sum(x.lo, y.lo);
    const FF u = ff_fast(s.hi, s.lo + t.hi);
    return ff_fast(u.hi, u.lo + t.lo);
}
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
    const FF p = ff_prod(x.hi, y.hi);
    return ff_fast(p.hi, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo)));
}
__device__ __forceinline__ FF ff_sqr(FF x) {
    const FF p = ff_prod(x.hi, x.hi);
    return ff_fast(p.hi, fmaf(2.0f * x.hi, x.lo, p.lo));
}
__device__ __forceinline__ FF ff_sqrt(FF x) {  // x >= 0: one Newton step from sqrtf(hi)
    if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
    const float r = sqrtf(x.hi);
    const FF rr = ff_prod(r, r);
    const float d = ((x.hi - rr.hi) - rr.lo) + x.lo;
    return ff_fast(r, d * (0.5f / r));
}
__device__ __forceinline__ FF ff_recip(FF x) {  // x > 0: one Newton step from 1 / hi
    const float q = 1.0f / x.hi;
    const FF p = ff_prod(q, x.hi);
    const float r = ((1.0f - p.hi) - p.lo) - q * x.lo;
    return ff_fast(q, q * r);
}

template <typename T>
__global__ void __launch_bounds__(kSetupThreads) k_setup(SetupArgs a) {
    using T2 = typename V2<T>::t;
    __shared__ double sbuf[32];
    __shared__ int warp_cnt[kSetupThreads / 32];
    const long long nv = a.geo.nv;
    const int nx = a.geo.nx, ny = a.geo.ny, nz = a.geo.nz, nc = a.nc, L = a.L;
    const long long nxy = (long long)nx * ny;
    const T2* y = (const T2*)a.y;
    const T2* sm = (const T2*)a.smap;
    T2* pairs = (T2*)a.pairs;
    T2* coils = (T2*)a.coils;
    T* w0 = (T*)a.w0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kChunk;
    int running = a.chunk_off[blockIdx.x];
    double kacc = 0.0;
    for (int q = 0; q < kChunk / kSetupThreads; ++q) {
        const long long j = base + q * kSetupThreads + threadIdx.x;
        const bool in = j < nv && in_mask(a.mask, j);
        // rank of this mask voxel in voxel order
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (lane == 0) warp_cnt[wid] = __popc(bal);
        __syncthreads();
        int off = running;
        for (int w = 0; w < wid; ++w) off += warp_cnt[w];
        int tot = 0;
        for (int w = 0; w < kSetupThreads / 32; ++w) tot += warp_cnt[w];
        const int k = off + __popc(bal & ((1u << lane) - 1u));
        __syncthreads();
        running += tot;
        if (j >= nv) continue;
        const int x = (int)(j % nx);
        const int yy = (int)((j / nx) % ny);
        const int z = (int)(j / nxy);
        uint8_t bits = 0;
        if (in) {
            bits = NB_IN;
            if (x > 0 && in_mask(a.mask, j - 1)) bits |= NB_XM;
            if (x + 1 < nx && in_mask(a.mask, j + 1)) bits |= NB_XP;
            if (yy > 0 && in_mask(a.mask, j - nx)) bits |= NB_YM;
            if (yy + 1 < ny && in_mask(a.mask, j + nx)) bits |= NB_YP;
            if (z > 0 && in_mask(a.mask, j - nxy)) bits |= NB_ZM;
            if (z + 1 < nz && in_mask(a.mask, j + nxy)) bits |= NB_ZP;
            if ((x + yy + z) & 1) bits |= NB_ODD;
        }
        a.nb[j] = bits;
        if (!in) {
            w0[j] = T(0);
            continue;
        }
        a.vlist[k] = (int)j;
        if (sizeof(T) == 4 && !a.wf) {
            // FP32 field-map case in float-float (see above): the same quantities as the
            // double path below, W_cm = conj(s_c) y_cm / sqrt(L S) formed from exact products
            // of the float inputs, the amplitudes and K_j carried to about 48 bits; the stored
            // polar forms and the Eq. 6 start are float.  Float-float has float's exponent
            // range, so the coil maps and the images are first scaled by exact powers of two
            // that bring their largest component near 1 (coil sensitivities fall to the
            // subnormal range at the edge of a field of view): W is unchanged by the coil-map
            // scale and scales by 2^-ey with the image scale, undone on the stored amplitudes
            // and on K_j.
            float smax = 0.0f, ymax = 0.0f;
            for (int c = 0; c < nc; ++c) {
                if (sm) smax = fmaxf(smax, fmaxf(fabsf((float)sm[(size_t)c * nv + j].x),
                                                 fabsf((float)sm[(size_t)c * nv + j].y)));
                for (int mm = 0; mm < L; ++mm) {
                    const T2 yv = y[((size_t)mm * nc + c) * nv + j];
                    ymax = fmaxf(ymax, fmaxf(fabsf((float)yv.x), fabsf((float)yv.y)));
                }
            }
            const int es = (sm && smax > 0.0f) ? ilogbf(smax) : 0, ey = ymax > 0.0f ? ilogbf(ymax) : 0;
            FF S = {0.0f, 0.0f};
            for (int c = 0; c < nc; ++c) {
                const float sr = sm ? ldexpf((float)sm[(size_t)c * nv + j].x, -es) : 1.0f;
                const float si = sm ? ldexpf((float)sm[(size_t)c * nv + j].y, -es) : 0.0f;
                S = ff_add(S, ff_add(ff_prod(sr, sr), ff_prod(si, si)));
            }
            const bool sok = S.hi > 0.0f;
            const FF scale = sok ? ff_recip(ff_sqrt(ff_mul(S, FF{(float)L, 0.0f}))) : FF{0.0f, 0.0f};
            FF Zr[FM_MAX_ECHO], Zi[FM_MAX_ECHO];
            FF sa = {0.0f, 0.0f}, sz = {0.0f, 0.0f};
            for (int mm = 0; mm < L; ++mm) {
                FF zr = {0.0f, 0.0f}, zi = {0.0f, 0.0f}, am = {0.0f, 0.0f};
                for (int c = 0; c < nc; ++c) {
                    const float sr = sm ? ldexpf((float)sm[(size_t)c * nv + j].x, -es) : 1.0f;
                    const float si = sm ? ldexpf((float)sm[(size_t)c * nv + j].y, -es) : 0.0f;
                    const T2 yv = y[((size_t)mm * nc + c) * nv + j];
                    const float yr = ldexpf((float)yv.x, -ey), yi = ldexpf((float)yv.y, -ey);
                    // conj(s) * y, scaled (2^-ey W)
                    const FF wr = ff_mul(ff_add(ff_prod(sr, yr), ff_prod(si, yi)), scale);
                    const FF wi = ff_mul(ff_add(ff_prod(sr, yi), ff_neg(ff_prod(si, yr))), scale);
                    zr = ff_add(zr, wr);
                    zi = ff_add(zi, wi);
                    const FF amp = ff_sqrt(ff_add(ff_sqr(wr), ff_sqr(wi)));
                    am = ff_add(am, amp);
                    if (coils) {
                        T2 o;
                        o.x = (T)ldexpf(amp.hi, ey);
                        // the angle as a fixed-point fraction of a turn (2^32 = one turn) in
                        // the float slot's bits, the form the FP32 curvature kernels read
                        const float ang = (wr.hi != 0.0f || wi.hi != 0.0f) ? atan2f(wi.hi, wr.hi) : 0.0f;
                        o.y = (T)__int_as_float(__double2int_rn((double)ang * 683565275.57643158));
                        coils[((size_t)mm * nc + c) * nv + k] = o;
                    }
                }
                Zr[mm] = zr;
                Zi[mm] = zi;
                sa = ff_add(sa, am);
                sz = ff_add(sz, ff_sqrt(ff_add(ff_sqr(zr), ff_sqr(zi))));
            }
            for (int p = 0; p < a.pr.P; ++p) {
                const int mm = a.pr.m[p], n = a.pr.n[p];
                // R = conj(Z_m) Z_n
                const float rr = Zr[mm].hi * Zr[n].hi + Zi[mm].hi * Zi[n].hi;
                const float ri = Zr[mm].hi * Zi[n].hi - Zi[mm].hi * Zr[n].hi;
                T2 o;
                o.x = (T)ldexpf(hypotf(rr, ri), 2 * ey);
                o.y = (T)((rr != 0.0f || ri != 0.0f) ? atan2f(ri, rr) : 0.0f);
                pairs[(size_t)p * nv + k] = o;
            }
            if (sok) {
                const FF kj = ff_mul(ff_add(sa, ff_neg(sz)), ff_add(sa, sz));
                kacc += ldexp((double)kj.hi + (double)kj.lo, 2 * ey);
            }
            if (a.rho) ((T*)a.rho)[k] = (T)ldexpf(sa.hi * sa.hi, 2 * ey);
            // Eq. 6: angle(conj(z_1) z_2) / (t_2 - t_1)
            const float er = Zr[0].hi * Zr[1].hi + Zi[0].hi * Zi[1].hi;
            const float ei = Zr[0].hi * Zi[1].hi - Zi[0].hi * Zr[1].hi;
            w0[j] = (T)((sok && (er != 0.0f || ei != 0.0f)) ? atan2f(ei, er) / (float)(a.te1 - a.te0) : 0.0f);
            continue;
        }
        double S = 0.0;
        for (int c = 0; c < nc; ++c) {
            const double sr = sm ? (double)sm[(size_t)c * nv + j].x : 1.0;
            const double si = sm ? (double)sm[(size_t)c * nv + j].y : 0.0;
            S += sr * sr + si * si;
        }
        const double scale = S > 0.0 ? 1.0 / sqrt((double)L * S) : 0.0;
        double Zr[FM_MAX_ECHO], Zi[FM_MAX_ECHO], Am[FM_MAX_ECHO];
        for (int mm = 0; mm < L; ++mm) {
            double zr = 0.0, zi = 0.0, am = 0.0;
            for (int c = 0; c < nc; ++c) {
                const double sr = sm ? (double)sm[(size_t)c * nv + j].x : 1.0;
                const double si = sm ? (double)sm[(size_t)c * nv + j].y : 0.0;
                const T2 yv = y[((size_t)mm * nc + c) * nv + j];
                const double yr = (double)yv.x, yi = (double)yv.y;
                // conj(s) * y, scaled
                const double wr = (sr * yr + si * yi) * scale;
                const double wi = (sr * yi - si * yr) * scale;
                zr += wr;
                zi += wi;
                const double amp = polar_amp<T>(wr, wi);
                am += amp;
                if (coils) {
                    T2 o;
                    o.x = (T)amp;
                    o.y = polar_angle<T>(wr, wi);
                    coils[((size_t)mm * nc + c) * nv + k] = o;
                }
            }
            Zr[mm] = zr;
            Zi[mm] = zi;
            Am[mm] = am;
        }
        for (int p = 0; p < a.pr.P; ++p) {
            const int mm = a.pr.m[p], n = a.pr.n[p];
            // R = conj(Z_m) Z_n (times L Gamma_mn in the water-fat model)
            double rr = Zr[mm] * Zr[n] + Zi[mm] * Zi[n];
            double ri = Zr[mm] * Zi[n] - Zi[mm] * Zr[n];
            if (a.wf) {
                const double gr = a.lgam[2 * (mm * L + n)], gi = a.lgam[2 * (mm * L + n) + 1];
                const double tr = gr * rr - gi * ri;
                ri = gr * ri + gi * rr;
                rr = tr;
            }
            T2 o;
            o.x = (T)polar_amp<T>(rr, ri);
            o.y = polar_angle<T>(rr, ri);
            pairs[(size_t)p * nv + k] = o;
        }
        if (a.wf) {
            double kj = 0.0, rj = 0.0;
            for (int mm = 0; mm < L; ++mm)
                for (int n = 0; n < L; ++n) {
                    const double gr = a.lgam[2 * (mm * L + n)], gi = a.lgam[2 * (mm * L + n) + 1];
                    const double g = sqrt(gr * gr + gi * gi);
                    const double zm = polar_amp<T>(Zr[mm], Zi[mm]), zn = polar_amp<T>(Zr[n], Zi[n]);
                    kj += g * (Am[mm] * Am[n] - zm * zn);
                    rj += g * Am[mm] * Am[n];
                }
            if (S > 0.0) kacc += kj;
            if (a.rho) ((T*)a.rho)[k] = (T)rj;
        } else {
            double sa = 0.0, sz = 0.0;
            for (int mm = 0; mm < L; ++mm) {
                sa += Am[mm];
                sz += polar_amp<T>(Zr[mm], Zi[mm]);
            }
            if (S > 0.0) kacc += (sa - sz) * (sa + sz);
            if (a.rho) ((T*)a.rho)[k] = (T)(sa * sa);
        }
        // Eq. 6: angle(conj(z_1) z_2) / (t_2 - t_1); z_m and Z_m differ by a positive scale
        const double er = Zr[0] * Zr[1] + Zi[0] * Zi[1];
        const double ei = Zr[0] * Zi[1] - Zi[0] * Zr[1];
        const double w = (S > 0.0 && (er != 0.0 || ei != 0.0)) ? atan2(ei, er) / (a.te1 - a.te0) : 0.0;
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
__global__ void __launch_bounds__(kSetupThreads) k_masked_copy(const T* in, T* out, const uint8_t* nb, long long nv) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nv; j += (long long)gridDim.x * blockDim.x)
        out[j] = (nb[j] & NB_IN) ? in[j] : T(0);
}

template <typename T>
cudaError_t launch_setup(const SetupArgs& a, cudaStream_t s) {
    const int nchunks = (int)((a.geo.nv + kChunk - 1) / kChunk);
    k_mask_count<<<nchunks, kSetupThreads, 0, s>>>(a.mask, a.geo.nv, a.chunk_off);
    k_chunk_scan<<<1, 1024, 0, s>>>(a.chunk_off, nchunks, a.istate + I_NMASK);
    k_setup<T><<<nchunks, kSetupThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_masked_copy(const void* in, void* out, const uint8_t* nb, long long nv, int grid, cudaStream_t s) {
    k_masked_copy<T><<<grid, kSetupThreads, 0, s>>>((const T*)in, (T*)out, nb, nv);
    return cudaGetLastError();
}

template cudaError_t launch_setup<float>(const SetupArgs&, cudaStream_t);
template cudaError_t launch_setup<double>(const SetupArgs&, cudaStream_t);
template cudaError_t launch_masked_copy<float>(const void*, void*, const uint8_t*, long long, int, cudaStream_t);
template cudaError_t launch_masked_copy<double>(const void*, void*, const uint8_t*, long long, int, cudaStream_t);

}  // namespace fm
