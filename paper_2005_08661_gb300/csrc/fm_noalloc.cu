// fm_noalloc.cu -- fm_cost_grad_noalloc: the cost / gradient / curvature evaluation of
// fm_cost_grad without a context and without allocating device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another component is
// capturing a CUDA graph on the same device, real-time pipelines that must not allocate
// after start-up, and plug-ins whose host runtime owns every device buffer and only hands
// them pointers.  This entry point takes the raw inputs and outputs from the caller and
// keeps its only scratch -- the per-block FP64 partial sums of the cost, a finished-block
// counter and the reduced total -- in one file-scope __device__ array of fixed size
// (about 128 KB), which every GPU that loads the library holds until the process exits.
//
// Per voxel it forms the same quantities as the context's precompute (k_setup.cu) and
// the same voxel arithmetic as the gradient pass (k_data.cu), directly from y and s.
#include <mutex>

#include "fm_internal.h"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerThread = 16;
constexpr long long kNaChunk = (long long)kNaThreads * kNaPerThread;  // voxels per block
constexpr int kNaMaxBlocks = 16384;
constexpr long long kNaMaxVoxels = kNaChunk * kNaMaxBlocks;           // 67,108,864 voxels
constexpr int kNaMaxDevices = 64;

struct NaScratch {
    double partial[kNaMaxBlocks];  // one FP64 partial cost per block
    double result;                 // reduced cost of the last call
    unsigned count;                // finished blocks of the current call (cleared per call)
};

static __device__ __align__(256) NaScratch g_na_scratch;

struct NaArgs {
    int nx, ny, nz, nc, L, literal;
    long long nv;
    int P;
    int pm[fm::kMaxPairs], pn[fm::kMaxPairs];
    double dt[fm::kMaxPairs];
    double beta;
    const void* y;
    const void* smap;
    const uint8_t* mask;
    const void* omega;
    void* grad;
    void* curv;
};

__device__ __forceinline__ float na_wrap(float t) {
    const float k = fmaf(t, 0.159154943091895336f, 12582912.0f) - 12582912.0f;
    return fmaf(k, -6.28318530717958648f, t);
}
__device__ __forceinline__ double na_wrap(double t) {
    return t - 6.283185307179586476925286766559 * rint(t * 0.15915494309189533576888376337251);
}
// sin(u)/u on [-pi, pi] by its Taylor series through (-u^2)^8 / 17!
__device__ __forceinline__ float na_sinc(float u) {
    const float v = u * u;
    float p = 2.81145725434552076e-15f;
    p = fmaf(p, v, -7.64716373181981647e-13f);
    p = fmaf(p, v, 1.60590438368216146e-10f);
    p = fmaf(p, v, -2.50521083854417188e-08f);
    p = fmaf(p, v, 2.75573192239858907e-06f);
    p = fmaf(p, v, -1.98412698412698413e-04f);
    p = fmaf(p, v, 8.33333333333333333e-03f);
    p = fmaf(p, v, -1.66666666666666667e-01f);
    return fmaf(p, v, 1.0f);
}
__device__ __forceinline__ double na_sinc(double u) { return u == 0.0 ? 1.0 : sin(u) / u; }
__device__ __forceinline__ void na_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void na_sincos(double x, double* s, double* c) { sincos(x, s, c); }

template <typename T>
__global__ void __launch_bounds__(kNaThreads) k_cost_grad_na(NaArgs a, NaScratch* scr) {
    using T2 = typename fm::V2<T>::t;
    __shared__ double sbuf[32];
    __shared__ bool s_last;
    const T2* y = (const T2*)a.y;
    const T2* sm = (const T2*)a.smap;
    const T* om = (const T*)a.omega;
    T* grad = (T*)a.grad;
    T* curv = (T*)a.curv;
    const long long nv = a.nv, nxy = (long long)a.nx * a.ny;
    const T beta = (T)a.beta;
    auto inm = [&](long long k) { return a.mask ? a.mask[k] != 0 : true; };
    double acc = 0.0;
    const long long base = (long long)blockIdx.x * kNaChunk;
    for (int q = 0; q < kNaPerThread; ++q) {
        const long long j = base + threadIdx.x + (long long)q * kNaThreads;
        if (j >= nv) break;
        if (!inm(j)) {
            if (grad) grad[j] = T(0);
            if (curv) curv[j] = T(0);
            continue;
        }
        const int x = (int)(j % a.nx), yy = (int)((j / a.nx) % a.ny), z = (int)(j / nxy);
        // W_cm = conj(s_c) y_cm / sqrt(L S), its polar form, Z_m = sum_c W_cm (double, then T)
        double S = 0.0;
        for (int c = 0; c < a.nc; ++c) {
            const double sr = sm ? (double)sm[(size_t)c * nv + j].x : 1.0;
            const double si = sm ? (double)sm[(size_t)c * nv + j].y : 0.0;
            S += sr * sr + si * si;
        }
        const double scale = S > 0.0 ? 1.0 / sqrt((double)a.L * S) : 0.0;
        T2 wpol[FM_MAX_ECHO][FM_MAX_COIL];
        double Zr[FM_MAX_ECHO], Zi[FM_MAX_ECHO], sa = 0.0, sz = 0.0;
        for (int m = 0; m < a.L; ++m) {
            double zr = 0.0, zi = 0.0, am = 0.0;
            for (int c = 0; c < a.nc; ++c) {
                const double sr = sm ? (double)sm[(size_t)c * nv + j].x : 1.0;
                const double si = sm ? (double)sm[(size_t)c * nv + j].y : 0.0;
                const T2 yv = y[((size_t)m * a.nc + c) * nv + j];
                const double wr = (sr * (double)yv.x + si * (double)yv.y) * scale;
                const double wi = (sr * (double)yv.y - si * (double)yv.x) * scale;
                const double amp = sqrt(wr * wr + wi * wi);
                wpol[m][c].x = (T)amp;
                wpol[m][c].y = (T)(amp > 0.0 ? atan2(wi, wr) : 0.0);
                zr += wr;
                zi += wi;
                am += amp;
            }
            Zr[m] = zr;
            Zi[m] = zi;
            sa += am;
            sz += sqrt(zr * zr + zi * zi);
        }
        const double Kj = S > 0.0 ? (sa - sz) * (sa + sz) : 0.0;
        const T w = om[j];
        T c_acc = 0, g_acc = 0, d_acc = 0;
        for (int p = 0; p < a.P; ++p) {
            const int m = a.pm[p], n = a.pn[p];
            const double rr = Zr[m] * Zr[n] + Zi[m] * Zi[n];
            const double ri = Zr[m] * Zi[n] - Zi[m] * Zr[n];
            const T Rabs = (T)sqrt(rr * rr + ri * ri);
            const T Rang = (T)((rr == 0.0 && ri == 0.0) ? 0.0 : atan2(ri, rr));
            const T dt = (T)a.dt[p];
            const T th = Rang + w * dt;
            T s, c;
            na_sincos(th * T(0.5), &s, &c);
            c_acc += Rabs * (s * s);
            g_acc += dt * Rabs * (s * c);
            if (a.literal) {
                T inner = 0;
                for (int cc = 0; cc < a.nc; ++cc) {
                    T acc2 = 0;
                    for (int dd = 0; dd < a.nc; ++dd)
                        acc2 += wpol[n][dd].x * na_sinc(na_wrap(wpol[n][dd].y + w * dt - wpol[m][cc].y));
                    inner += wpol[m][cc].x * acc2;
                }
                d_acc += dt * dt * inner;
            } else {
                d_acc += dt * dt * Rabs * na_sinc(na_wrap(th));
            }
        }
        // regulariser stencil between 6-neighbours inside the mask (Eq. 5, Eq. 8)
        T lap = 0, reg = 0;
        if (x > 0 && inm(j - 1)) lap += w - om[j - 1];
        if (yy > 0 && inm(j - a.nx)) lap += w - om[j - a.nx];
        if (z > 0 && inm(j - nxy)) lap += w - om[j - nxy];
        if (x + 1 < a.nx && inm(j + 1)) { const T e = w - om[j + 1]; lap += e; reg += e * e; }
        if (yy + 1 < a.ny && inm(j + a.nx)) { const T e = w - om[j + a.nx]; lap += e; reg += e * e; }
        if (z + 1 < a.nz && inm(j + nxy)) { const T e = w - om[j + nxy]; lap += e; reg += e * e; }
        if (grad) grad[j] = T(4) * g_acc + beta * lap;
        if (curv) curv[j] = T(2) * d_acc;
        acc += Kj + (double)(T(4) * c_acc) + 0.5 * a.beta * (double)reg;
    }
    double v[1] = {acc};
    fm::block_sum<1>(v, sbuf);
    if (threadIdx.x == 0) {
        scr->partial[blockIdx.x] = v[0];
        __threadfence();
        const unsigned prev = atomicAdd(&scr->count, 1u);
        s_last = (prev == gridDim.x - 1);
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (!s_last) return;
    double tot[1];
    fm::sum_partials<1>(scr->partial, gridDim.x, tot, sbuf);
    if (threadIdx.x == 0) {
        scr->result = tot[0];
        scr->count = 0u;
    }
}

std::mutex g_na_mu;
NaScratch* g_na_addr[kNaMaxDevices] = {};

// Device address of the scratch array on `dev` (the current device), looked up once per
// device with cudaGetSymbolAddress: in host code g_na_scratch names only a host-side
// stand-in, never the device memory.
cudaError_t na_scratch(int dev, NaScratch** out) {
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return e;
        g_na_addr[dev] = (NaScratch*)p;
    }
    *out = g_na_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int fm_cost_grad_noalloc(int nx, int ny, int nz, int ncoil, int necho, const fm_opts* opts,
                                    const void* y, const void* smap, const double* te, const uint8_t* mask,
                                    double beta, const void* omega, double* cost, void* grad, void* curv,
                                    int device, void* cuda_stream) {
    if (nx < 1 || ny < 1 || nz < 1 || ncoil < 1 || ncoil > FM_MAX_COIL || necho < 2 || necho > FM_MAX_ECHO)
        return FM_ERR_ARG;
    if (!y || !te || !omega || (!smap && ncoil != 1)) return FM_ERR_ARG;
    if (!(beta >= 0.0) || !(beta < 1e300)) return FM_ERR_ARG;
    for (int l = 0; l < necho; ++l)
        if (!(te[l] == te[l]) || te[l] > 1e300 || te[l] < -1e300) return FM_ERR_ARG;
    fm_opts o;
    fm_default_opts(&o);
    if (opts) o = *opts;
    if ((o.precision != FM_FP32 && o.precision != FM_FP64) ||
        (o.curvature != FM_CURV_LITERAL && o.curvature != FM_CURV_COMBINED))
        return FM_ERR_ARG;
    const long long nv = (long long)nx * ny * nz;
    if (nv > kNaMaxVoxels) return FM_ERR_SIZE;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev || device >= kNaMaxDevices)
        return FM_ERR_CUDA;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return FM_ERR_CUDA;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return FM_ERR_CUDA;
    int rc = FM_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    NaScratch* scr = nullptr;
    NaArgs a{};
    a.nx = nx; a.ny = ny; a.nz = nz; a.nc = ncoil; a.L = necho; a.nv = nv;
    a.literal = (ncoil > 1 && o.curvature == FM_CURV_LITERAL) ? 1 : 0;
    for (int m = 0; m < necho; ++m)
        for (int n = m + 1; n < necho; ++n) {
            a.pm[a.P] = m;
            a.pn[a.P] = n;
            a.dt[a.P] = te[m] - te[n];
            ++a.P;
        }
    a.beta = beta;
    a.y = y; a.smap = smap; a.mask = mask; a.omega = omega; a.grad = grad; a.curv = curv;
    const int blocks = (int)((nv + kNaChunk - 1) / kNaChunk);
    cudaError_t e = na_scratch(device, &scr);
    if (e == cudaSuccess) e = cudaMemsetAsync(&scr->count, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        if (o.precision == FM_FP64) k_cost_grad_na<double><<<blocks, kNaThreads, 0, s>>>(a, scr);
        else k_cost_grad_na<float><<<blocks, kNaThreads, 0, s>>>(a, scr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && cost) {
        e = cudaMemcpyAsync(cost, &scr->result, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        // as fm_cost_grad: a non-finite input inside the mask makes the cost non-finite
        if (e == cudaSuccess && !(*cost - *cost == 0.0)) rc = FM_ERR_NONFINITE;
    }
    if (e != cudaSuccess) rc = FM_ERR_CUDA;
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return rc;
}
