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
// Voxels outside the mask are identity rows (p_j = 0) and never couple.
//
// Parallel schedule: voxel (x, y, z) depends on (x-1, y, z), (x, y-1, z), (x, y, z-1), so
// every hyperplane x + y + z = const is independent.  The grid is cut into 32 x 32 x TZ
// tiles; a CTA claims tiles through an atomic ticket in a dependency-respecting order (a
// tile's predecessors always hold smaller tickets, so no co-residency is assumed), waits on
// the predecessors' ready flags (bounded spin), and sweeps the tile's 64 + TZ - 2 local
// hyperplanes: lane = y, warp = z, and each thread walks its x row one step per
// hyperplane, taking the -y value from the neighbouring lane by shuffle, the -z value from
// the warp below through shared memory and the -x value from its own register.  Inputs
// are staged in shared memory and outputs are written back row-coalesced.  Pivots are
// carried in double in every precision mode; their tile faces go through a small FP64
// face buffer.
#include "fm_internal.h"

namespace fm {

constexpr int kTZ = 8;
constexpr int kFace = 32 * kTZ + 32 * kTZ + 32 * 32;  // doubles per tile: +x, +y, +z faces

template <typename T>
struct FwdSmem {
    static constexpr size_t bytes =
        2 * kTZ * 1024 * sizeof(T) + kTZ * 1024 +                   // g->v, d->ip, nb
        (kTZ * 32 * 2 + 1024 + 2 * kTZ * 32) * sizeof(double) +     // ip faces + z exchange
        (kTZ * 32 * 2 + 1024 + 2 * kTZ * 32) * sizeof(T);           // v faces + z exchange
};
template <typename T>
struct BwdSmem {
    static constexpr size_t bytes = 2 * kTZ * 1024 * sizeof(T) + kTZ * 1024 +
                                    (kTZ * 32 * 2 + 1024 + 2 * kTZ * 32) * sizeof(T);
};

template <typename T>
__global__ void __launch_bounds__(32 * kTZ) k_ic_fwd(IcArgs a, int mode) {
    extern __shared__ __align__(16) unsigned char smem[];
    T* sg = (T*)smem;                                   // [kTZ][32][32]: g, then v
    T* sd = sg + kTZ * 1024;                            // d (or stored 1/pi), then 1/pi
    double* fx_ip = (double*)(sd + kTZ * 1024);         // [kTZ][32] (lz, ly)
    double* fy_ip = fx_ip + kTZ * 32;                   // [kTZ][32] (lz, lx)
    double* fz_ip = fy_ip + kTZ * 32;                   // [32][32]  (ly, lx)
    double* zb_ip = fz_ip + 1024;                       // [2][kTZ][32]
    T* fx_v = (T*)(zb_ip + 2 * kTZ * 32);
    T* fy_v = fx_v + kTZ * 32;
    T* fz_v = fy_v + kTZ * 32;
    T* zb_v = fz_v + 1024;
    uint8_t* snb = (uint8_t*)(zb_v + 2 * kTZ * 32);     // [kTZ][32][32]
    __shared__ int s_tile;

    const int nx = a.geo.nx, ny = a.geo.ny, nz = a.geo.nz;
    const long long nxy = (long long)nx * ny;
    const int tid = threadIdx.x, lane = tid & 31, wz = tid >> 5;
    const T* g = (const T*)a.g;
    const T* d = (const T*)a.d;
    const T* ipin = (const T*)a.ip_in;
    T* v = (T*)a.v;
    T* ipo = (T*)a.ip_out;
    const T betaT = (T)a.beta;
    const double beta = a.beta, beta2 = a.beta * a.beta;

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

        // stage this tile's inputs (they do not depend on other tiles)
        for (int i = tid; i < kTZ * 1024; i += blockDim.x) {
            const int x = x0 + (i & 31), y = y0 + ((i >> 5) & 31), z = z0 + (i >> 10);
            T gv = 0, dv = 0;
            uint8_t b = 0;
            if (x < nx && y < ny && z < nz) {
                const long long j = (long long)z * nxy + (long long)y * nx + x;
                gv = g[j];
                dv = mode == 0 ? d[j] : ipin[j];
                b = a.nb[j];
            }
            sg[i] = gv;
            sd[i] = dv;
            snb[i] = b;
        }
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
        // faces produced by the neighbour tiles in this launch (read through L2)
        for (int i = tid; i < kTZ * 32; i += blockDim.x) {
            const int hi = i >> 5, lo = i & 31;  // x-face: (lz, ly); y-face: (lz, lx)
            double ip = 0.0;
            T vv = 0;
            if (X > 0 && y0 + lo < ny && z0 + hi < nz) {
                const long long j = (long long)(z0 + hi) * nxy + (long long)(y0 + lo) * nx + (x0 - 1);
                vv = __ldcg(v + j);
                if (mode == 0) ip = __ldcg(a.face + (size_t)(tile - 1) * kFace + i);
            }
            fx_ip[i] = ip;
            fx_v[i] = vv;
            ip = 0.0;
            vv = 0;
            if (Y > 0 && x0 + lo < nx && z0 + hi < nz) {
                const long long j = (long long)(z0 + hi) * nxy + (long long)(y0 - 1) * nx + (x0 + lo);
                vv = __ldcg(v + j);
                if (mode == 0) ip = __ldcg(a.face + (size_t)(tile - a.ntx) * kFace + 32 * kTZ + i);
            }
            fy_ip[i] = ip;
            fy_v[i] = vv;
        }
        for (int i = tid; i < 1024; i += blockDim.x) {
            const int ly = i >> 5, lx = i & 31;
            double ip = 0.0;
            T vv = 0;
            if (Z > 0 && x0 + lx < nx && y0 + ly < ny) {
                const long long j = (long long)(z0 - 1) * nxy + (long long)(y0 + ly) * nx + (x0 + lx);
                vv = __ldcg(v + j);
                if (mode == 0)
                    ip = __ldcg(a.face + (size_t)(tile - a.ntx * a.nty) * kFace + 64 * kTZ + i);
            }
            fz_ip[i] = ip;
            fz_v[i] = vv;
        }
        __syncthreads();

        // sweep the local hyperplanes s = lx + ly + lz
        const int ly = lane, lz = wz;
        double out_ip = 0.0;
        T out_v = 0;
        bool bad = false;
        for (int s = 0; s < 64 + kTZ - 2; ++s) {
            const double up_ip = __shfl_up_sync(0xffffffffu, out_ip, 1);
            const T up_v = __shfl_up_sync(0xffffffffu, out_v, 1);
            const int lx = s - ly - lz;
            if (lx >= 0 && lx < 32) {
                const int i = (lz * 32 + ly) * 32 + lx;
                const uint8_t b = snb[i];
                double ipj = 0.0;
                T vj = 0;
                if (b & NB_IN) {
                    double sip = 0.0;
                    T sv = 0;
                    if (b & NB_XM) {
                        if (lx == 0) { sip += fx_ip[lz * 32 + ly]; sv += fx_v[lz * 32 + ly]; }
                        else { sip += out_ip; sv += out_v; }
                    }
                    if (b & NB_YM) {
                        if (ly == 0) { sip += fy_ip[lz * 32 + lx]; sv += fy_v[lz * 32 + lx]; }
                        else { sip += up_ip; sv += up_v; }
                    }
                    if (b & NB_ZM) {
                        if (lz == 0) { sip += fz_ip[ly * 32 + lx]; sv += fz_v[ly * 32 + lx]; }
                        else {
                            const int q = ((s - 1) & 1) * kTZ * 32 + (lz - 1) * 32 + ly;
                            sip += zb_ip[q];
                            sv += zb_v[q];
                        }
                    }
                    if (mode == 0) {
                        const int cnt = __popc((unsigned)(b >> 1) & 0x3fu);
                        const double piv = (double)sd[i] + beta * (double)cnt - beta2 * sip;
                        if (piv > 0.0) ipj = 1.0 / piv;
                        else bad = true;
                    } else {
                        ipj = (double)sd[i];
                    }
                    vj = (sg[i] + betaT * sv) * (T)ipj;
                }
                sg[i] = vj;
                sd[i] = (T)ipj;
                out_ip = ipj;
                out_v = vj;
                zb_ip[(s & 1) * kTZ * 32 + lz * 32 + ly] = ipj;
                zb_v[(s & 1) * kTZ * 32 + lz * 32 + ly] = vj;
                if (mode == 0) {
                    double* f = a.face + (size_t)tile * kFace;
                    if (lx == 31) f[lz * 32 + ly] = ipj;
                    if (ly == 31) f[32 * kTZ + lz * 32 + lx] = ipj;
                    if (lz == kTZ - 1) f[64 * kTZ + ly * 32 + lx] = ipj;
                }
            }
            __syncthreads();
        }
        if (bad) set_err(a.istate, FM_ERR_NOT_PD);

        // write back, then publish the tile
        for (int i = tid; i < kTZ * 1024; i += blockDim.x) {
            const int x = x0 + (i & 31), y = y0 + ((i >> 5) & 31), z = z0 + (i >> 10);
            if (x < nx && y < ny && z < nz) {
                const long long j = (long long)z * nxy + (long long)y * nx + x;
                v[j] = sg[i];
                if (mode == 0 && ipo) ipo[j] = sd[i];
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
    T* sip = sv + kTZ * 1024;         // 1/pi
    T* fx = sip + kTZ * 1024;         // [kTZ][32] (lz, ly) p at x0 + 32
    T* fy = fx + kTZ * 32;            // [kTZ][32] (lz, lx) p at y0 + 32
    T* fz = fy + kTZ * 32;            // [32][32] (ly, lx) p at z0 + kTZ
    T* zb = fz + 1024;                // [2][kTZ][32]
    uint8_t* snb = (uint8_t*)(zb + 2 * kTZ * 32);
    __shared__ int s_tile;
    __shared__ bool s_last;
    __shared__ double sbuf[2 * 32];

    const int nx = a.geo.nx, ny = a.geo.ny, nz = a.geo.nz;
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

        for (int i = tid; i < kTZ * 1024; i += blockDim.x) {
            const int x = x0 + (i & 31), y = y0 + ((i >> 5) & 31), z = z0 + (i >> 10);
            T vv = 0, iv = 0;
            uint8_t b = 0;
            if (x < nx && y < ny && z < nz) {
                const long long j = (long long)z * nxy + (long long)y * nx + x;
                vv = vin[j];
                iv = ipb[j];
                b = a.nb[j];
            }
            sv[i] = vv;
            sip[i] = iv;
            snb[i] = b;
        }
        if (tid == 0) {
            bool ok = true;
            if (X + 1 < a.ntx) ok = spin_until(a.flags + tile + 1, 1, a.spin_limit) && ok;
            if (Y + 1 < a.nty) ok = spin_until(a.flags + tile + a.ntx, 1, a.spin_limit) && ok;
            if (Z + 1 < a.ntz) ok = spin_until(a.flags + tile + a.ntx * a.nty, 1, a.spin_limit) && ok;
            if (!ok) set_err(a.istate, FM_ERR_TIMEOUT);
            __threadfence();
        }
        __syncthreads();
        for (int i = tid; i < kTZ * 32; i += blockDim.x) {
            const int hi = i >> 5, lo = i & 31;
            T q = 0;
            if (X + 1 < a.ntx && y0 + lo < ny && z0 + hi < nz)
                q = __ldcg(p + (long long)(z0 + hi) * nxy + (long long)(y0 + lo) * nx + (x0 + 32));
            fx[i] = q;
            q = 0;
            if (Y + 1 < a.nty && x0 + lo < nx && z0 + hi < nz)
                q = __ldcg(p + (long long)(z0 + hi) * nxy + (long long)(y0 + 32) * nx + (x0 + lo));
            fy[i] = q;
        }
        for (int i = tid; i < 1024; i += blockDim.x) {
            const int ly = i >> 5, lx = i & 31;
            T q = 0;
            if (Z + 1 < a.ntz && x0 + lx < nx && y0 + ly < ny)
                q = __ldcg(p + (long long)(z0 + kTZ) * nxy + (long long)(y0 + ly) * nx + (x0 + lx));
            fz[i] = q;
        }
        __syncthreads();

        const int ly = lane, lz = wz;
        T out = 0;
        for (int s = 64 + kTZ - 3; s >= 0; --s) {
            const T dn = __shfl_down_sync(0xffffffffu, out, 1);
            const int lx = s - ly - lz;
            if (lx >= 0 && lx < 32) {
                const int i = (lz * 32 + ly) * 32 + lx;
                const uint8_t b = snb[i];
                T pj = 0;
                if (b & NB_IN) {
                    T sum = 0;
                    if (b & NB_XP) sum += lx == 31 ? fx[lz * 32 + ly] : out;
                    if (b & NB_YP) sum += ly == 31 ? fy[lz * 32 + lx] : dn;
                    if (b & NB_ZP)
                        sum += lz == kTZ - 1 ? fz[ly * 32 + lx]
                                             : zb[((s + 1) & 1) * kTZ * 32 + (lz + 1) * 32 + ly];
                    pj = sv[i] + beta * sip[i] * sum;
                }
                sv[i] = pj;
                out = pj;
                zb[(s & 1) * kTZ * 32 + lz * 32 + ly] = pj;
            }
            __syncthreads();
        }

        double acc[2] = {0.0, 0.0};
        for (int i = tid; i < kTZ * 1024; i += blockDim.x) {
            const int x = x0 + (i & 31), y = y0 + ((i >> 5) & 31), z = z0 + (i >> 10);
            if (x < nx && y < ny && z < nz) {
                const long long j = (long long)z * nxy + (long long)y * nx + x;
                const T pj = sv[i];
                p[j] = pj;
                if (gd) acc[0] += (double)(gd[j] * pj);
                if (gpd) acc[1] += (double)(gpd[j] * pj);
            }
        }
        block_sum<2>(acc, sbuf);
        if (tid == 0) {
            if (a.tile_part) {
                a.tile_part[tile] = acc[0];
                a.tile_part[a.ntiles + tile] = acc[1];
            }
            __threadfence();
            st_release(a.flags + tile, 1);
            const int prev = atomicAdd(a.done, 1);
            s_last = (prev == a.ntiles - 1);
            if (s_last) __threadfence();
        }
        __syncthreads();
        if (s_last && a.tile_part) {
            double tot[2];
            sum_partials<2>(a.tile_part, a.ntiles, tot, sbuf);
            if (tid == 0) {
                a.scal[S_GP] = tot[0];
                a.scal[S_GPREVP] = tot[1];
                if (!isfinite(tot[0]) || !isfinite(tot[1])) set_err(a.istate, FM_ERR_NONFINITE);
            }
        }
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
