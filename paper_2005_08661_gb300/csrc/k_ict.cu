// k_ict.cu -- IC with a drop tolerance (Sec. III-B: the paper's L_t and the preconditioner
// of its NCG-MLS-IC; FM_PC_ICT).
//
// The paper zeroes every factor entry whose magnitude is below tau = droptol * H_max, H_max
// being the largest |H_jk| of the outer iteration's H = diag(d) + beta C'C.  Unlike IC(0)
// this keeps fill-in.  Eliminating an earlier neighbour k of two voxels i > j couples them:
// in natural order the first fill lands at the three "level-1" offsets (x+1, y-1, z),
// (x+1, y, z-1) and (x, y+1, z-1) from a row's voxel.  The kernels here hold the pattern P
// of IC(0)'s offsets a = (-1,0,0), b = (0,-1,0), c = (0,0,-1) plus those fill offsets
// d = (1,-1,0), e = (1,0,-1), f = (0,1,-1); row i of L has L_ii and L_{i,i+o}, o in P.
//
// Row i, in increasing column order c, e, f, b, d, a (each entry needs the row's earlier
// entries and the neighbour row j = i + o):
//   L_{i,j} = (H_ij - sum_{k < j} L_ik L_jk) / L_jj, set to 0 if |L_{i,j}| < tau,
//   L_ii = sqrt(H_ii - sum_o L_{i,i+o}^2),
// where the sums run over the common earlier neighbours inside P -- by offset arithmetic
// a: (b, d), (c, e); b: (c, f); c: none; d: (b, a), (e, f); e: (c, a); f: (c, b), (e, d),
// each pair (p1, p2) meaning L_{i,i+p1} L_{j,j+p2}.  The forward substitution L y = g is
// fused with the factorisation; the back substitution solves L' x = y.
//
// Schedule.  The fill offsets d, e, f link voxels of one x + y + z hyperplane, so the IC(0)
// wavefront does not apply.  With level t = x + 2y + 3z every offset in P points to a strictly
// lower level (t(a) = t(d) = t(f) = -1, t(b) = t(e) = -2, t(c) = -3), so one persistent kernel
// sweeps the levels in order -- thread <-> (y, z) column, voxel x = t - 2y - 3z -- with a
// barrier between levels; the back substitution sweeps them in reverse.  A level's work is
// FP64 arithmetic on the active columns, so the blocks are sized to spread the columns over
// every SM (a volume with few columns runs one-warp blocks), and the barrier is the bounded
// grid barrier of a cooperative launch -- or a block barrier when one block holds every
// column.  The factor stores 1 / L_ii, so every entry costs a multiply, and each row issues
// all of its loads from the earlier rows before the dependency chain starts.
//
// Deeper fill.  When the tolerance keeps entries beyond level 1, the pattern P grows: the host
// holds any set of offsets (up to kIctMaxOffsets), builds the correction pairs of each offset
// by the same offset arithmetic (pairs (p1, p2) with o_p1 - o_p2 = o) and a level function
// t = x + B y + C z under which every held offset points to a lower level, and the
// table-driven kernels k_ictg_fwd / k_ictg_bwd sweep it.
//
// Exactness.  The held factor is the exact drop-tolerance factor as long as no entry outside
// the held pattern survives.  With the factor in hand, k_ict_check forms every would-be entry
// just outside it -- at each offset q = o_p1 - o_p2 (p1, p2 held, q not held, pointing to an
// earlier voxel) -- and flags the offsets where one reaches tau.  If none does, no entry
// outside the pattern ever appears (by induction over the columns); otherwise the first
// column where one does sees exactly this value, since all earlier columns agree.  Holding a
// flagged offset where the exact factor turns out to drop every entry changes nothing (the
// entries are computed and dropped exactly as the definition does), so the host adds every
// flagged offset and factors again until nothing is flagged.  For the base pattern the
// candidates are (-1,1,-1): (c,d); (-1,2,-1): (f,d); (0,2,-1): (f,b); (1,1,-1): (e,b), (f,a);
// (2,-1,0): (d,a); (2,0,-1): (e,a).
//
// A pivot <= 0 is reported (FM_ERR_NOT_PD) by the back sweep, after the check, so that
// FM_ERR_FILL wins when fill outside the held pattern is the cause.
//
// Arithmetic is double in both precision modes (the voxel type only for d, g and p): the
// sweeps are latency-bound, not bound by the FP64 pipe.
#include "fm_internal.h"

namespace fm {

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ------------------------------------------------------------------ tau = droptol * H_max

template <typename T>
__global__ void __launch_bounds__(kThreads) k_ict_tau(DataArgs a, double droptol) {
    __shared__ double sbuf[32];
    __shared__ bool s_last;
    const T* d = (const T*)a.d;
    const double beta = a.beta;
    const long long nm = a.istate[I_NMASK];
    double m = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
         k += (long long)gridDim.x * blockDim.x) {
        const long long j = a.vlist[k];
        const int n = __popc((unsigned)(a.nb[j] >> 1) & 0x3fu);
        m = fmax(m, fabs((double)d[j] + beta * (double)n));  // H_jj
        if (n > 0) m = fmax(m, fabs(beta));                 // H_jk = -beta
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    m = warp_max(m);
    if (lane == 0) sbuf[wid] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) m = fmax(m, sbuf[w]);
        a.partials[blockIdx.x] = m;
        __threadfence();
        const unsigned prev = atomicAdd((unsigned*)(a.istate + I_DONE0), 1u);
        s_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double h = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) h = fmax(h, __ldcg(a.partials + i));
    h = warp_max(h);
    __syncthreads();
    if (lane == 0) sbuf[wid] = h;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) h = fmax(h, sbuf[w]);
        a.scal[S_ICT_TAU] = droptol * h;
        a.istate[I_DONE0] = 0;
        if (!isfinite(h)) set_err(a.istate, FM_ERR_NONFINITE);
    }
}

// ------------------------------------------------------------------ the sweeps

// Plane indices of the factor storage.
enum : int { PL_R = 0, PL_A, PL_B, PL_C, PL_D1, PL_E, PL_F, PL_Y };  // PL_R: 1 / L_ii

// 1 / sqrt(s) for s > 0 in double: a float seed refined by two Newton-Raphson steps
// r <- r (3 - s r^2) / 2, each of which squares the relative error (about 2^-22 for the
// seed, so the second step reaches double rounding).  The GB300 FP64 pipe issues about
// 1/64 as fast as FP32, and this chain sits on every row's critical path.
__device__ __forceinline__ double rsqrt_nr(double s) {
    double r = (double)rsqrtf((float)s);
    const double hs = 0.5 * s;
    r = r * fma(-hs * r, r, 1.5);
    r = r * fma(-hs * r, r, 1.5);
    return r;
}

// A value another thread wrote at an earlier level: with one block the writer shares this
// SM's L1 and the block barrier orders the two, so a plain (L1-cached) load is safe; across
// blocks the load must bypass L1.
__device__ __forceinline__ double ld_level(const double* p) { return gridDim.x == 1 ? *p : __ldcg(p); }

// Separates two levels: a block barrier when one block holds every column, else the
// bounded grid barrier (every block is resident: cooperative launch, grid sized by occupancy).
__device__ __forceinline__ bool level_sync(const IctArgs& a) {
    if (gridDim.x == 1) {
        __syncthreads();
        return true;
    }
    return grid_barrier(a.istate, a.spin_limit);
}

template <typename T>
__global__ void __launch_bounds__(kIctThreads) k_ict_fwd(IctArgs a) {
    const int nx = a.geo.nx, ny = a.geo.ny, nz = a.geo.nz;
    const long long nxy = (long long)nx * ny, nv = a.geo.nv;
    double* Lp = a.L;
    auto P = [&](int k, long long j) -> double* { return Lp + (size_t)k * nv + j; };
    const T* d = (const T*)a.d;
    const T* g = (const T*)a.g;
    T* ipo = (T*)a.ip_out;
    const bool factor = d != nullptr;
    const double beta = a.beta;
    const double tau = factor ? a.scal[S_ICT_TAU] : 0.0;
    const int npair = ny * nz;
    const int tmax = (nx - 1) + 2 * (ny - 1) + 3 * (nz - 1);
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    bool bad = false;
    for (int t = 0; t <= tmax; ++t) {
        for (int pr = gtid; pr < npair; pr += nthr) {
            const int y = pr % ny, z = pr / ny, x = t - 2 * y - 3 * z;
            if (x < 0 || x >= nx) continue;
            const long long i = x + (long long)nx * y + nxy * z;
            const uint8_t b = a.nb[i];
            if (!(b & NB_IN)) continue;
            const long long ja = i - 1, jb = i - nx, jc = i - nxy, jd = i + 1 - nx, je = i + 1 - nxy, jf = i + nx - nxy;
            const bool ha = b & NB_XM, hb = b & NB_YM, hc = b & NB_ZM;
            const bool hd = x + 1 < nx && y > 0 && (a.nb[jd] & NB_IN);
            const bool he = x + 1 < nx && z > 0 && (a.nb[je] & NB_IN);
            const bool hf = y + 1 < ny && z > 0 && (a.nb[jf] & NB_IN);
            auto ld = [&](bool h, int k, long long j) { return h ? ld_level(P(k, j)) : 0.0; };
            // every value from the earlier rows first (independent loads), then the chain
            const double yc = ld(hc, PL_Y, jc), ye = ld(he, PL_Y, je), yf = ld(hf, PL_Y, jf),
                         yb = ld(hb, PL_Y, jb), yd = ld(hd, PL_Y, jd), ya = ld(ha, PL_Y, ja);
            double la, lb, lc, l_d, le, lf, rii;
            if (factor) {
                const double rc = ld(hc, PL_R, jc), re = ld(he, PL_R, je), rf = ld(hf, PL_R, jf),
                             rb = ld(hb, PL_R, jb), rd = ld(hd, PL_R, jd), ra = ld(ha, PL_R, ja);
                const double e_a = ld(he, PL_A, je), f_b = ld(hf, PL_B, jf), f_d = ld(hf, PL_D1, jf),
                             b_f = ld(hb, PL_F, jb), d_a = ld(hd, PL_A, jd), d_f = ld(hd, PL_F, jd),
                             a_d = ld(ha, PL_D1, ja), a_e = ld(ha, PL_E, ja);
                auto keep = [&](bool h, double v) { return h && fabs(v) >= tau ? v : 0.0; };
                lc = keep(hc, -beta * rc);
                le = keep(he, -(lc * e_a) * re);
                lf = keep(hf, -(lc * f_b + le * f_d) * rf);
                lb = keep(hb, (-beta - lc * b_f) * rb);
                l_d = keep(hd, -(lb * d_a + le * d_f) * rd);
                la = keep(ha, (-beta - lb * a_d - lc * a_e) * ra);
                const double h = (double)d[i] + beta * (double)__popc((unsigned)(b >> 1) & 0x3fu);
                const double s = h - (((la * la + lb * lb) + (lc * lc + l_d * l_d)) + (le * le + lf * lf));
                if (!(s > 0.0)) bad = true;
                rii = s > 0.0 ? rsqrt_nr(s) : 1.0;  // the error is reported; keep the arithmetic finite
                *P(PL_R, i) = rii;
                *P(PL_A, i) = la;
                *P(PL_B, i) = lb;
                *P(PL_C, i) = lc;
                *P(PL_D1, i) = l_d;
                *P(PL_E, i) = le;
                *P(PL_F, i) = lf;
                if (ipo) ipo[i] = (T)(rii * rii);
            } else {
                rii = *P(PL_R, i);
                la = *P(PL_A, i);
                lb = *P(PL_B, i);
                lc = *P(PL_C, i);
                l_d = *P(PL_D1, i);
                le = *P(PL_E, i);
                lf = *P(PL_F, i);
            }
            const double acc = (double)g[i] - ((lc * yc + le * ye) + (lf * yf + lb * yb) + (l_d * yd + la * ya));
            *P(PL_Y, i) = acc * rii;
        }
        if (t < tmax && !level_sync(a)) return;
    }
    // reported by the back sweep, after k_ict_check: fill beyond the held pattern (which can
    // itself make a pivot of the restricted factor non-positive) takes precedence
    if (bad) atomicExch(a.istate + I_ICT_BAD, 1);
}

template <typename T>
__global__ void __launch_bounds__(kIctThreads) k_ict_bwd(IctArgs a) {
    __shared__ double sbuf[2 * 32];
    const int nx = a.geo.nx, ny = a.geo.ny, nz = a.geo.nz;
    const long long nxy = (long long)nx * ny, nv = a.geo.nv;
    double* Lp = a.L;
    auto P = [&](int k, long long j) -> double* { return Lp + (size_t)k * nv + j; };
    T* p = (T*)a.p;
    const T* gd = (const T*)a.gdot;
    const T* gpd = (const T*)a.gpdot;
    const int npair = ny * nz;
    const int tmax = (nx - 1) + 2 * (ny - 1) + 3 * (nz - 1);
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    double acc2[2] = {0.0, 0.0};
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.istate[I_ICT_BAD]) {
        set_err(a.istate, FM_ERR_NOT_PD);
        a.istate[I_ICT_BAD] = 0;
    }
    for (int t = tmax; t >= 0; --t) {
        for (int pr = gtid; pr < npair; pr += nthr) {
            const int y = pr % ny, z = pr / ny, x = t - 2 * y - 3 * z;
            if (x < 0 || x >= nx) continue;
            const long long i = x + (long long)nx * y + nxy * z;
            const uint8_t b = a.nb[i];
            if (!(b & NB_IN)) {
                p[i] = T(0);
                continue;
            }
            // the later rows r = i - o that hold an entry in column i: L_{r,i} = plane o of row r
            const long long ra = i + 1, rb = i + nx, rc = i + nxy, rd = i - 1 + nx, re = i - 1 + nxy, rf = i - nx + nxy;
            const bool ha = b & NB_XP, hb = b & NB_YP, hc = b & NB_ZP;
            const bool hd = x > 0 && y + 1 < ny && (a.nb[rd] & NB_IN);
            const bool he = x > 0 && z + 1 < nz && (a.nb[re] & NB_IN);
            const bool hf = y > 0 && z + 1 < nz && (a.nb[rf] & NB_IN);
            auto ld = [&](bool h, int k, long long j) { return h ? ld_level(P(k, j)) : 0.0; };
            const double s = *P(PL_Y, i) - ((ld(ha, PL_A, ra) * ld(ha, PL_Y, ra) + ld(hd, PL_D1, rd) * ld(hd, PL_Y, rd)) +
                                            (ld(hf, PL_F, rf) * ld(hf, PL_Y, rf) + ld(hb, PL_B, rb) * ld(hb, PL_Y, rb)) +
                                            (ld(he, PL_E, re) * ld(he, PL_Y, re) + ld(hc, PL_C, rc) * ld(hc, PL_Y, rc)));
            const double xi = s * *P(PL_R, i);
            *P(PL_Y, i) = xi;  // y_i becomes x_i: every row that still needs y_i is this one
            p[i] = (T)xi;
            if (gd) acc2[0] += (double)gd[i] * (double)(T)xi;
            if (gpd) acc2[1] += (double)gpd[i] * (double)(T)xi;
        }
        if (t > 0 && !level_sync(a)) return;
    }
    if (gd || gpd) {
        double out[2];
        if (last_block_reduce<2>(acc2, a.partials, (unsigned*)(a.istate + I_DONE0), out, sbuf)) {
            if (threadIdx.x == 0) {
                a.scal[S_GP] = out[0];
                a.scal[S_GPREVP] = out[1];
                if (!isfinite(out[0]) || !isfinite(out[1])) set_err(a.istate, FM_ERR_NONFINITE);
            }
        }
    }
}

// ------------------------------------------------------------------ table-driven sweeps

// Voxel at offset (dx, dy, dz) from (x, y, z), or -1 when it lies outside the grid or the mask.
__device__ __forceinline__ long long ict_nbr(const IctArgs& a, int x, int y, int z, int dx, int dy, int dz) {
    const int xj = x + dx, yj = y + dy, zj = z + dz;
    if ((unsigned)xj >= (unsigned)a.geo.nx || (unsigned)yj >= (unsigned)a.geo.ny || (unsigned)zj >= (unsigned)a.geo.nz)
        return -1;
    const long long j = xj + (long long)a.geo.nx * (yj + (long long)a.geo.ny * zj);
    return (a.nb[j] & NB_IN) ? j : -1;
}

// The same factorisation and substitutions as k_ict_fwd / k_ict_bwd for any held pattern
// (a.tb): row i's entries in increasing column order, L_{i,j} = (H_ij - sum over the pairs
// (p1, p2) of o of L_{i,i+o_p1} L_{j,j+o_p2}) / L_jj, dropped below tau, then L_ii and y_i.
// Level t = x + B y + C z, with B and C chosen by the host so that every held offset points
// to a strictly lower level.
template <typename T>
__global__ void __launch_bounds__(kIctThreads) k_ictg_fwd(IctArgs a) {
    const int nx = a.geo.nx, ny = a.geo.ny, nz = a.geo.nz;
    const long long nxy = (long long)nx * ny, nv = a.geo.nv;
    const IctTables tb = a.tb;
    const int nh = tb.nh, PY = 1 + nh;
    double* Lp = a.L;
    auto P = [&](int k, long long j) -> double* { return Lp + (size_t)k * nv + j; };
    const T* d = (const T*)a.d;
    const T* g = (const T*)a.g;
    T* ipo = (T*)a.ip_out;
    const bool factor = d != nullptr;
    const double beta = a.beta;
    const double tau = factor ? a.scal[S_ICT_TAU] : 0.0;
    const int npair = ny * nz;
    const int tmax = (nx - 1) + tb.B * (ny - 1) + tb.C * (nz - 1);
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    bool bad = false;
    double lrow[kIctMaxOffsets];
    for (int t = 0; t <= tmax; ++t) {
        for (int pr = gtid; pr < npair; pr += nthr) {
            const int y = pr % ny, z = pr / ny, x = t - tb.B * y - tb.C * z;
            if (x < 0 || x >= nx) continue;
            const long long i = x + (long long)nx * y + nxy * z;
            const uint8_t b = a.nb[i];
            if (!(b & NB_IN)) continue;
            double rii;
            if (factor) {
                for (int k = 0; k < nh; ++k) {
                    const int h = tb.ord[k];
                    const long long j = ict_nbr(a, x, y, z, tb.off[3 * h], tb.off[3 * h + 1], tb.off[3 * h + 2]);
                    if (j < 0) {
                        lrow[h] = 0.0;
                        continue;
                    }
                    double sj = tb.hs[h] ? -beta : 0.0;
                    for (int q = tb.pp[h]; q < tb.pp[h + 1]; ++q) {
                        const double l1 = lrow[tb.pr[2 * q]];
                        if (l1 != 0.0) sj -= l1 * ld_level(P(1 + tb.pr[2 * q + 1], j));
                    }
                    const double v = sj * ld_level(P(0, j));
                    lrow[h] = fabs(v) >= tau ? v : 0.0;
                }
                double sq = 0.0;
                for (int h = 0; h < nh; ++h) sq += lrow[h] * lrow[h];
                const double sdiag = (double)d[i] + beta * (double)__popc((unsigned)(b >> 1) & 0x3fu) - sq;
                if (!(sdiag > 0.0)) bad = true;
                rii = sdiag > 0.0 ? rsqrt_nr(sdiag) : 1.0;  // the error is reported; keep the arithmetic finite
                *P(0, i) = rii;
                for (int h = 0; h < nh; ++h) *P(1 + h, i) = lrow[h];
                if (ipo) ipo[i] = (T)(rii * rii);
            } else {
                rii = *P(0, i);
                for (int h = 0; h < nh; ++h) lrow[h] = *P(1 + h, i);
            }
            double acc = (double)g[i];
            for (int h = 0; h < nh; ++h) {
                if (lrow[h] == 0.0) continue;
                const long long j = ict_nbr(a, x, y, z, tb.off[3 * h], tb.off[3 * h + 1], tb.off[3 * h + 2]);
                acc -= lrow[h] * ld_level(P(PY, j));
            }
            *P(PY, i) = acc * rii;
        }
        if (t < tmax && !level_sync(a)) return;
    }
    if (bad) atomicExch(a.istate + I_ICT_BAD, 1);
}

template <typename T>
__global__ void __launch_bounds__(kIctThreads) k_ictg_bwd(IctArgs a) {
    __shared__ double sbuf[2 * 32];
    const int nx = a.geo.nx, ny = a.geo.ny, nz = a.geo.nz;
    const long long nxy = (long long)nx * ny, nv = a.geo.nv;
    const IctTables tb = a.tb;
    const int nh = tb.nh, PY = 1 + nh;
    double* Lp = a.L;
    auto P = [&](int k, long long j) -> double* { return Lp + (size_t)k * nv + j; };
    T* p = (T*)a.p;
    const T* gd = (const T*)a.gdot;
    const T* gpd = (const T*)a.gpdot;
    const int npair = ny * nz;
    const int tmax = (nx - 1) + tb.B * (ny - 1) + tb.C * (nz - 1);
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    double acc2[2] = {0.0, 0.0};
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.istate[I_ICT_BAD]) {
        set_err(a.istate, FM_ERR_NOT_PD);
        a.istate[I_ICT_BAD] = 0;
    }
    for (int t = tmax; t >= 0; --t) {
        for (int pr = gtid; pr < npair; pr += nthr) {
            const int y = pr % ny, z = pr / ny, x = t - tb.B * y - tb.C * z;
            if (x < 0 || x >= nx) continue;
            const long long i = x + (long long)nx * y + nxy * z;
            if (!(a.nb[i] & NB_IN)) {
                p[i] = T(0);
                continue;
            }
            // the later rows r = i - o_h that hold an entry in column i: L_{r,i} = plane h of row r
            double sacc = *P(PY, i);
            for (int h = 0; h < nh; ++h) {
                const long long r = ict_nbr(a, x, y, z, -tb.off[3 * h], -tb.off[3 * h + 1], -tb.off[3 * h + 2]);
                if (r < 0) continue;
                const double l = ld_level(P(1 + h, r));
                if (l != 0.0) sacc -= l * ld_level(P(PY, r));
            }
            const double xi = sacc * *P(0, i);
            *P(PY, i) = xi;  // y_i becomes x_i: every row that still needs y_i is this one
            p[i] = (T)xi;
            if (gd) acc2[0] += (double)gd[i] * (double)(T)xi;
            if (gpd) acc2[1] += (double)gpd[i] * (double)(T)xi;
        }
        if (t > 0 && !level_sync(a)) return;
    }
    if (gd || gpd) {
        double out[2];
        if (last_block_reduce<2>(acc2, a.partials, (unsigned*)(a.istate + I_DONE0), out, sbuf)) {
            if (threadIdx.x == 0) {
                a.scal[S_GP] = out[0];
                a.scal[S_GPREVP] = out[1];
                if (!isfinite(out[0]) || !isfinite(out[1])) set_err(a.istate, FM_ERR_NONFINITE);
            }
        }
    }
}

// ------------------------------------------------------------------ fill beyond the held pattern

// Every would-be entry just outside the held pattern: at each candidate offset q (q = o_p1 -
// o_p2 for held p1, p2, pointing to an earlier voxel, not held), -(sum over its pairs of
// L_{i,i+o_p1} L_{j,j+o_p2}) / L_jj with j = i + q.  One that reaches tau sets its bit in
// tb.qflags and reports FM_ERR_FILL; the host then holds those offsets too and factors again.
// With nothing flagged no entry outside the pattern ever appears (by induction over the
// columns), so the held factor is the exact drop-tolerance factor.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_ict_check(IctArgs a) {
    const int nx = a.geo.nx, ny = a.geo.ny;
    const long long nxy = (long long)nx * ny, nv = a.geo.nv;
    const double* Lp = a.L;
    auto P = [&](int k, long long j) -> double { return Lp[(size_t)k * nv + j]; };
    const IctTables tb = a.tb;
    const double tau = a.scal[S_ICT_TAU];
    const long long nm = a.istate[I_NMASK];
    bool fill = false;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nm;
         k += (long long)gridDim.x * blockDim.x) {
        const long long i = a.vlist[k];
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / nxy);
        for (int q = 0; q < tb.nq; ++q) {
            double sq = 0.0;
            long long j = -2;
            for (int e = tb.qp[q]; e < tb.qp[q + 1]; ++e) {
                const double l1 = P(1 + tb.qpr[2 * e], i);
                if (l1 == 0.0) continue;
                if (j == -2) j = ict_nbr(a, x, y, z, tb.qoff[3 * q], tb.qoff[3 * q + 1], tb.qoff[3 * q + 2]);
                if (j < 0) break;
                sq += l1 * P(1 + tb.qpr[2 * e + 1], j);
            }
            if (j >= 0 && sq != 0.0 && fabs(sq * P(0, j)) >= tau) {
                atomicOr(tb.qflags + (q >> 5), 1u << (q & 31));
                fill = true;
            }
        }
    }
    if (fill) set_err(a.istate, FM_ERR_FILL);
}

// ------------------------------------------------------------------ launches

template <typename T>
int ictg_max_blocks_per_sm(int block) {
    int f = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&f, k_ictg_fwd<T>, block, 0) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ictg_bwd<T>, block, 0) != cudaSuccess) return 0;
    return f < b ? f : b;
}

template <typename T>
int ict_max_blocks_per_sm(int block) {
    int f = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&f, k_ict_fwd<T>, block, 0) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ict_bwd<T>, block, 0) != cudaSuccess) return 0;
    return f < b ? f : b;
}

template <typename T>
cudaError_t launch_ict_tau(const DataArgs& a, double droptol, int grid, cudaStream_t s) {
    k_ict_tau<T><<<grid, kThreads, 0, s>>>(a, droptol);
    return cudaGetLastError();
}
// The level sweeps wait at a grid barrier, so every block must be resident at once.  A
// cooperative launch guarantees that (or refuses the launch) even when other kernels run
// beside the sweep, e.g. the other volumes' branches of a batched graph.
template <typename T>
cudaError_t launch_ict_fwd(const IctArgs& a, int grid, int block, cudaStream_t s) {
    IctArgs copy = a;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void*)k_ict_fwd<T>, dim3(grid), dim3(block), args, 0, s);
}
template <typename T>
cudaError_t launch_ict_bwd(const IctArgs& a, int grid, int block, cudaStream_t s) {
    IctArgs copy = a;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void*)k_ict_bwd<T>, dim3(grid), dim3(block), args, 0, s);
}
template <typename T>
cudaError_t launch_ictg_fwd(const IctArgs& a, int grid, int block, cudaStream_t s) {
    IctArgs copy = a;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void*)k_ictg_fwd<T>, dim3(grid), dim3(block), args, 0, s);
}
template <typename T>
cudaError_t launch_ictg_bwd(const IctArgs& a, int grid, int block, cudaStream_t s) {
    IctArgs copy = a;
    void* args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void*)k_ictg_bwd<T>, dim3(grid), dim3(block), args, 0, s);
}
template <typename T>
cudaError_t launch_ict_check(const IctArgs& a, int grid, cudaStream_t s) {
    k_ict_check<T><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

#define FM_ICT_INST(T)                                                                   \
    template cudaError_t launch_ict_tau<T>(const DataArgs&, double, int, cudaStream_t); \
    template cudaError_t launch_ict_fwd<T>(const IctArgs&, int, int, cudaStream_t);     \
    template cudaError_t launch_ict_bwd<T>(const IctArgs&, int, int, cudaStream_t);     \
    template cudaError_t launch_ict_check<T>(const IctArgs&, int, cudaStream_t);        \
    template cudaError_t launch_ictg_fwd<T>(const IctArgs&, int, int, cudaStream_t);    \
    template cudaError_t launch_ictg_bwd<T>(const IctArgs&, int, int, cudaStream_t);    \
    template int ict_max_blocks_per_sm<T>(int);                                         \
    template int ictg_max_blocks_per_sm<T>(int);
FM_ICT_INST(float)
FM_ICT_INST(double)

}  // namespace fm
