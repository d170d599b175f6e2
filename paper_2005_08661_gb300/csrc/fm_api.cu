// fm_api.cu -- host side of the C ABI declared in include/fm.h: context, argument
// checking, buffer ownership, and the launch sequence of one NCG-MLS-IC outer iteration
// (Algorithm box), replayed from a captured CUDA graph.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fm_internal.h"

using namespace fm;

struct fm_ctx {
    int nx = 0, ny = 0, nz = 0, nc = 0, L = 0;
    long long nv = 0;
    fm_opts o{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t ts = 4;  // sizeof voxel type
    bool literal = false;
    bool have_data = false, have_factor = false;
    double beta = 0.0;
    double te[FM_MAX_ECHO] = {};
    Pairs pr{};
    // water-fat model (Eq. gamma); set by fm_set_fat_model, applied by fm_set_data
    bool wf = false;
    std::vector<double> fat_amp, fat_freq;
    double fat_re[FM_MAX_ECHO] = {}, fat_im[FM_MAX_ECHO] = {};  // phi_l = sum_p a_p e^{i 2 pi f_p t_l}
    double ginv[8] = {};                                         // (gamma^H gamma)^{-1}
    void* rho = nullptr;                                         // T compact [nv]: sum |r_cdmn|
    // device buffers
    void *pairs = nullptr, *coils = nullptr, *w0 = nullptr;
    uint8_t* nb = nullptr;
    int *vlist = nullptr, *chunk_off = nullptr;
    void *w[2] = {nullptr, nullptr}, *z[2] = {nullptr, nullptr}, *g[2] = {nullptr, nullptr};
    void *d = nullptr, *p = nullptr, *v = nullptr, *ip = nullptr;
    double *scal = nullptr, *partials = nullptr, *tile_part = nullptr;
    void* face = nullptr;
    size_t face_bytes = 0;  // per-tile IC face buffers (the forward part starts unset: all bits set)
    double *hist_cost = nullptr, *hist_alpha = nullptr, *hist_mu = nullptr;
    int hist_cap = 0;
    int hist_gen = 0;      // bumped when the history buffers move (captured graphs hold them)
    int* istate = nullptr;
    int* icint = nullptr;  // IC sweeps: [0] forward ticket, [1] back-substitution ticket, [2] its done count, [3] pad
    int* order = nullptr;
    int ntx = 0, nty = 0, ntz = 0, ntiles = 0;
    int ic_wxy = 2, ic_wz = 1;  // forward tile claim order weights
    int nsm = 0, grid_data = 0, grid_ls = 0, grid_ic = 0, grid_icb = 0;  // grid_icb: backward IC sweep
    int base_data = 0, base_ls = 0, base_ic = 0, base_icb = 0;
    int occ_icb = 0;  // resident back-substitution blocks per SM the kernel allows
    int grid_ict = 0, base_ict = 0, block_ict = 0;  // drop-tolerance IC sweeps (persistent, level barriers)
    int grid_ictg = 0, base_ictg = 0;                // the same for the table-driven sweeps
    // drop-tolerance IC: the held pattern (dx, dy, dz per offset, plane order), its device
    // tables, the factor planes [nh + 2][nv] and the candidate fill offsets of the check
    std::vector<int> ict_off, ict_qoff;
    int* ict_tab = nullptr;
    unsigned* ict_qflags = nullptr;
    IctTables ict_tb{};
    int ict_nplanes = 0;
    double* ict_L = nullptr;
    void* ict_w0 = nullptr;  // a solve's start map, kept while a growing pattern reruns the solve
    int last_niter = 0;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphExec_t cg_gexec = nullptr;  // adjoint CG iterations (tolerance and limit are arguments)
    double cg_tol2 = -1.0;
    int cg_maxiter = -1;
    bool profiling = false;
    cudaEvent_t ev[2][FM_NKERNEL][2] = {};
    bool ev_rec[2][FM_NKERNEL] = {};
    // host-buffer entry points: two staging sets of device inputs, filled on a copy stream
    // while the other set's acquisition is being solved, and the field map's device copy
    cudaStream_t copy_stream = nullptr;
    void *st_y[2] = {nullptr, nullptr}, *st_s[2] = {nullptr, nullptr};
    uint8_t* st_m[2] = {nullptr, nullptr};
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_read[2] = {nullptr, nullptr};
    int st_next = 0;
    void* w_io = nullptr;
    float* ip_lo = nullptr;  // fm_ic_factor64 in FP32 mode: low parts of the inverse pivots
    std::string err;
};

namespace {

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int fail(fm_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(fm_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) return fail(c, FM_ERR_OOM, std::string(what) + ": out of device memory");
    return fail(c, FM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define FM_CK(call, what)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

template <typename P>
cudaError_t dalloc(P** ptr, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    *ptr = (P*)q;
    return e;
}

void free_all(fm_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cg_gexec) cudaGraphExecDestroy(c->cg_gexec);
    for (auto& a : c->ev)
        for (auto& b : a)
            for (cudaEvent_t& e : b)
                if (e) cudaEventDestroy(e);
    void* bufs[] = {c->pairs, c->coils, c->w0, c->nb, c->vlist, c->chunk_off, c->w[0], c->w[1], c->z[0], c->z[1], c->g[0],
                    c->g[1], c->d, c->p, c->v, c->ip, c->scal, c->partials, c->face, c->tile_part, c->rho,
                    c->hist_cost, c->hist_alpha, c->hist_mu, c->istate, c->icint, c->order, c->ict_L,
                    c->st_y[0], c->st_y[1], c->st_s[0], c->st_s[1], c->st_m[0], c->st_m[1], c->w_io, c->ip_lo,
                    c->ict_tab, c->ict_qflags, c->ict_w0};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (int k = 0; k < 2; ++k) {
        if (c->ev_copied[k]) cudaEventDestroy(c->ev_copied[k]);
        if (c->ev_read[k]) cudaEventDestroy(c->ev_read[k]);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

// The grid barrier's arrival count.  A block that gives up in grid_barrier (FM_ERR_TIMEOUT)
// leaves its arrival counted; if the count survived into the next launch sequence, a later
// barrier would open before every block had arrived.  So every launch sequence starts from
// a zero count (stream-ordered after the launch that timed out has finished), and an error
// read back clears it together with the error word.  The error word itself is cleared only
// when it is read: an error of an earlier asynchronous call is reported by the next call
// that synchronises.
cudaError_t reset_barrier(fm_ctx* c) {
    return cudaMemsetAsync(c->istate + I_BAR_COUNT, 0, sizeof(int), c->stream);
}
// After a device error the IC forward sweep's face entries may hold values that no reader
// consumed (a fetch that gave up), so they are set back to the unset pattern too.
cudaError_t reset_dev(fm_ctx* c) {
    cudaError_t e = cudaMemsetAsync(c->istate + I_ERR, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = reset_barrier(c);
    if (e == cudaSuccess && c->face) e = cudaMemsetAsync(c->face, 0xff, c->face_bytes, c->stream);
    return e;
}

// Records a profiling event: inside a stream capture as an external event node of the graph
// (so replays time the kernels), outside one as a plain record.  A failed record only loses
// a timing, so its error is cleared rather than left for the next launch check to find.
void prof_record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaError_t r = cudaStreamIsCapturing(s, &st);
    if (r == cudaSuccess)
        r = st == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                                 : cudaEventRecord(e, s);
    if (r != cudaSuccess) cudaGetLastError();
}

// Read back the device error word and clear it.
int check_dev(fm_ctx* c) {
    int e = 0;
    cudaError_t ce = cudaMemcpyAsync(&e, c->istate + I_ERR, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "synchronise");
    if (e != 0) {
        reset_dev(c);
        const char* what = e == FM_ERR_NOT_PD ? "IC(0) pivot <= 0 (H not positive definite on the mask)"
                         : e == FM_ERR_TIMEOUT ? "device-side wait exceeded spin_limit"
                         : e == FM_ERR_NONFINITE ? "non-finite global reduction"
                         : e == FM_ERR_FILL ? "drop tolerance keeps fill-in outside the held pattern"
                         : "device error";
        return fail(c, e, what);
    }
    return FM_OK;
}

DataArgs base_args(fm_ctx* c) {
    DataArgs a{};
    a.geo = Geo{c->nx, c->ny, c->nz, c->nv};
    a.nc = c->nc;
    a.L = c->L;
    a.pr = c->pr;
    a.beta = c->beta;
    a.literal = c->literal ? 1 : 0;
    a.wf = c->wf ? 1 : 0;
    a.pairs = c->pairs;
    a.coils = c->coils;
    a.nb = c->nb;
    a.vlist = c->vlist;
    a.scal = c->scal;
    a.partials = c->partials;
    a.istate = c->istate;
    a.nls = c->o.nls;
    a.spin_limit = c->o.spin_limit;
    return a;
}

IcArgs ic_args(fm_ctx* c) {
    IcArgs a{};
    a.geo = Geo{c->nx, c->ny, c->nz, c->nv};
    a.ntx = c->ntx;
    a.nty = c->nty;
    a.ntz = c->ntz;
    a.ntiles = c->ntiles;
    a.order = c->order;
    a.beta = c->beta;
    a.nb = c->nb;
    a.face = c->face;
    a.scal = c->scal;
    a.istate = c->istate;
    a.spin_limit = c->o.spin_limit;
    return a;
}

template <typename T>
cudaError_t run_grad(fm_ctx* c, const void* w_in, const void* zdir, void* w_out, void* g, void* d,
                     double* hist) {
    DataArgs a = base_args(c);
    a.w_in = w_in;
    a.z = zdir;
    a.w_out = w_out;
    a.g = g;
    a.d = d;
    a.cost_hist = hist;
    return launch_grad<T>(a, c->grid_data, c->stream);
}

// forward (pivots when d != null) + backward substitution: p = (L L')^{-1} g
template <typename T>
cudaError_t run_ic0(fm_ctx* c, const void* d, const void* g, void* p, const void* gdot, const void* gpdot,
                    int slot, float* ip_lo = nullptr) {
    cudaError_t e = cudaMemsetAsync(c->icint, 0, 4 * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    IcArgs f = ic_args(c);
    f.ticket = c->icint + 0;
    f.d = d;
    f.ip_in = d ? nullptr : c->ip;
    f.g = g;
    f.v = c->v;
    f.ip_out = c->ip;
    f.ip_lo_out = ip_lo;
    {
        fm_ctx* pc = slot >= 0 ? c : nullptr;
        if (pc && pc->profiling) prof_record(pc->ev[slot][FM_K_IC_FWD][0], c->stream);
        e = launch_ic_fwd<T>(f, c->grid_ic, c->stream);
        if (pc && pc->profiling) {
            prof_record(pc->ev[slot][FM_K_IC_FWD][1], c->stream);
            pc->ev_rec[slot][FM_K_IC_FWD] = true;
        }
    }
    if (e != cudaSuccess) return e;
    IcArgs b = ic_args(c);
    b.ticket = c->icint + 1;
    b.done = c->icint + 2;
    b.order = c->order + c->ntiles;
    b.vin = c->v;
    b.ipb = c->ip;
    b.p = p;
    b.gdot = gdot;
    b.gpdot = gpdot;
    b.tile_part = (gdot || gpdot) ? c->tile_part : nullptr;
    if (slot >= 0 && c->profiling) prof_record(c->ev[slot][FM_K_IC_BWD][0], c->stream);
    e = launch_ic_bwd<T>(b, c->grid_icb, c->stream);
    if (slot >= 0 && c->profiling) {
        prof_record(c->ev[slot][FM_K_IC_BWD][1], c->stream);
        c->ev_rec[slot][FM_K_IC_BWD] = true;
    }
    return e;
}

// ------------------------------------------------------------------ drop-tolerance IC pattern

// lexicographic (dz, dy, dx) order of offsets = natural order of the voxels they point to
bool lex_less(const int* a, const int* b) {
    if (a[2] != b[2]) return a[2] < b[2];
    if (a[1] != b[1]) return a[1] < b[1];
    return a[0] < b[0];
}

int ceil_div_pos(long long num, long long den) {  // ceil(num / den), den > 0
    return (int)(num >= 0 ? (num + den - 1) / den : -((-num) / den));
}

// Builds the device tables of the held pattern c->ict_off (see IctTables), the level
// coefficients, the candidate fill offsets, and (re)allocates the factor planes.  Synchronous.
int ict_build(fm_ctx* c) {
    const int nh = (int)c->ict_off.size() / 3;
    const int* off = c->ict_off.data();
    std::vector<int> ord(nh), hs(nh), pp(nh + 1, 0), pr, qoff, qp(1, 0), qpr;
    for (int h = 0; h < nh; ++h) ord[h] = h;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return lex_less(off + 3 * a, off + 3 * b); });
    for (int h = 0; h < nh; ++h) {
        const int* o = off + 3 * h;
        hs[h] = (std::abs(o[0]) + std::abs(o[1]) + std::abs(o[2])) == 1 ? 1 : 0;
    }
    auto held = [&](int dx, int dy, int dz) {
        for (int h = 0; h < nh; ++h)
            if (off[3 * h] == dx && off[3 * h + 1] == dy && off[3 * h + 2] == dz) return h;
        return -1;
    };
    for (int h = 0; h < nh; ++h) {  // pairs (p1, p2) with o_p1 - o_p2 = o_h
        for (int p2 = 0; p2 < nh; ++p2) {
            const int p1 = held(off[3 * h] + off[3 * p2], off[3 * h + 1] + off[3 * p2 + 1], off[3 * h + 2] + off[3 * p2 + 2]);
            if (p1 >= 0) { pr.push_back(p1); pr.push_back(p2); }
        }
        pp[h + 1] = (int)pr.size() / 2;
    }
    // candidate fill: q = o_p1 - o_p2 pointing to an earlier voxel, not held
    std::vector<std::vector<int>> cand;  // per candidate: dx, dy, dz, then its pairs
    for (int p1 = 0; p1 < nh; ++p1)
        for (int p2 = 0; p2 < nh; ++p2) {
            const int q[3] = {off[3 * p1] - off[3 * p2], off[3 * p1 + 1] - off[3 * p2 + 1], off[3 * p1 + 2] - off[3 * p2 + 2]};
            const int zero[3] = {0, 0, 0};
            if (!lex_less(q, zero) || held(q[0], q[1], q[2]) >= 0) continue;
            size_t k = 0;
            for (; k < cand.size(); ++k)
                if (cand[k][0] == q[0] && cand[k][1] == q[1] && cand[k][2] == q[2]) break;
            if (k == cand.size()) cand.push_back({q[0], q[1], q[2]});
            cand[k].push_back(p1);
            cand[k].push_back(p2);
        }
    if ((int)cand.size() > kIctMaxCand) return fail(c, FM_ERR_FILL, "drop-tolerance IC: too many candidate fill offsets");
    for (auto& q : cand) {
        qoff.insert(qoff.end(), q.begin(), q.begin() + 3);
        qpr.insert(qpr.end(), q.begin() + 3, q.end());
        qp.push_back((int)qpr.size() / 2);
    }
    // level t = x + B y + C z with t(o) <= -1 for every held offset
    int B = 1, C = 1;
    for (int h = 0; h < nh; ++h) {
        const int* o = off + 3 * h;
        if (o[2] == 0 && o[1] < 0) B = std::max(B, ceil_div_pos((long long)o[0] + 1, -o[1]));
    }
    for (int h = 0; h < nh; ++h) {
        const int* o = off + 3 * h;
        if (o[2] < 0) C = std::max(C, ceil_div_pos((long long)o[0] + (long long)B * o[1] + 1, -o[2]));
    }
    const int nq = (int)cand.size();
    std::vector<int> tab;
    auto put = [&](const std::vector<int>& v) { const size_t at = tab.size(); tab.insert(tab.end(), v.begin(), v.end()); return at; };
    const size_t a_off = put(c->ict_off), a_ord = put(ord), a_hs = put(hs), a_pp = put(pp), a_pr = put(pr),
                 a_qoff = put(qoff), a_qp = put(qp), a_qpr = put(qpr);
    if (c->ict_tab) { cudaFree(c->ict_tab); c->ict_tab = nullptr; }
    if (c->ict_qflags) { cudaFree(c->ict_qflags); c->ict_qflags = nullptr; }
    const int nflag = std::max(1, (nq + 31) / 32);
    if (dalloc(&c->ict_tab, std::max<size_t>(tab.size(), 1) * sizeof(int)) != cudaSuccess ||
        dalloc(&c->ict_qflags, nflag * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, FM_ERR_OOM, "drop-tolerance IC tables");
    }
    FM_CK(cudaMemcpy(c->ict_tab, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice), "upload tables");
    FM_CK(cudaMemset(c->ict_qflags, 0, nflag * sizeof(unsigned)), "clear flags");
    IctTables& t = c->ict_tb;
    t.nh = nh;
    t.nq = nq;
    t.B = B;
    t.C = C;
    t.off = c->ict_tab + a_off;
    t.ord = c->ict_tab + a_ord;
    t.hs = c->ict_tab + a_hs;
    t.pp = c->ict_tab + a_pp;
    t.pr = c->ict_tab + a_pr;
    t.qoff = c->ict_tab + a_qoff;
    t.qp = c->ict_tab + a_qp;
    t.qpr = c->ict_tab + a_qpr;
    t.qflags = c->ict_qflags;
    c->ict_qoff = qoff;
    if (nh + 2 > c->ict_nplanes) {  // grow the factor planes (the old factor is discarded)
        FM_CK(cudaStreamSynchronize(c->stream), "synchronise");
        if (c->ict_L) cudaFree(c->ict_L);
        c->ict_L = nullptr;
        c->ict_nplanes = 0;
        if (dalloc(&c->ict_L, (size_t)(nh + 2) * c->nv * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, FM_ERR_OOM, "drop-tolerance IC factor planes");
        }
        c->ict_nplanes = nh + 2;
        c->have_factor = false;
    }
    FM_CK(cudaMemset(c->ict_L, 0, (size_t)c->ict_nplanes * c->nv * sizeof(double)), "clear factor");
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }  // the tables are kernel arguments
    if (c->cg_gexec) { cudaGraphExecDestroy(c->cg_gexec); c->cg_gexec = nullptr; }
    return FM_OK;
}

// After a factorisation reported FM_ERR_FILL: hold every flagged candidate offset too.  Returns
// 1 when the pattern grew, 0 when nothing was flagged, or an error (FM_ERR_FILL beyond
// kIctMaxOffsets held offsets).  Synchronous.
int ict_grow(fm_ctx* c) {
    if (c->o.precond != FM_PC_ICT || !c->ict_qflags) return 0;
    const int nq = c->ict_tb.nq;
    std::vector<unsigned> fl(std::max(1, (nq + 31) / 32), 0u);
    FM_CK(cudaMemcpy(fl.data(), c->ict_qflags, fl.size() * sizeof(unsigned), cudaMemcpyDeviceToHost), "read flags");
    int added = 0;
    for (int q = 0; q < nq; ++q)
        if (fl[q >> 5] & (1u << (q & 31))) {
            c->ict_off.insert(c->ict_off.end(), c->ict_qoff.begin() + 3 * q, c->ict_qoff.begin() + 3 * q + 3);
            ++added;
        }
    if (!added) return 0;
    if ((int)c->ict_off.size() / 3 > kIctMaxOffsets)
        return fail(c, FM_ERR_FILL, "drop-tolerance IC: the kept fill needs more than 64 offsets");
    const int rc = ict_build(c);
    return rc == FM_OK ? 1 : rc;
}

// The same with the drop-tolerance IC (k_ict.cu): tau from H_max, factor + forward sweep,
// the exactness check, back sweep; or, with d null, the two sweeps on the stored factor.
template <typename T>
cudaError_t run_ict(fm_ctx* c, const void* d, const void* g, void* p, const void* gdot, const void* gpdot,
                    int slot) {
    cudaError_t e = cudaSuccess;
    IctArgs a{};
    a.geo = Geo{c->nx, c->ny, c->nz, c->nv};
    a.beta = c->beta;
    a.nb = c->nb;
    a.vlist = c->vlist;
    a.d = d;
    a.g = g;
    a.L = c->ict_L;
    a.tb = c->ict_tb;
    a.ip_out = d ? c->ip : nullptr;
    a.p = p;
    a.gdot = gdot;
    a.gpdot = gpdot;
    a.scal = c->scal;
    a.partials = c->partials;
    a.istate = c->istate;
    a.spin_limit = c->o.spin_limit;
    const bool prof = slot >= 0 && c->profiling;
    if (d) {
        DataArgs t = base_args(c);
        t.d = const_cast<void*>(d);  // read only here
        e = launch_ict_tau<T>(t, c->o.droptol, c->grid_data, c->stream);
        if (e != cudaSuccess) return e;
    }
    const bool base = c->ict_tb.nh == kIctBaseOffsets;  // the unrolled kernels hold exactly the base pattern
    if (prof) prof_record(c->ev[slot][FM_K_IC_FWD][0], c->stream);
    e = base ? launch_ict_fwd<T>(a, c->grid_ict, c->block_ict, c->stream)
             : launch_ictg_fwd<T>(a, c->grid_ictg, c->block_ict, c->stream);
    if (prof) {
        prof_record(c->ev[slot][FM_K_IC_FWD][1], c->stream);
        c->ev_rec[slot][FM_K_IC_FWD] = true;
    }
    if (e != cudaSuccess) return e;
    if (d) {  // exact only while nothing outside the held pattern survives: FM_ERR_FILL otherwise
        e = launch_ict_check<T>(a, c->grid_data, c->stream);
        if (e != cudaSuccess) return e;
    }
    if (prof) prof_record(c->ev[slot][FM_K_IC_BWD][0], c->stream);
    e = base ? launch_ict_bwd<T>(a, c->grid_ict, c->block_ict, c->stream)
             : launch_ictg_bwd<T>(a, c->grid_ictg, c->block_ict, c->stream);
    if (prof) {
        prof_record(c->ev[slot][FM_K_IC_BWD][1], c->stream);
        c->ev_rec[slot][FM_K_IC_BWD] = true;
    }
    return e;
}

// p = (L L')^{-1} g with the context's incomplete factor (recomputed from d when non-null)
template <typename T>
cudaError_t run_ic(fm_ctx* c, const void* d, const void* g, void* p, const void* gdot, const void* gpdot,
                   int slot = -1) {
    if (c->o.precond == FM_PC_ICT) return run_ict<T>(c, d, g, p, gdot, gpdot, slot);
    return run_ic0<T>(c, d, g, p, gdot, gpdot, slot);
}

// Brackets one kernel class of iteration slot `cur` with events when profiling.
struct Mark {
    fm_ctx* c;
    int cur, k;
    Mark(fm_ctx* c_, int cur_, int k_) : c(c_), cur(cur_), k(k_) {
        if (c->profiling) prof_record(c->ev[cur][k][0], c->stream);
    }
    ~Mark() {
        if (c->profiling) {
            prof_record(c->ev[cur][k][1], c->stream);
            c->ev_rec[cur][k] = true;
        }
    }
};

// One outer iteration (Algorithm box) with cur = i & 1 selecting the ping-pong buffers.
template <typename T>
cudaError_t iteration(fm_ctx* c, int cur) {
    const int nxt = cur ^ 1;
    cudaError_t e;
    {
        Mark m(c, cur, FM_K_GRAD);
        e = run_grad<T>(c, c->w[cur], c->z[cur], c->w[nxt], c->g[cur], c->d, c->hist_cost);
    }
    if (e != cudaSuccess) return e;
    if (c->o.precond == FM_PC_IC0 || c->o.precond == FM_PC_ICT) {
        e = run_ic<T>(c, c->d, c->g[cur], c->p, c->g[cur], c->g[nxt], cur);
    } else if (c->o.precond == FM_PC_RB) {
        DataArgs a = base_args(c);
        a.g = c->g[cur];
        a.g_prev = c->g[nxt];
        a.d = c->d;
        a.z_new = c->p;
        {
            Mark m(c, cur, FM_K_IC_FWD);
            e = launch_rb_black<T>(a, c->grid_data, c->stream);
        }
        if (e == cudaSuccess) {
            Mark m(c, cur, FM_K_IC_BWD);
            e = launch_rb_red<T>(a, c->grid_data, c->stream);
        }
    } else {
        Mark m(c, cur, FM_K_IC_BWD);
        DataArgs a = base_args(c);
        a.g = c->g[cur];
        a.g_prev = c->g[nxt];
        a.d = c->d;
        a.z_new = c->p;
        e = launch_pdiag<T>(a, c->o.precond == FM_PC_DIAG ? 1 : 2, c->grid_data, c->stream);
    }
    if (e != cudaSuccess) return e;
    DataArgs a = base_args(c);
    a.p = c->p;
    a.z_old = c->z[cur];
    a.z_new = c->z[nxt];
    a.w_out = c->w[nxt];
    a.g = c->g[cur];
    a.d = c->d;
    a.mu_hist = c->hist_mu;
    a.alpha_hist = c->hist_alpha;
    {
        Mark m(c, cur, FM_K_LS);  // direction + line search
        e = launch_ls<T>(a, c->grid_ls, c->stream);
    }
    return e;
}

// Enqueue everything a solve needs before its first outer iteration.
template <typename T>
int solve_begin(fm_ctx* c, void* omega, int init, int niter, bool host_io = false) {
    if (niter + 1 > c->hist_cap) {
        if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
        cudaFree(c->hist_cost); cudaFree(c->hist_alpha); cudaFree(c->hist_mu);
        c->hist_cost = c->hist_alpha = c->hist_mu = nullptr;
        c->hist_cap = 0;
        const int cap = std::max(niter + 1, 128);
        FM_CK(dalloc(&c->hist_cost, cap * sizeof(double)), "allocate history");
        FM_CK(dalloc(&c->hist_alpha, cap * sizeof(double)), "allocate history");
        FM_CK(dalloc(&c->hist_mu, cap * sizeof(double)), "allocate history");
        c->hist_cap = cap;
        c->hist_gen++;
    }
    const size_t vb = (size_t)c->nv * c->ts;
    cudaStream_t s = c->stream;
    FM_CK(reset_barrier(c), "reset");
    // the kernels write mask voxels only: every entry outside the mask starts (and stays) 0
    if (init) {
        FM_CK(cudaMemcpyAsync(c->w[0], c->w0, vb, cudaMemcpyDeviceToDevice, s), "copy omega");
    } else if (host_io) {  // through w[1], which is cleared next
        FM_CK(cudaMemcpyAsync(c->w[1], omega, vb, cudaMemcpyHostToDevice, s), "copy omega in");
        FM_CK(launch_masked_copy<T>(c->w[1], c->w[0], c->nb, c->nv, c->grid_data, s), "copy omega");
    } else {
        FM_CK(launch_masked_copy<T>(omega, c->w[0], c->nb, c->nv, c->grid_data, s), "copy omega");
    }
    FM_CK(cudaMemsetAsync(c->w[1], 0, vb, s), "reset field map");
    for (int k = 0; k < 2; ++k) {
        FM_CK(cudaMemsetAsync(c->z[k], 0, vb, s), "reset direction");
        FM_CK(cudaMemsetAsync(c->g[k], 0, vb, s), "reset gradient");
    }
    FM_CK(cudaMemsetAsync(c->p, 0, vb, s), "reset preconditioned gradient");
    FM_CK(cudaMemsetAsync(c->scal + S_ALPHA, 0, sizeof(double), s), "reset step");
    FM_CK(cudaMemsetAsync(c->scal + S_GP, 0, 4 * sizeof(double), s), "reset dots");
    FM_CK(cudaMemsetAsync(c->istate + I_ITER, 0, sizeof(int), s), "reset counter");
    return FM_OK;
}

// Enqueue the last update, the copy of the field map out and of the cost history.
template <typename T>
int solve_end(fm_ctx* c, void* omega, int niter, double* cost_hist, bool host_io = false) {
    const size_t vb = (size_t)c->nv * c->ts;
    cudaStream_t s = c->stream;
    const int cur = niter & 1;
    FM_CK(run_grad<T>(c, c->w[cur], c->z[cur], c->w[cur ^ 1], c->g[cur], c->d, c->hist_cost), "final update");
    if (host_io) {
        Mark m(c, 0, FM_K_D2H);
        FM_CK(cudaMemcpyAsync(omega, c->w[cur ^ 1], vb, cudaMemcpyDeviceToHost, s), "copy omega out");
    } else {
        FM_CK(cudaMemcpyAsync(omega, c->w[cur ^ 1], vb, cudaMemcpyDeviceToDevice, s), "copy omega out");
    }
    if (cost_hist)
        FM_CK(cudaMemcpyAsync(cost_hist, c->hist_cost, (niter + 1) * sizeof(double), cudaMemcpyDeviceToHost, s),
              "copy cost history");
    c->last_niter = niter;
    return FM_OK;
}

constexpr int kIctMaxRounds = 64;  // pattern growths one call may go through

// Enqueues the whole solve; synchronises (and reports device errors) only when the cost
// history is requested -- or with the drop-tolerance IC, which checks every solve: when a
// factorisation keeps fill outside the held pattern, the pattern grows and the solve runs
// again from the same start (a larger held pattern gives the identical factor, so the result
// is the drop-tolerance solve itself).
template <typename T>
int solve_once(fm_ctx* c, const void* omega_in, bool in_host, void* omega_out, bool out_host, int init, int niter,
               double* cost_hist);

template <typename T>
int solve_t(fm_ctx* c, void* omega, int init, int niter, double* cost_hist, bool host_io = false) {
    if (c->o.precond != FM_PC_ICT) {
        const int rc = solve_once<T>(c, omega, host_io, omega, host_io, init, niter, cost_hist);
        if (rc != FM_OK) return rc;
        return cost_hist ? check_dev(c) : FM_OK;
    }
    const void* in = omega;
    bool in_host = host_io;
    if (!init) {  // keep the start map: the output overwrites omega
        const size_t vb = (size_t)c->nv * c->ts;
        if (!c->ict_w0 && dalloc(&c->ict_w0, vb) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, FM_ERR_OOM, "allocate start map");
        }
        FM_CK(cudaMemcpyAsync(c->ict_w0, omega, vb, host_io ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                              c->stream), "keep start map");
        in = c->ict_w0;
        in_host = false;
    }
    for (int round = 0;; ++round) {
        int rc = solve_once<T>(c, in, in_host, omega, host_io, init, niter, cost_hist);
        if (rc != FM_OK) return rc;
        rc = check_dev(c);
        if (rc != FM_ERR_FILL || round >= kIctMaxRounds) return rc;
        const int g = ict_grow(c);
        if (g <= 0) return g < 0 ? g : rc;
    }
}

template <typename T>
int solve_once(fm_ctx* c, const void* omega_in, bool in_host, void* omega_out, bool out_host, int init, int niter,
               double* cost_hist) {
    int rc = solve_begin<T>(c, const_cast<void*>(omega_in), init, niter, in_host);
    if (rc != FM_OK) return rc;
    cudaStream_t s = c->stream;
    int i = 0;
    if (c->o.use_graph && niter >= 2) {
        if (!c->gexec) {
            cudaGraph_t graph = nullptr;
            FM_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
            cudaError_t e0 = iteration<T>(c, 0);
            cudaError_t e1 = e0 == cudaSuccess ? iteration<T>(c, 1) : e0;
            cudaError_t ee = cudaStreamEndCapture(s, &graph);
            if (e1 != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(c, e1, "capture iteration"); }
            FM_CK(ee, "end capture");
            cudaError_t ei = cudaGraphInstantiate(&c->gexec, graph, 0);
            cudaGraphDestroy(graph);
            FM_CK(ei, "instantiate graph");
        }
        for (; i + 2 <= niter; i += 2) FM_CK(cudaGraphLaunch(c->gexec, s), "launch graph");
    }
    for (; i < niter; ++i) FM_CK(iteration<T>(c, i & 1), "launch iteration");
    return solve_end<T>(c, omega_out, niter, cost_hist, out_host);
}

// ------------------------------------------------------------------ implicit differentiation

AdjArgs adj_args(fm_ctx* c) {
    AdjArgs a{};
    a.geo = Geo{c->nx, c->ny, c->nz, c->nv};
    a.nc = c->nc;
    a.L = c->L;
    a.pr = c->pr;
    a.beta = c->beta;
    for (int l = 0; l < FM_MAX_ECHO; ++l) a.te[l] = l < c->L ? c->te[l] : 0.0;
    for (int l = 0; l < FM_MAX_ECHO; ++l) { a.fat_re[l] = c->fat_re[l]; a.fat_im[l] = c->fat_im[l]; }
    for (int k = 0; k < 8; ++k) a.ginv[k] = c->ginv[k];
    a.rho = c->rho;
    a.pairs = c->pairs;
    a.nb = c->nb;
    a.vlist = c->vlist;
    a.scal = c->scal;
    a.partials = c->partials;
    a.istate = c->istate;
    return a;
}

constexpr int kCgPerGraph = 8;  // CG iterations per graph replay (even: the p buffers ping-pong)

// Buffers of the adjoint CG (the solver's, which fm_solve re-initialises): x = w[0],
// r = g[0], z = p, p ping-pong = z[0] / z[1], q = g[1], h = w[1].
template <typename T>
cudaError_t cg_iteration(fm_ctx* c, double tol2, int maxiter, int par) {
    AdjArgs a = adj_args(c);
    a.tol2 = tol2;
    a.maxiter = maxiter;
    a.x = c->w[0];
    a.r = c->g[0];
    a.z = c->p;
    a.p_old = c->z[par];
    a.p_new = c->z[par ^ 1];
    a.q = c->g[1];
    a.h = c->w[1];
    cudaError_t e = launch_cg_dir<T>(a, c->grid_data, c->stream);
    if (e == cudaSuccess) e = launch_cg_upd<T>(a, c->grid_data, c->stream);
    if (e == cudaSuccess) e = run_ic<T>(c, nullptr, c->g[0], c->p, c->g[0], nullptr);
    return e;
}

template <typename T>
int adjoint_t(fm_ctx* c, const void* w_hat, const void* rhs, void* lambda, double tol, int maxiter, int* iters,
              double* relres) {
    cudaStream_t s = c->stream;
    const size_t vb = (size_t)c->nv * c->ts;
    const double tol2 = tol * tol;
    FM_CK(reset_barrier(c), "reset");
    // majoriser curvature d(w_hat) for the preconditioner (Eq. 9-12)
    FM_CK(run_grad<T>(c, w_hat, nullptr, c->w[1], c->g[1], c->d, nullptr), "curvature");
    void* zero[] = {c->w[0], c->g[0], c->z[0], c->z[1], c->g[1]};
    for (void* b : zero) FM_CK(cudaMemsetAsync(b, 0, vb, s), "clear CG vectors");
    AdjArgs a = adj_args(c);
    a.w = w_hat;
    a.rhs = rhs;
    a.h = c->w[1];
    a.r = c->g[0];
    a.maxiter = maxiter;
    a.tol2 = tol2;
    FM_CK(launch_cg_init<T>(a, c->grid_data, s), "CG start");
    FM_CK(run_ic<T>(c, c->d, c->g[0], c->p, c->g[0], nullptr), "IC(0) factor");  // z_0 and r_0'z_0
    c->have_factor = true;
    if (c->cg_gexec && (c->cg_tol2 != tol2 || c->cg_maxiter != maxiter)) {
        cudaGraphExecDestroy(c->cg_gexec);
        c->cg_gexec = nullptr;
    }
    if (c->o.use_graph && !c->cg_gexec) {
        cudaGraph_t graph = nullptr;
        FM_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < kCgPerGraph && e == cudaSuccess; ++i) e = cg_iteration<T>(c, tol2, maxiter, i & 1);
        cudaError_t ee = cudaStreamEndCapture(s, &graph);
        if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(c, e, "capture CG"); }
        FM_CK(ee, "end capture");
        cudaError_t ei = cudaGraphInstantiate(&c->cg_gexec, graph, 0);
        cudaGraphDestroy(graph);
        FM_CK(ei, "instantiate graph");
        c->cg_tol2 = tol2;
        c->cg_maxiter = maxiter;
    }
    // every batch of kCgPerGraph iterations ends with a look at the device stop flag; the
    // kernels themselves stop at convergence or at maxiter
    const int nbatch = (maxiter + kCgPerGraph - 1) / kCgPerGraph;
    for (int k = 0; k < nbatch; ++k) {
        int st[2] = {0, 0};
        FM_CK(cudaMemcpyAsync(st, c->istate + I_CG_IT, 2 * sizeof(int), cudaMemcpyDeviceToHost, s), "read state");
        FM_CK(cudaStreamSynchronize(s), "synchronise");
        if (st[1] != 0) break;
        if (c->cg_gexec) {
            FM_CK(cudaGraphLaunch(c->cg_gexec, s), "launch CG graph");
        } else {
            for (int i = 0; i < kCgPerGraph; ++i) FM_CK(cg_iteration<T>(c, tol2, maxiter, i & 1), "CG iteration");
        }
    }
    FM_CK(cudaMemcpyAsync(lambda, c->w[0], vb, cudaMemcpyDeviceToDevice, s), "copy lambda");
    int it = 0;
    double sc[2] = {0.0, 0.0};
    FM_CK(cudaMemcpyAsync(&it, c->istate + I_CG_IT, sizeof(int), cudaMemcpyDeviceToHost, s), "read state");
    FM_CK(cudaMemcpyAsync(sc, c->scal + S_CG_RR, 2 * sizeof(double), cudaMemcpyDeviceToHost, s), "read state");
    int rc = check_dev(c);
    if (iters) *iters = it;
    if (relres) *relres = sc[1] > 0.0 ? std::sqrt(sc[0] / sc[1]) : 0.0;
    return rc;
}

template <typename T>
int implicit_t(fm_ctx* c, const void* y, const void* smap, const void* w_hat, const void* lam, void* dl_dy,
               double* dl_dbeta) {
    AdjArgs a = adj_args(c);
    a.w = w_hat;
    a.lam = lam;
    a.y = y;
    a.smap = smap;
    a.dldy = dl_dy;
    FM_CK(reset_barrier(c), "reset");
    if (dl_dy) FM_CK(launch_dldy<T>(a, c->grid_data, c->stream), "image derivative kernel");
    if (dl_dbeta) {
        FM_CK(launch_lap_dot<T>(a, c->grid_data, c->stream), "beta derivative kernel");
        double dot = 0.0;
        FM_CK(cudaMemcpyAsync(&dot, c->scal + S_ADJ_DOT, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
              "copy");
        int rc = check_dev(c);
        if (rc != FM_OK) return rc;
        *dl_dbeta = -dot;
    }
    return FM_OK;
}

#ifndef FM_IC_BXY
#define FM_IC_BXY 2
#endif
#ifndef FM_IC_BBLK
#define FM_IC_BBLK 2
#endif
#ifndef FM_IC_BZ
#define FM_IC_BZ 1
#endif

// Tile claim orders: a weighted tile hyperplane wxy (X + Y) + wz Z (ties: z, y, x).  Every
// weight is positive, so a tile's -x, -y, -z neighbours always come first.  Both sweeps
// stream faces, and a tile starts about 38 steps plus one hand-off behind its x / y
// predecessors and 14 steps plus one hand-off behind its z predecessor, so the forward order
// takes wxy : wz (default 2 : 1) and the back substitution walks FM_IC_BXY : FM_IC_BZ
// (2 : 1; measured on the 256 x 256 x 128 volume against 1 : 1 and 3 : 2) backwards.
// Uploads both orders synchronously.
bool set_ic_order(fm_ctx* c, int wxy, int wz) {
    std::vector<int> ord(2 * (size_t)c->ntiles);
    const int ntx = c->ntx, nty = c->nty;
    for (int pass = 0; pass < 2; ++pass) {
        const int a_xy = pass == 0 ? wxy : FM_IC_BXY, a_z = pass == 0 ? wz : FM_IC_BZ;
        auto first = ord.begin() + (size_t)pass * c->ntiles;
        for (int t = 0; t < c->ntiles; ++t) first[t] = t;
        std::stable_sort(first, first + c->ntiles, [&](int a, int b) {
            const int ha = a_xy * (a % ntx + (a / ntx) % nty) + a_z * (a / (ntx * nty));
            const int hb = a_xy * (b % ntx + (b / ntx) % nty) + a_z * (b / (ntx * nty));
            return ha != hb ? ha < hb : a < b;
        });
    }
    c->ic_wxy = wxy;
    c->ic_wz = wz;
    return cudaMemcpy(c->order, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
}

// Cooperative line-search grid: every block must be co-resident, so the grid follows the
// occupancy of the kernel variant the context launches.
template <typename T>
int pwls_t(fm_ctx* c, const void* wt, int niter, void* w0) {
    cudaStream_t s = c->stream;
    const size_t vb = (size_t)c->nv * c->ts;
    FM_CK(reset_barrier(c), "reset");
    void* zero[] = {c->w[0], c->g[0], c->z[0], c->z[1], c->g[1]};
    for (void* b : zero) FM_CK(cudaMemsetAsync(b, 0, vb, s), "clear CG vectors");
    AdjArgs a = adj_args(c);
    a.x0 = wt;
    a.h = c->w[1];
    a.x = c->w[0];
    a.r = c->g[0];
    a.z = c->g[0];  // no preconditioner: z = r
    a.q = c->g[1];
    a.maxiter = niter;
    a.tol2 = 0.0;   // a fixed number of iterations (stops early only at r = 0)
    a.identity_pc = 1;
    FM_CK(launch_pwls_init<T>(a, c->grid_data, s), "PWLS start");
    for (int i = 0; i < niter; ++i) {
        a.p_old = c->z[i & 1];
        a.p_new = c->z[(i & 1) ^ 1];
        FM_CK(launch_cg_dir<T>(a, c->grid_data, s), "PWLS direction");
        FM_CK(launch_cg_upd<T>(a, c->grid_data, s), "PWLS update");
    }
    FM_CK(cudaMemcpyAsync(w0, c->w[0], vb, cudaMemcpyDeviceToDevice, s), "copy omega");
    return check_dev(c);
}

bool set_ls_grid(fm_ctx* c) {
    DataArgs probe{};
    probe.nc = c->nc;
    probe.literal = c->literal;
    probe.wf = c->wf;
    const int occ = c->o.precision == FM_FP64 ? ls_max_blocks_per_sm<double>(probe) : ls_max_blocks_per_sm<float>(probe);
    if (occ < 1) return false;
    const long long nblk = (c->nv + kThreads - 1) / kThreads;
    c->grid_ls = (int)std::max(1LL, std::min<long long>(nblk, (long long)occ * c->nsm));
    c->base_ls = c->grid_ls;
    return true;
}

bool valid_opts(const fm_opts& o) {
    return (o.precision == FM_FP32 || o.precision == FM_FP64) && o.nls >= 1 && o.nls <= 1000 &&
           (o.precond == FM_PC_IC0 || o.precond == FM_PC_DIAG || o.precond == FM_PC_NONE || o.precond == FM_PC_RB ||
            o.precond == FM_PC_ICT) &&
           (o.curvature == FM_CURV_LITERAL || o.curvature == FM_CURV_COMBINED) && o.spin_limit >= 1 &&
           (o.precond != FM_PC_ICT || (std::isfinite(o.droptol) && o.droptol >= 0.0));
}

}  // namespace

extern "C" {

void fm_default_opts(fm_opts* o) {
    if (!o) return;
    o->precision = FM_FP32;
    o->nls = 5;
    o->precond = FM_PC_IC0;
    o->curvature = FM_CURV_LITERAL;
    o->spin_limit = 1LL << 21;
    o->use_graph = 1;
    o->droptol = 1e-3;
}

const char* fm_strerror(int s) {
    switch (s) {
        case FM_OK: return "ok";
        case FM_ERR_ARG: return "invalid argument";
        case FM_ERR_STATE: return "call order: required earlier call missing";
        case FM_ERR_CUDA: return "CUDA error";
        case FM_ERR_NOT_PD: return "IC(0) pivot not positive";
        case FM_ERR_TIMEOUT: return "device-side wait timed out";
        case FM_ERR_NONFINITE: return "non-finite reduction";
        case FM_ERR_OOM: return "out of memory";
        case FM_ERR_SIZE: return "problem exceeds a fixed-size buffer of the call";
        case FM_ERR_FILL: return "drop tolerance keeps fill-in beyond level 1 (FM_PC_ICT's held pattern)";
        default: return "unknown status";
    }
}

const char* fm_last_error(const fm_ctx* c) { return c ? c->err.c_str() : ""; }

int fm_create(fm_ctx** out, int nx, int ny, int nz, int ncoil, int necho, const fm_opts* opts, int device,
              void* cuda_stream) {
    if (!out) return FM_ERR_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || ncoil < 1 || ncoil > FM_MAX_COIL || necho < 2 || necho > FM_MAX_ECHO)
        return FM_ERR_ARG;
    if ((long long)nx * ny * nz >= (1LL << 31)) return FM_ERR_ARG;  // voxel indices are 32-bit
    fm_opts o;
    fm_default_opts(&o);
    if (opts) o = *opts;
    if (!valid_opts(o)) return FM_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FM_ERR_CUDA;
    fm_ctx* c = new (std::nothrow) fm_ctx();
    if (!c) return FM_ERR_OOM;
    DevGuard guard(device);
    c->nx = nx; c->ny = ny; c->nz = nz; c->nc = ncoil; c->L = necho;
    c->nv = (long long)nx * ny * nz;
    c->o = o;
    c->device = device;
    c->ts = o.precision == FM_FP64 ? 8 : 4;
    c->literal = (ncoil > 1 && o.curvature == FM_CURV_LITERAL);
    auto bail = [&](int code) { free_all(c); delete c; return code; };
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreate(&c->stream) != cudaSuccess) return bail(FM_ERR_CUDA);
        c->own_stream = true;
    }
    if (cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return bail(FM_ERR_CUDA);
    const long long nblk = (c->nv + kThreads - 1) / kThreads;
    c->grid_data = (int)std::max(1LL, std::min<long long>(nblk, 4LL * c->nsm));
    if (!set_ls_grid(c)) return bail(FM_ERR_CUDA);
    c->ntx = (nx + kTileX - 1) / kTileX;
    c->nty = (ny + kTileY - 1) / kTileY;
    const int tz = o.precision == FM_FP64 ? ic_tz<double>() : ic_tz<float>();
    c->ntz = (nz + tz - 1) / tz;
    c->ntiles = c->ntx * c->nty * c->ntz;
    {
        // the two sweeps claim tiles from their own tickets, so each sizes its own grid: the
        // forward sweep by its footprint (1 block/SM), the back substitution by its footprint
        // capped at 2 blocks/SM -- a third block per SM only adds tiles waiting on their
        // successors' flags (256x256x128 volume: 0.328 / 0.284 / 0.293 ms per sweep at 1 / 2 / 3)
        const bool f64 = o.precision == FM_FP64;
        const int occ_f = f64 ? ic_max_blocks_per_sm<double>(false) : ic_max_blocks_per_sm<float>(false);
        const int occ_b = f64 ? ic_max_blocks_per_sm<double>(true) : ic_max_blocks_per_sm<float>(true);
        if (occ_f < 1 || occ_b < 1) return bail(FM_ERR_CUDA);
        c->grid_ic = std::max(1, std::min(c->ntiles, occ_f * c->nsm));
        c->grid_icb = std::max(1, std::min(c->ntiles, std::min(occ_b, FM_IC_BBLK) * c->nsm));
        c->occ_icb = occ_b;
    }
    c->base_data = c->grid_data;
    c->base_ls = c->grid_ls;
    c->base_ic = c->grid_ic;
    c->base_icb = c->grid_icb;
    if (o.precond == FM_PC_ICT) {
        // one thread per (y, z) column of the level sweep, the columns spread over every SM
        // (the sweeps are bound by FP64 issue), every block resident (grid barrier)
        const long long cols = (long long)ny * nz;
        const long long per_sm = (cols + c->nsm - 1) / c->nsm;
        c->block_ict = (int)std::min<long long>(kIctThreads, std::max<long long>(32, (per_sm + 31) / 32 * 32));
        const int occ = o.precision == FM_FP64 ? ict_max_blocks_per_sm<double>(c->block_ict)
                                               : ict_max_blocks_per_sm<float>(c->block_ict);
        if (occ < 1) return bail(FM_ERR_CUDA);
        c->grid_ict = (int)std::max(1LL, std::min<long long>((cols + c->block_ict - 1) / c->block_ict,
                                                             (long long)occ * c->nsm));
        c->base_ict = c->grid_ict;
        const int occg = o.precision == FM_FP64 ? ictg_max_blocks_per_sm<double>(c->block_ict)
                                                : ictg_max_blocks_per_sm<float>(c->block_ict);
        if (occg < 1) return bail(FM_ERR_CUDA);
        c->grid_ictg = (int)std::max(1LL, std::min<long long>((cols + c->block_ict - 1) / c->block_ict,
                                                              (long long)occg * c->nsm));
        c->base_ictg = c->grid_ictg;
    }
    const size_t vb = (size_t)c->nv * c->ts;
    const int P = necho * (necho - 1) / 2;
    bool ok = true;
    auto A = [&](auto** ptr, size_t bytes) { if (ok && dalloc(ptr, bytes) != cudaSuccess) ok = false; };
    A(&c->pairs, (size_t)P * 2 * vb);
    if (c->literal) A(&c->coils, (size_t)necho * ncoil * 2 * vb);
    A(&c->nb, (size_t)c->nv);
    const long long nchunks = (c->nv + kChunk - 1) / kChunk;
    A(&c->vlist, (size_t)c->nv * sizeof(int));
    A(&c->chunk_off, (size_t)nchunks * sizeof(int));
    A(&c->w0, vb);
    for (int k = 0; k < 2; ++k) { A(&c->w[k], vb); A(&c->z[k], vb); A(&c->g[k], vb); }
    A(&c->d, vb); A(&c->p, vb); A(&c->v, vb); A(&c->ip, vb); A(&c->rho, vb);
    A(&c->scal, S_NSCAL * sizeof(double));
    A(&c->partials, std::max<size_t>(8 * (size_t)std::max(c->grid_data, c->grid_ls), nchunks) * sizeof(double));
    c->face_bytes = (size_t)c->ntiles *
                    (o.precision == FM_FP64 ? ic_face_bytes_per_tile<double>() : ic_face_bytes_per_tile<float>());
    A(&c->face, c->face_bytes);
    A(&c->tile_part, 2 * (size_t)c->ntiles * sizeof(double));
    A(&c->istate, I_NISTATE * sizeof(int));
    A(&c->icint, 4 * sizeof(int));
    A(&c->order, 2 * (size_t)c->ntiles * sizeof(int));  // forward order, then the back substitution's

    if (!ok) { cudaGetLastError(); return bail(FM_ERR_OOM); }
#ifndef FM_IC_WXY
#define FM_IC_WXY 2
#endif
#ifndef FM_IC_WZ
#define FM_IC_WZ 1
#endif
    if (o.precond == FM_PC_ICT) {  // IC(0)'s offsets and the level-1 fill offsets, in plane order
        c->ict_off = {-1, 0, 0, 0, -1, 0, 0, 0, -1, 1, -1, 0, 1, 0, -1, 0, 1, -1};
        if (ict_build(c) != FM_OK) return bail(FM_ERR_OOM);
    }
    if (!set_ic_order(c, FM_IC_WXY, FM_IC_WZ) ||
        cudaMemset(c->scal, 0, S_NSCAL * sizeof(double)) != cudaSuccess ||
        cudaMemset(c->istate, 0, I_NISTATE * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->nb, 0, (size_t)c->nv) != cudaSuccess ||
        cudaMemset(c->face, 0xff, c->face_bytes) != cudaSuccess)  // forward faces start unset
        return bail(FM_ERR_CUDA);
    *out = c;
    return FM_OK;
}

int fm_destroy(fm_ctx* c) {
    if (!c) return FM_OK;
    {
        DevGuard guard(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        free_all(c);
    }
    delete c;
    return FM_OK;
}

int fm_set_data(fm_ctx* c, const void* y, const void* smap, const double* te, const uint8_t* mask, double beta) {
    if (!c) return FM_ERR_ARG;
    if (!y || !te) return fail(c, FM_ERR_ARG, "y and te are required");
    if (!smap && c->nc != 1) return fail(c, FM_ERR_ARG, "smap may be NULL only with one coil");
    if (!(beta >= 0.0) || !std::isfinite(beta)) return fail(c, FM_ERR_ARG, "beta must be finite and >= 0");
    for (int l = 0; l < c->L; ++l)
        if (!std::isfinite(te[l])) return fail(c, FM_ERR_ARG, "echo times must be finite");
    if (te[1] == te[0]) return fail(c, FM_ERR_ARG, "t_2 == t_1 (Eq. 6 divides by t_2 - t_1)");
    DevGuard guard(c->device);
    const double old_beta = c->beta;
    c->beta = beta;
    for (int l = 0; l < c->L; ++l) c->te[l] = te[l];
    // Eq. gamma: Gamma = 1/L, or gamma (gamma^H gamma)^{-1} gamma^H with gamma = [1, phi]
    std::vector<std::complex<double>> lgam((size_t)c->L * c->L, std::complex<double>(1.0, 0.0));
    if (c->wf) {
        using cd = std::complex<double>;
        std::vector<cd> phi(c->L);
        for (int l = 0; l < c->L; ++l) {
            cd acc(0.0, 0.0);
            for (size_t q = 0; q < c->fat_amp.size(); ++q)
                acc += c->fat_amp[q] * std::polar(1.0, 6.283185307179586476925286766559 * c->fat_freq[q] * te[l]);
            phi[l] = acc;
            c->fat_re[l] = acc.real();
            c->fat_im[l] = acc.imag();
        }
        cd g01(0.0, 0.0);
        double g11 = 0.0;
        for (int l = 0; l < c->L; ++l) {
            g01 += phi[l];
            g11 += std::norm(phi[l]);
        }
        const double g00 = (double)c->L, det = g00 * g11 - std::norm(g01);
        if (!(det > 1e-12 * g00 * g11)) return fail(c, FM_ERR_ARG, "fat basis is collinear with water at these echo times");
        const cd i00 = g11 / det, i01 = -g01 / det, i10 = -std::conj(g01) / det, i11 = g00 / det;
        const cd gi[4] = {i00, i01, i10, i11};
        for (int k = 0; k < 4; ++k) { c->ginv[2 * k] = gi[k].real(); c->ginv[2 * k + 1] = gi[k].imag(); }
        for (int m = 0; m < c->L; ++m)
            for (int n = 0; n < c->L; ++n) {
                // Gamma_mn = sum_{k,k'} gamma_mk Ginv_kk' conj(gamma_nk'), gamma_l0 = 1, gamma_l1 = phi_l
                const cd gm[2] = {cd(1.0, 0.0), phi[m]}, gn[2] = {cd(1.0, 0.0), phi[n]};
                cd acc(0.0, 0.0);
                for (int k = 0; k < 2; ++k)
                    for (int kk = 0; kk < 2; ++kk) acc += gm[k] * gi[2 * k + kk] * std::conj(gn[kk]);
                lgam[(size_t)m * c->L + n] = (double)c->L * acc;
            }
    }
    Pairs pr{};
    for (int m = 0; m < c->L; ++m)
        for (int n = m + 1; n < c->L; ++n) {
            pr.m[pr.P] = m;
            pr.n[pr.P] = n;
            pr.dt[pr.P] = te[m] - te[n];
            pr.dtt[pr.P] = (float)(pr.dt[pr.P] * 683565275.57643158);  // 2^32 / (2 pi)
            pr.gmag[pr.P] = std::abs(lgam[(size_t)m * c->L + n]);
            pr.gph[pr.P] = c->wf ? std::arg(lgam[(size_t)m * c->L + n]) : 0.0;
            ++pr.P;
        }
    // beta and the pair constants are kernel arguments of the captured graphs: keep the
    // graphs only when they are unchanged (every buffer the graphs use belongs to the context)
    bool same = c->have_data && beta == old_beta && pr.P == c->pr.P;
    for (int q = 0; same && q < pr.P; ++q)
        same = pr.m[q] == c->pr.m[q] && pr.n[q] == c->pr.n[q] && pr.dt[q] == c->pr.dt[q] &&
               pr.gmag[q] == c->pr.gmag[q] && pr.gph[q] == c->pr.gph[q];
    c->pr = pr;
    if (!same) {
        if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
        if (c->cg_gexec) { cudaGraphExecDestroy(c->cg_gexec); c->cg_gexec = nullptr; }
    }
    SetupArgs a{};
    a.geo = Geo{c->nx, c->ny, c->nz, c->nv};
    a.nc = c->nc;
    a.L = c->L;
    a.pr = pr;
    a.y = y;
    a.smap = smap;
    a.mask = mask;
    a.te0 = te[0];
    a.te1 = te[1];
    a.wf = c->wf ? 1 : 0;
    for (int m = 0; m < c->L; ++m)
        for (int n = 0; n < c->L; ++n) {
            a.lgam[2 * (m * c->L + n)] = lgam[(size_t)m * c->L + n].real();
            a.lgam[2 * (m * c->L + n) + 1] = lgam[(size_t)m * c->L + n].imag();
        }
    a.rho = c->rho;
    a.pairs = c->pairs;
    a.coils = c->coils;
    a.nb = c->nb;
    a.w0 = c->w0;
    a.vlist = c->vlist;
    a.chunk_off = c->chunk_off;
    a.partials = c->partials;
    a.scal = c->scal;
    a.istate = c->istate;
    cudaError_t e = c->o.precision == FM_FP64 ? launch_setup<double>(a, c->stream)
                                              : launch_setup<float>(a, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "setup kernel");
    // rows outside the new mask must read as empty in the drop-tolerance factor
    if (c->ict_L)
        FM_CK(cudaMemsetAsync(c->ict_L, 0, (size_t)c->ict_nplanes * c->nv * sizeof(double), c->stream), "clear factor");
    c->have_data = true;
    c->have_factor = false;
    return FM_OK;
}

int fm_init_omega(fm_ctx* c, void* omega) {
    if (!c) return FM_ERR_ARG;
    if (!omega) return fail(c, FM_ERR_ARG, "omega is required");
    if (!c->have_data) return fail(c, FM_ERR_STATE, "fm_set_data first");
    DevGuard guard(c->device);
    FM_CK(cudaMemcpyAsync(omega, c->w0, (size_t)c->nv * c->ts, cudaMemcpyDeviceToDevice, c->stream), "copy");
    return FM_OK;
}

int fm_cost_grad(fm_ctx* c, const void* omega, double* cost, void* grad, void* curv) {
    if (!c) return FM_ERR_ARG;
    if (!omega) return fail(c, FM_ERR_ARG, "omega is required");
    if (!c->have_data) return fail(c, FM_ERR_STATE, "fm_set_data first");
    DevGuard guard(c->device);
    void* g = grad ? grad : c->g[0];
    void* d = curv ? curv : c->d;
    const size_t vb = (size_t)c->nv * c->ts;
    FM_CK(cudaMemsetAsync(g, 0, vb, c->stream), "clear gradient");  // entries outside the mask stay 0
    FM_CK(cudaMemsetAsync(d, 0, vb, c->stream), "clear curvature");
    cudaError_t e = c->o.precision == FM_FP64
                        ? run_grad<double>(c, omega, nullptr, c->w[0], g, d, nullptr)
                        : run_grad<float>(c, omega, nullptr, c->w[0], g, d, nullptr);
    if (e != cudaSuccess) return cuda_fail(c, e, "gradient kernel");
    if (cost) {
        FM_CK(cudaMemcpyAsync(cost, c->scal + S_COST, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy cost");
        return check_dev(c);
    }
    return FM_OK;
}

// The preconditioner factor of H = diag(d) + beta C'C with d already in c->d (Eq. 9, 12).
int ic_factor_from_d(fm_ctx* c, void* inv_pivot) {
    const bool f64 = c->o.precision == FM_FP64;
    cudaError_t e;
    if (c->o.precond == FM_PC_RB) {  // red-black pivots of both colours
        DataArgs a = base_args(c);
        a.d = c->d;
        a.g = c->g[0];
        a.z_new = c->p;
        a.ip_out = c->ip;
        FM_CK(cudaMemsetAsync(c->ip, 0, (size_t)c->nv * c->ts, c->stream), "clear pivots");
        e = f64 ? launch_rb_black<double>(a, c->grid_data, c->stream) : launch_rb_black<float>(a, c->grid_data, c->stream);
    } else {
        e = f64 ? run_ic<double>(c, c->d, c->g[0], c->p, nullptr, nullptr)
                : run_ic<float>(c, c->d, c->g[0], c->p, nullptr, nullptr);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "IC(0) kernels");
    if (c->o.precond == FM_PC_ICT) {  // grow the held pattern until the factor is exact (synchronous)
        for (int round = 0;; ++round) {
            const int rc = check_dev(c);
            if (rc != FM_ERR_FILL || round >= kIctMaxRounds) {
                if (rc != FM_OK) return rc;
                break;
            }
            const int g = ict_grow(c);
            if (g <= 0) return g < 0 ? g : rc;
            e = f64 ? run_ic<double>(c, c->d, c->g[0], c->p, nullptr, nullptr)
                    : run_ic<float>(c, c->d, c->g[0], c->p, nullptr, nullptr);
            if (e != cudaSuccess) return cuda_fail(c, e, "IC kernels");
        }
    }
    if (inv_pivot)
        FM_CK(cudaMemcpyAsync(inv_pivot, c->ip, (size_t)c->nv * c->ts, cudaMemcpyDeviceToDevice, c->stream), "copy");
    c->have_factor = true;
    return FM_OK;
}

int fm_ic_factor(fm_ctx* c, const void* omega, void* inv_pivot) {
    if (!c) return FM_ERR_ARG;
    if (!omega) return fail(c, FM_ERR_ARG, "omega is required");
    if (!c->have_data) return fail(c, FM_ERR_STATE, "fm_set_data first");
    DevGuard guard(c->device);
    FM_CK(reset_barrier(c), "reset barrier");
    cudaError_t e = c->o.precision == FM_FP64 ? run_grad<double>(c, omega, nullptr, c->w[0], c->g[0], c->d, nullptr)
                                              : run_grad<float>(c, omega, nullptr, c->w[0], c->g[0], c->d, nullptr);
    if (e != cudaSuccess) return cuda_fail(c, e, "gradient kernel");
    return ic_factor_from_d(c, inv_pivot);
}

int fm_ic_factor_curv(fm_ctx* c, const void* curv, void* inv_pivot) {
    if (!c) return FM_ERR_ARG;
    if (!curv) return fail(c, FM_ERR_ARG, "curv is required");
    if (!c->have_data) return fail(c, FM_ERR_STATE, "fm_set_data first");
    DevGuard guard(c->device);
    FM_CK(reset_barrier(c), "reset barrier");
    const size_t vb = (size_t)c->nv * c->ts;
    // only mask voxels are read by the factor kernels
    FM_CK(cudaMemcpyAsync(c->d, curv, vb, cudaMemcpyDeviceToDevice, c->stream), "copy curvature");
    FM_CK(cudaMemsetAsync(c->g[0], 0, vb, c->stream), "clear");
    return ic_factor_from_d(c, inv_pivot);
}

int fm_ict_pattern(fm_ctx* c, int* n_offsets, int* offsets, double* planes) {
    if (!c || !n_offsets) return FM_ERR_ARG;
    if (c->o.precond != FM_PC_ICT) return fail(c, FM_ERR_STATE, "fm_ict_pattern is for FM_PC_ICT");
    DevGuard guard(c->device);
    const int nh = c->ict_tb.nh;
    *n_offsets = nh;
    if (offsets) std::memcpy(offsets, c->ict_off.data(), 3 * (size_t)nh * sizeof(int));
    if (planes) {
        if (!c->have_factor) return fail(c, FM_ERR_STATE, "fm_ic_factor first");
        FM_CK(cudaStreamSynchronize(c->stream), "synchronise");
        FM_CK(cudaMemcpy(planes, c->ict_L, (size_t)(nh + 1) * c->nv * sizeof(double), cudaMemcpyDeviceToHost),
              "copy factor");
    }
    return FM_OK;
}

int fm_ic_factor64(fm_ctx* c, const void* omega, double* inv_pivot) {
    if (!c) return FM_ERR_ARG;
    if (!omega || !inv_pivot) return fail(c, FM_ERR_ARG, "omega and inv_pivot are required");
    if (!c->have_data) return fail(c, FM_ERR_STATE, "fm_set_data first");
    if (c->o.precond != FM_PC_IC0) return fail(c, FM_ERR_STATE, "fm_ic_factor64 is for the IC(0) preconditioner");
    if (c->o.precision == FM_FP64) return fm_ic_factor(c, omega, inv_pivot);
    DevGuard guard(c->device);
    if (!c->ip_lo && dalloc(&c->ip_lo, (size_t)c->nv * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, FM_ERR_OOM, "allocate pivot buffer");
    }
    FM_CK(reset_barrier(c), "reset barrier");
    FM_CK(run_grad<float>(c, omega, nullptr, c->w[0], c->g[0], c->d, nullptr), "gradient kernel");
    FM_CK(cudaMemsetAsync(c->ip_lo, 0, (size_t)c->nv * sizeof(float), c->stream), "clear");
    FM_CK(run_ic0<float>(c, c->d, c->g[0], c->p, nullptr, nullptr, -1, c->ip_lo), "IC(0) kernels");
    FM_CK(launch_inv_pivot64((const float*)c->ip, c->ip_lo, inv_pivot, c->nv, c->grid_data, c->stream), "combine");
    c->have_factor = true;
    return FM_OK;
}

int fm_ic_apply(fm_ctx* c, const void* g, void* p) {
    if (!c) return FM_ERR_ARG;
    if (!g || !p || g == p) return fail(c, FM_ERR_ARG, "g and p must be distinct device arrays");
    if (!c->have_factor) return fail(c, FM_ERR_STATE, "fm_ic_factor first");
    DevGuard guard(c->device);
    FM_CK(reset_barrier(c), "reset barrier");
    cudaError_t e;
    if (c->o.precond == FM_PC_RB) {
        DataArgs a = base_args(c);
        a.g = const_cast<void*>(g);  // read only here
        a.z_new = p;
        a.ip_in = c->ip;
        const bool f64 = c->o.precision == FM_FP64;
        FM_CK(cudaMemsetAsync(p, 0, (size_t)c->nv * c->ts, c->stream), "clear");
        e = f64 ? launch_rb_black<double>(a, c->grid_data, c->stream) : launch_rb_black<float>(a, c->grid_data, c->stream);
        if (e == cudaSuccess)
            e = f64 ? launch_rb_red<double>(a, c->grid_data, c->stream) : launch_rb_red<float>(a, c->grid_data, c->stream);
    } else {
        e = c->o.precision == FM_FP64 ? run_ic<double>(c, nullptr, g, p, nullptr, nullptr)
                                      : run_ic<float>(c, nullptr, g, p, nullptr, nullptr);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "IC(0) kernels");
    return FM_OK;
}

int fm_solve(fm_ctx* c, void* omega, int init_from_data, int niter, double* cost_hist) {
    if (!c) return FM_ERR_ARG;
    if (!omega) return fail(c, FM_ERR_ARG, "omega is required");
    if (niter < 0) return fail(c, FM_ERR_ARG, "niter must be >= 0");
    if (!c->have_data) return fail(c, FM_ERR_STATE, "fm_set_data first");
    DevGuard guard(c->device);
    c->have_factor = false;  // the solve reuses the factor buffers
    return c->o.precision == FM_FP64 ? solve_t<double>(c, omega, init_from_data, niter, cost_hist)
                                     : solve_t<float>(c, omega, init_from_data, niter, cost_hist);
}

int fm_set_data_host(fm_ctx* c, const void* y, const void* smap, const double* te, const uint8_t* mask,
                     double beta) {
    if (!c) return FM_ERR_ARG;
    if (!y || !te) return fail(c, FM_ERR_ARG, "y and te are required");
    if (!smap && c->nc != 1) return fail(c, FM_ERR_ARG, "smap may be NULL only with one coil");
    if (!(beta >= 0.0) || !std::isfinite(beta)) return fail(c, FM_ERR_ARG, "beta must be finite and >= 0");
    for (int l = 0; l < c->L; ++l)
        if (!std::isfinite(te[l])) return fail(c, FM_ERR_ARG, "echo times must be finite");
    if (te[1] == te[0]) return fail(c, FM_ERR_ARG, "t_2 == t_1 (Eq. 6 divides by t_2 - t_1)");
    DevGuard guard(c->device);
    const size_t cb = 2 * c->ts;  // one complex value
    const size_t yb = (size_t)c->L * c->nc * c->nv * cb, sb = (size_t)c->nc * c->nv * cb, mb = (size_t)c->nv;
    if (!c->copy_stream) {
        FM_CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "create copy stream");
        for (int k = 0; k < 2; ++k) {
            FM_CK(cudaEventCreateWithFlags(&c->ev_copied[k], cudaEventDisableTiming), "create event");
            FM_CK(cudaEventCreateWithFlags(&c->ev_read[k], cudaEventDisableTiming), "create event");
        }
    }
    const int k = c->st_next;
    if (!c->st_y[k]) {
        bool ok = dalloc(&c->st_y[k], yb) == cudaSuccess && dalloc(&c->st_s[k], sb) == cudaSuccess &&
                  dalloc(&c->st_m[k], mb) == cudaSuccess;
        if (!ok) { cudaGetLastError(); return fail(c, FM_ERR_OOM, "allocate staging buffers"); }
    }
    c->st_next ^= 1;
    cudaStream_t cs = c->copy_stream;
    // the precompute that last read this staging set must be done before it is overwritten
    FM_CK(cudaStreamWaitEvent(cs, c->ev_read[k], 0), "order copy");
    const bool prof = c->profiling && c->ev[k][FM_K_H2D][0];
    if (prof) FM_CK(cudaEventRecord(c->ev[k][FM_K_H2D][0], cs), "record");
    FM_CK(cudaMemcpyAsync(c->st_y[k], y, yb, cudaMemcpyHostToDevice, cs), "copy y");
    if (smap) FM_CK(cudaMemcpyAsync(c->st_s[k], smap, sb, cudaMemcpyHostToDevice, cs), "copy smap");
    if (mask) FM_CK(cudaMemcpyAsync(c->st_m[k], mask, mb, cudaMemcpyHostToDevice, cs), "copy mask");
    if (prof) {
        FM_CK(cudaEventRecord(c->ev[k][FM_K_H2D][1], cs), "record");
        c->ev_rec[k][FM_K_H2D] = true;
    }
    FM_CK(cudaEventRecord(c->ev_copied[k], cs), "record copy");
    FM_CK(cudaStreamWaitEvent(c->stream, c->ev_copied[k], 0), "order precompute");
    const int rc = fm_set_data(c, c->st_y[k], smap ? c->st_s[k] : nullptr, te, mask ? c->st_m[k] : nullptr, beta);
    FM_CK(cudaEventRecord(c->ev_read[k], c->stream), "record precompute");
    return rc;
}

int fm_solve_host(fm_ctx* c, void* omega, int init_from_data, int niter, double* cost_hist) {
    if (!c) return FM_ERR_ARG;
    if (!omega) return fail(c, FM_ERR_ARG, "omega is required");
    if (niter < 0) return fail(c, FM_ERR_ARG, "niter must be >= 0");
    if (!c->have_data) return fail(c, FM_ERR_STATE, "fm_set_data first");
    DevGuard guard(c->device);
    c->have_factor = false;
    return c->o.precision == FM_FP64 ? solve_t<double>(c, omega, init_from_data, niter, cost_hist, true)
                                     : solve_t<float>(c, omega, init_from_data, niter, cost_hist, true);
}

int fm_synchronize(fm_ctx* c) {
    if (!c) return FM_ERR_ARG;
    DevGuard guard(c->device);
    if (c->copy_stream) FM_CK(cudaStreamSynchronize(c->copy_stream), "synchronise copies");
    return check_dev(c);
}

int fm_true_curv(fm_ctx* c, const void* omega, void* h) {
    if (!c) return FM_ERR_ARG;
    if (!omega || !h) return fail(c, FM_ERR_ARG, "omega and h are required");
    if (!c->have_data) return fail(c, FM_ERR_STATE, "fm_set_data first");
    DevGuard guard(c->device);
    FM_CK(cudaMemsetAsync(h, 0, (size_t)c->nv * c->ts, c->stream), "clear");
    AdjArgs a = adj_args(c);
    a.w = omega;
    a.h = h;
    cudaError_t e = c->o.precision == FM_FP64 ? launch_true_curv<double>(a, c->grid_data, c->stream)
                                              : launch_true_curv<float>(a, c->grid_data, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "true curvature kernel");
    return FM_OK;
}

int fm_adjoint_solve(fm_ctx* c, const void* omega_hat, const void* rhs, void* lambda, double tol, int maxiter,
                     int* iters, double* relres) {
    if (!c) return FM_ERR_ARG;
    if (!omega_hat || !rhs || !lambda) return fail(c, FM_ERR_ARG, "omega_hat, rhs and lambda are required");
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(c, FM_ERR_ARG, "tol must be finite and >= 0");
    if (maxiter < 0) return fail(c, FM_ERR_ARG, "maxiter must be >= 0");
    if (!c->have_data) return fail(c, FM_ERR_STATE, "fm_set_data first");
    DevGuard guard(c->device);
    for (int round = 0;; ++round) {  // with the drop-tolerance IC: grow its pattern and solve again
        const int rc = c->o.precision == FM_FP64
                           ? adjoint_t<double>(c, omega_hat, rhs, lambda, tol, maxiter, iters, relres)
                           : adjoint_t<float>(c, omega_hat, rhs, lambda, tol, maxiter, iters, relres);
        if (rc != FM_ERR_FILL || round >= kIctMaxRounds) return rc;
        const int g = ict_grow(c);
        if (g <= 0) return g < 0 ? g : rc;
    }
}

int fm_implicit_grad(fm_ctx* c, const void* y, const void* smap, const void* omega_hat, const void* lambda,
                     void* dl_dy, double* dl_dbeta) {
    if (!c) return FM_ERR_ARG;
    if (!omega_hat || !lambda) return fail(c, FM_ERR_ARG, "omega_hat and lambda are required");
    if (dl_dy && !y) return fail(c, FM_ERR_ARG, "dl_dy needs y");
    if (dl_dy && !smap && c->nc != 1) return fail(c, FM_ERR_ARG, "smap may be NULL only with one coil");
    if (dl_dy && c->wf) return fail(c, FM_ERR_STATE, "dl_dy is implemented for the field-map model only");
    if (!c->have_data) return fail(c, FM_ERR_STATE, "fm_set_data first");
    DevGuard guard(c->device);
    return c->o.precision == FM_FP64 ? implicit_t<double>(c, y, smap, omega_hat, lambda, dl_dy, dl_dbeta)
                                     : implicit_t<float>(c, y, smap, omega_hat, lambda, dl_dy, dl_dbeta);
}

int fm_set_fat_model(fm_ctx* c, int npeak, const double* rel_amp, const double* freq) {
    if (!c) return FM_ERR_ARG;
    if (npeak < 0 || npeak > 64) return fail(c, FM_ERR_ARG, "npeak must be in 0..64");
    if (npeak > 0 && (!rel_amp || !freq)) return fail(c, FM_ERR_ARG, "rel_amp and freq are required");
    for (int q = 0; q < npeak; ++q)
        if (!std::isfinite(rel_amp[q]) || !std::isfinite(freq[q]))
            return fail(c, FM_ERR_ARG, "fat amplitudes and frequencies must be finite");
    DevGuard guard(c->device);
    c->wf = npeak > 0;
    c->fat_amp.assign(rel_amp, rel_amp + npeak);
    c->fat_freq.assign(freq, freq + npeak);
    for (int l = 0; l < FM_MAX_ECHO; ++l) c->fat_re[l] = c->fat_im[l] = 0.0;
    for (double& g : c->ginv) g = 0.0;
    if (!set_ls_grid(c)) return fail(c, FM_ERR_CUDA, "occupancy query");
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    if (c->cg_gexec) { cudaGraphExecDestroy(c->cg_gexec); c->cg_gexec = nullptr; }
    c->have_data = false;  // the pair weights depend on Gamma: fm_set_data again
    c->have_factor = false;
    return FM_OK;
}

int fm_wf_sweep(fm_ctx* c, int nsweep, double w_lo, double w_hi, void* omega_tilde) {
    if (!c) return FM_ERR_ARG;
    if (!omega_tilde) return fail(c, FM_ERR_ARG, "omega_tilde is required");
    if (nsweep < 1 || !std::isfinite(w_lo) || !std::isfinite(w_hi))
        return fail(c, FM_ERR_ARG, "nsweep >= 1 and finite bounds are required");
    if (!c->have_data) return fail(c, FM_ERR_STATE, "fm_set_data first");
    DevGuard guard(c->device);
    FM_CK(cudaMemsetAsync(omega_tilde, 0, (size_t)c->nv * c->ts, c->stream), "clear");
    AdjArgs a = adj_args(c);
    a.x = omega_tilde;
    cudaError_t e = c->o.precision == FM_FP64 ? launch_wf_sweep<double>(a, nsweep, w_lo, w_hi, c->grid_data, c->stream)
                                              : launch_wf_sweep<float>(a, nsweep, w_lo, w_hi, c->grid_data, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "sweep kernel");
    return FM_OK;
}

int fm_wf_sweep_range(const fm_ctx* c, double* w_lo, double* w_hi) {
    if (!c || !w_lo || !w_hi) return FM_ERR_ARG;
    if (!c->wf || c->fat_amp.empty()) return FM_ERR_STATE;
    // reading of Sec. III-A's |Delta_f|: the frequency of the largest-amplitude fat peak (the
    // first one on a tie); the half-width |Delta_f / 2| in cycles is pi |f| in radians
    size_t q = 0;
    for (size_t k = 1; k < c->fat_amp.size(); ++k)
        if (c->fat_amp[k] > c->fat_amp[q]) q = k;
    const double half = 3.14159265358979323846264338327950 * std::fabs(c->fat_freq[q]);
    *w_lo = -half;
    *w_hi = half;
    return FM_OK;
}

int fm_pwls_init(fm_ctx* c, const void* omega_tilde, int niter, void* omega0) {
    if (!c) return FM_ERR_ARG;
    if (!omega_tilde || !omega0) return fail(c, FM_ERR_ARG, "omega_tilde and omega0 are required");
    if (niter < 0) return fail(c, FM_ERR_ARG, "niter must be >= 0");
    if (!c->have_data) return fail(c, FM_ERR_STATE, "fm_set_data first");
    DevGuard guard(c->device);
    c->have_factor = false;  // the solver's work buffers are reused
    return c->o.precision == FM_FP64 ? pwls_t<double>(c, omega_tilde, niter, omega0)
                                     : pwls_t<float>(c, omega_tilde, niter, omega0);
}

int fm_wf_amplitudes(fm_ctx* c, const void* y, const void* smap, const void* omega, void* water, void* fat) {
    if (!c) return FM_ERR_ARG;
    if (!y || !omega || !water || !fat) return fail(c, FM_ERR_ARG, "y, omega, water and fat are required");
    if (!smap && c->nc != 1) return fail(c, FM_ERR_ARG, "smap may be NULL only with one coil");
    if (!c->have_data || !c->wf) return fail(c, FM_ERR_STATE, "fm_set_fat_model and fm_set_data first");
    DevGuard guard(c->device);
    AdjArgs a = adj_args(c);
    a.y = y;
    a.smap = smap;
    a.w = omega;
    a.water = water;
    a.fat = fat;
    cudaError_t e = c->o.precision == FM_FP64 ? launch_wf_amp<double>(a, c->grid_data, c->stream)
                                              : launch_wf_amp<float>(a, c->grid_data, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "amplitude kernel");
    return FM_OK;
}

int fm_set_spin_limit(fm_ctx* c, long long spin_limit) {
    if (!c) return FM_ERR_ARG;
    if (spin_limit < 1) return fail(c, FM_ERR_ARG, "spin_limit must be >= 1");
    DevGuard guard(c->device);
    c->o.spin_limit = spin_limit;
    // the limit is a kernel argument of the captured graphs
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    if (c->cg_gexec) { cudaGraphExecDestroy(c->cg_gexec); c->cg_gexec = nullptr; }
    return FM_OK;
}

int fm_set_profiling(fm_ctx* c, int on) {
    if (!c) return FM_ERR_ARG;
    DevGuard guard(c->device);
    if (on && !c->ev[0][0][0]) {
        for (auto& a : c->ev)
            for (auto& b : a)
                for (cudaEvent_t& e : b) FM_CK(cudaEventCreate(&e), "create event");
    }
    if ((on != 0) != c->profiling && c->gexec) {  // the captured graph holds the event nodes
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    c->profiling = on != 0;
    std::memset(c->ev_rec, 0, sizeof(c->ev_rec));
    return FM_OK;
}

int fm_kernel_times(fm_ctx* c, double* avg_ms, int* count) {
    if (!c || !avg_ms || !count) return FM_ERR_ARG;
    DevGuard guard(c->device);
    FM_CK(cudaStreamSynchronize(c->stream), "synchronise");
    for (int k = 0; k < FM_NKERNEL; ++k) {
        double tot = 0.0;
        int n = 0;
        for (int s = 0; s < 2; ++s) {
            if (!c->ev_rec[s][k]) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c->ev[s][k][0], c->ev[s][k][1]) == cudaSuccess) {
                tot += ms;
                ++n;
            } else {
                cudaGetLastError();
            }
        }
        avg_ms[k] = n ? tot / n : 0.0;
        count[k] = n;
    }
    return FM_OK;
}

int fm_get_history(fm_ctx* c, double* alpha_hist, double* mu_hist, int n) {
    if (!c) return FM_ERR_ARG;
    if (n < 0 || n > c->last_niter) return fail(c, FM_ERR_ARG, "n exceeds the last solve's niter");
    DevGuard guard(c->device);
    if (n == 0) return FM_OK;
    if (alpha_hist)
        FM_CK(cudaMemcpyAsync(alpha_hist, c->hist_alpha, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy");
    if (mu_hist)
        FM_CK(cudaMemcpyAsync(mu_hist, c->hist_mu, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy");
    FM_CK(cudaStreamSynchronize(c->stream), "synchronise");
    return FM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batched form

struct fm_batch {
    std::vector<fm_ctx*> v;
    int device = 0;
    int precision = FM_FP32;
    cudaStream_t origin = nullptr;
    bool own_origin = false;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t gexec = nullptr;
    std::vector<int> gen;  // history generations the captured graph was built with
    double fraction = 1.0;
    int icb_per_sm = 2;  // back-substitution blocks per SM (before the fraction)
    std::string err;
};

namespace {

void batch_free(fm_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (fm_ctx* c : b->v) fm_destroy(c);
    if (b->own_origin && b->origin) cudaStreamDestroy(b->origin);
}

void batch_apply_fraction(fm_batch* b) {
    for (fm_ctx* c : b->v) {
        c->grid_data = std::max(1, (int)std::lround(c->base_data * b->fraction));
        c->grid_ls = std::max(1, (int)std::lround(c->base_ls * b->fraction));
        c->grid_ic = std::max(1, (int)std::lround(c->base_ic * b->fraction));
        const int icb = std::max(1, std::min(c->ntiles, std::min(c->occ_icb, b->icb_per_sm) * c->nsm));
        c->grid_icb = std::max(1, (int)std::lround(icb * b->fraction));
        if (c->base_ict) c->grid_ict = std::max(1, (int)std::lround(c->base_ict * b->fraction));
        if (c->base_ictg) c->grid_ictg = std::max(1, (int)std::lround(c->base_ictg * b->fraction));
        if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    }
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
}

// origin -> every volume stream
cudaError_t batch_fork(fm_batch* b) {
    cudaError_t e = cudaEventRecord(b->fork, b->origin);
    for (fm_ctx* c : b->v)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, b->fork, 0);
    return e;
}

// every volume stream -> origin
cudaError_t batch_join(fm_batch* b) {
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < b->v.size() && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->join[k], b->v[k]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->join[k], 0);
    }
    return e;
}

template <typename T>
int batch_solve_t(fm_batch* b, void* const* omega_in, void* const* omega, int init, int niter,
                  double* const* cost_hist) {
    const size_t n = b->v.size();
    auto fail_b = [&](int code, const std::string& m) { b->err = m; return code; };
    if (batch_fork(b) != cudaSuccess) return fail_b(FM_ERR_CUDA, "fork");
    for (size_t k = 0; k < n; ++k) {
        const int rc = solve_begin<T>(b->v[k], omega_in[k], init, niter);
        if (rc != FM_OK) return fail_b(rc, "volume " + std::to_string(k) + ": " + b->v[k]->err);
    }
    int i = 0;
    if (niter >= 2) {
        bool stale = !b->gexec || b->gen.size() != n;
        for (size_t k = 0; k < n && !stale; ++k) stale = b->gen[k] != b->v[k]->hist_gen;
        if (stale) {
            if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) e = batch_fork(b);
            for (size_t k = 0; k < n && e == cudaSuccess; ++k) {
                e = iteration<T>(b->v[k], 0);
                if (e == cudaSuccess) e = iteration<T>(b->v[k], 1);
            }
            if (e == cudaSuccess) e = batch_join(b);
            cudaError_t ee = cudaStreamEndCapture(b->origin, &graph);
            if (e != cudaSuccess || ee != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return fail_b(FM_ERR_CUDA, std::string("capture batch iteration: ") +
                                               cudaGetErrorString(e != cudaSuccess ? e : ee));
            }
            e = cudaGraphInstantiate(&b->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return fail_b(FM_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
            b->gen.resize(n);
            for (size_t k = 0; k < n; ++k) b->gen[k] = b->v[k]->hist_gen;
        }
        // the volumes' set-up work runs on their own streams before the graph
        if (batch_join(b) != cudaSuccess) return fail_b(FM_ERR_CUDA, "join");
        for (; i + 2 <= niter; i += 2)
            if (cudaGraphLaunch(b->gexec, b->origin) != cudaSuccess) return fail_b(FM_ERR_CUDA, "launch graph");
        if (batch_fork(b) != cudaSuccess) return fail_b(FM_ERR_CUDA, "fork");
    }
    for (size_t k = 0; k < n; ++k) {
        fm_ctx* c = b->v[k];
        for (int ii = i; ii < niter; ++ii)
            if (iteration<T>(c, ii & 1) != cudaSuccess) return fail_b(FM_ERR_CUDA, "launch iteration");
        const int rc = solve_end<T>(c, omega[k], niter, cost_hist ? cost_hist[k] : nullptr);
        if (rc != FM_OK) return fail_b(rc, "volume " + std::to_string(k) + ": " + c->err);
    }
    if (batch_join(b) != cudaSuccess) return fail_b(FM_ERR_CUDA, "join");
    int first = FM_OK;
    for (size_t k = 0; k < n; ++k) {
        const int rc = check_dev(b->v[k]);
        if (rc != FM_OK && first == FM_OK) {
            first = rc;
            b->err = "volume " + std::to_string(k) + ": " + b->v[k]->err;
        }
    }
    return first;
}

int batch_solve_io(fm_batch* b, void* const* omega_in, void* const* omega, int init, int niter,
                   double* const* cost_hist) {
    return b->precision == FM_FP64 ? batch_solve_t<double>(b, omega_in, omega, init, niter, cost_hist)
                                   : batch_solve_t<float>(b, omega_in, omega, init, niter, cost_hist);
}

int batch_solve(fm_batch* b, void* const* omega, int init, int niter, double* const* cost_hist) {
    return batch_solve_io(b, omega, omega, init, niter, cost_hist);
}

}  // namespace

extern "C" {

int fm_batch_create(fm_batch** out, int n, const int* dims, const fm_opts* opts, int device, void* cuda_stream) {
    if (!out) return FM_ERR_ARG;
    *out = nullptr;
    if (n < 1 || !dims) return FM_ERR_ARG;
    fm_batch* b = new (std::nothrow) fm_batch();
    if (!b) return FM_ERR_OOM;
    b->device = device;
    fm_opts o;
    fm_default_opts(&o);
    if (opts) o = *opts;
    b->precision = o.precision;
    for (int k = 0; k < n; ++k) {
        fm_ctx* c = nullptr;
        const int* d = dims + 5 * k;
        const int rc = fm_create(&c, d[0], d[1], d[2], d[3], d[4], &o, device, nullptr);
        if (rc != FM_OK) {
            batch_free(b);
            delete b;
            return rc;
        }
        b->v.push_back(c);
    }
    DevGuard guard(device);
    bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    b->join.assign(n, nullptr);
    for (int k = 0; k < n && ok; ++k) ok = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
        if (cuda_stream) {
            b->origin = (cudaStream_t)cuda_stream;
        } else {
            ok = cudaStreamCreate(&b->origin) == cudaSuccess;
            b->own_origin = ok;
        }
    }
    if (!ok) {
        batch_free(b);
        delete b;
        return FM_ERR_CUDA;
    }
    *out = b;
    return FM_OK;
}

int fm_batch_set_data(fm_batch* b, int k, const void* y, const void* smap, const double* te, const uint8_t* mask,
                      double beta) {
    if (!b || k < 0 || k >= (int)b->v.size()) return FM_ERR_ARG;
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }  // beta / dt are graph arguments
    return fm_set_data(b->v[k], y, smap, te, mask, beta);
}

int fm_batch_solve(fm_batch* b, void* const* omega, int init_from_data, int niter, double* const* cost_hist) {
    if (!b || !omega || niter < 0) return FM_ERR_ARG;
    for (size_t k = 0; k < b->v.size(); ++k) {
        if (!omega[k]) return FM_ERR_ARG;
        if (!b->v[k]->have_data) return FM_ERR_STATE;
    }
    DevGuard guard(b->device);
    // the drop-tolerance IC: a volume whose factor keeps fill outside its held pattern grows the
    // pattern and the batch runs again from the same starts
    std::vector<void*> w0;
    std::vector<void*> in(omega, omega + b->v.size());
    if (!init_from_data && b->v[0]->o.precond == FM_PC_ICT) {
        for (size_t k = 0; k < b->v.size(); ++k) {
            fm_ctx* c = b->v[k];
            const size_t vb = (size_t)c->nv * c->ts;
            if (!c->ict_w0 && dalloc(&c->ict_w0, vb) != cudaSuccess) { cudaGetLastError(); return FM_ERR_OOM; }
            if (cudaMemcpyAsync(c->ict_w0, omega[k], vb, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
                return FM_ERR_CUDA;
            in[k] = c->ict_w0;
        }
    }
    for (int round = 0;; ++round) {
        int rc = batch_solve_io(b, in.data(), omega, init_from_data, niter, cost_hist);
        if (rc != FM_ERR_FILL || round >= kIctMaxRounds) return rc;
        int grew = 0;
        for (fm_ctx* c : b->v) {
            const int g = ict_grow(c);
            if (g < 0) return g;
            grew += g;
        }
        if (!grew) return rc;
        if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    }
}

int fm_batch_set_fraction(fm_batch* b, double fraction) {
    if (!b || !(fraction > 0.0) || fraction > 1.0) return FM_ERR_ARG;
    DevGuard guard(b->device);
    b->fraction = fraction;
    batch_apply_fraction(b);
    return FM_OK;
}

int fm_batch_autotune(fm_batch* b, int niter_probe, double* best_fraction, double* best_ms) {
    if (!b || niter_probe < 2) return FM_ERR_ARG;
    for (fm_ctx* c : b->v)
        if (!c->have_data) return FM_ERR_STATE;
    DevGuard guard(b->device);
    std::vector<void*> w(b->v.size(), nullptr);
    bool ok = true;
    for (size_t k = 0; k < b->v.size() && ok; ++k) ok = dalloc(&w[k], (size_t)b->v[k]->nv * b->v[k]->ts) == cudaSuccess;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ok = ok && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    const double cand[4] = {1.0, 0.5, 0.25, 0.125};
    const int wcand[3][2] = {{2, 1}, {1, 1}, {3, 2}};  // forward tile claim order weights (X + Y, Z)
    const int bcand[3] = {1, 2, 3};                    // back-substitution blocks per SM
    double bestf = b->fraction, bestt = 1e300;
    int bestw = 0, bestb = b->icb_per_sm;
    int rc = ok ? FM_OK : FM_ERR_OOM;
    auto probe = [&](double f, int wq, int bq) {
        b->fraction = f;
        b->icb_per_sm = bcand[bq];
        batch_apply_fraction(b);
        rc = batch_solve(b, w.data(), 1, niter_probe, nullptr);  // warm-up and capture
        if (rc != FM_OK) return;
        cudaEventRecord(e0, b->origin);
        rc = batch_solve(b, w.data(), 1, niter_probe, nullptr);
        cudaEventRecord(e1, b->origin);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rc == FM_OK && ms < bestt) {
            bestt = ms;
            bestf = f;
            bestw = wq;
            bestb = bcand[bq];
        }
    };
    // grid fraction x forward claim order at two back-substitution blocks per SM, then the
    // back substitution's blocks per SM at the best of those
    for (int wq = 0; wq < 3 && rc == FM_OK; ++wq) {
        for (fm_ctx* c : b->v)
            if (!set_ic_order(c, wcand[wq][0], wcand[wq][1])) rc = FM_ERR_CUDA;
        for (int q = 0; q < 4 && rc == FM_OK; ++q) probe(cand[q], wq, 1);
    }
    for (fm_ctx* c : b->v)
        if (rc == FM_OK && !set_ic_order(c, wcand[bestw][0], wcand[bestw][1])) rc = FM_ERR_CUDA;
    for (int bq = 0; bq < 3 && rc == FM_OK; ++bq)
        if (bcand[bq] != 2) probe(bestf, bestw, bq);
    for (void* p : w)
        if (p) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (fm_ctx* c : b->v)
        if (!set_ic_order(c, wcand[bestw][0], wcand[bestw][1]) && rc == FM_OK) rc = FM_ERR_CUDA;
    b->fraction = bestf;
    b->icb_per_sm = bestb;
    batch_apply_fraction(b);
    if (best_fraction) *best_fraction = bestf;
    if (best_ms) *best_ms = bestt;
    return rc;
}

int fm_batch_schedule(const fm_batch* b, double* fraction, int* order_wxy, int* order_wz) {
    if (!b || b->v.empty()) return FM_ERR_ARG;
    if (fraction) *fraction = b->fraction;
    if (order_wxy) *order_wxy = b->v[0]->ic_wxy;
    if (order_wz) *order_wz = b->v[0]->ic_wz;
    return FM_OK;
}

int fm_batch_bwd_blocks(const fm_batch* b, int* blocks_per_sm) {
    if (!b || !blocks_per_sm) return FM_ERR_ARG;
    *blocks_per_sm = b->icb_per_sm;
    return FM_OK;
}

fm_ctx* fm_batch_ctx(fm_batch* b, int k) {
    if (!b || k < 0 || k >= (int)b->v.size()) return nullptr;
    return b->v[k];
}

int fm_batch_destroy(fm_batch* b) {
    if (!b) return FM_OK;
    {
        DevGuard guard(b->device);
        if (b->origin) cudaStreamSynchronize(b->origin);
        batch_free(b);
    }
    delete b;
    return FM_OK;
}

}  // extern "C"
