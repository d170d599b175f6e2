// fm_api.cu -- host side of the C ABI declared in include/fm.h: context, argument
// checking, buffer ownership, and the launch sequence of one NCG-MLS-IC outer iteration
// (Algorithm box), replayed from a captured CUDA graph.
#include <algorithm>
#include <cmath>
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
    // device buffers
    void *pairs = nullptr, *coils = nullptr, *w0 = nullptr;
    uint8_t* nb = nullptr;
    int *vlist = nullptr, *chunk_off = nullptr;
    void *w[2] = {nullptr, nullptr}, *z[2] = {nullptr, nullptr}, *g[2] = {nullptr, nullptr};
    void *d = nullptr, *p = nullptr, *v = nullptr, *ip = nullptr;
    double *scal = nullptr, *partials = nullptr, *tile_part = nullptr;
    void* face = nullptr;
    double *hist_cost = nullptr, *hist_alpha = nullptr, *hist_mu = nullptr;
    int hist_cap = 0;
    int* istate = nullptr;
    int* icint = nullptr;  // [0] fwd ticket, [1] bwd ticket, [2] bwd done, [3] pad, flags fwd[nt], flags bwd[nt]
    int* order = nullptr;
    int ntx = 0, nty = 0, ntz = 0, ntiles = 0;
    int nsm = 0, grid_data = 0, grid_ls = 0, grid_ic = 0;
    int last_niter = 0;
    cudaGraphExec_t gexec = nullptr;
    bool profiling = false;
    cudaEvent_t ev[2][FM_NKERNEL][2] = {};
    bool ev_rec[2][FM_NKERNEL] = {};
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
    for (auto& a : c->ev)
        for (auto& b : a)
            for (cudaEvent_t& e : b)
                if (e) cudaEventDestroy(e);
    void* bufs[] = {c->pairs, c->coils, c->w0, c->nb, c->vlist, c->chunk_off, c->w[0], c->w[1], c->z[0], c->z[1], c->g[0],
                    c->g[1], c->d, c->p, c->v, c->ip, c->scal, c->partials, c->face, c->tile_part,
                    c->hist_cost, c->hist_alpha, c->hist_mu, c->istate, c->icint, c->order};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

// Read back the device error word and clear it.
int check_dev(fm_ctx* c) {
    int e = 0;
    cudaError_t ce = cudaMemcpyAsync(&e, c->istate + I_ERR, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "synchronise");
    if (e != 0) {
        cudaMemsetAsync(c->istate + I_ERR, 0, sizeof(int), c->stream);
        const char* what = e == FM_ERR_NOT_PD ? "IC(0) pivot <= 0 (H not positive definite on the mask)"
                         : e == FM_ERR_TIMEOUT ? "device-side wait exceeded spin_limit"
                         : e == FM_ERR_NONFINITE ? "non-finite global reduction"
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
cudaError_t run_ic(fm_ctx* c, const void* d, const void* g, void* p, const void* gdot, const void* gpdot,
                   int slot = -1) {
    const size_t nint = 4 + 2 * (size_t)c->ntiles;
    cudaError_t e = cudaMemsetAsync(c->icint, 0, nint * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    IcArgs f = ic_args(c);
    f.flags = c->icint + 4;
    f.ticket = c->icint + 0;
    f.d = d;
    f.ip_in = d ? nullptr : c->ip;
    f.g = g;
    f.v = c->v;
    f.ip_out = c->ip;
    {
        fm_ctx* pc = slot >= 0 ? c : nullptr;
        if (pc && pc->profiling) cudaEventRecordWithFlags(pc->ev[slot][FM_K_IC_FWD][0], c->stream, cudaEventRecordExternal);
        e = launch_ic_fwd<T>(f, c->grid_ic, c->stream);
        if (pc && pc->profiling) {
            cudaEventRecordWithFlags(pc->ev[slot][FM_K_IC_FWD][1], c->stream, cudaEventRecordExternal);
            pc->ev_rec[slot][FM_K_IC_FWD] = true;
        }
    }
    if (e != cudaSuccess) return e;
    IcArgs b = ic_args(c);
    b.flags = c->icint + 4 + c->ntiles;
    b.ticket = c->icint + 1;
    b.done = c->icint + 2;
    b.vin = c->v;
    b.ipb = c->ip;
    b.p = p;
    b.gdot = gdot;
    b.gpdot = gpdot;
    b.tile_part = (gdot || gpdot) ? c->tile_part : nullptr;
    if (slot >= 0 && c->profiling) cudaEventRecordWithFlags(c->ev[slot][FM_K_IC_BWD][0], c->stream, cudaEventRecordExternal);
    e = launch_ic_bwd<T>(b, c->grid_ic, c->stream);
    if (slot >= 0 && c->profiling) {
        cudaEventRecordWithFlags(c->ev[slot][FM_K_IC_BWD][1], c->stream, cudaEventRecordExternal);
        c->ev_rec[slot][FM_K_IC_BWD] = true;
    }
    return e;
}

// Brackets one kernel class of iteration slot `cur` with events when profiling.
struct Mark {
    fm_ctx* c;
    int cur, k;
    Mark(fm_ctx* c_, int cur_, int k_) : c(c_), cur(cur_), k(k_) {
        if (c->profiling) cudaEventRecordWithFlags(c->ev[cur][k][0], c->stream, cudaEventRecordExternal);
    }
    ~Mark() {
        if (c->profiling) {
            cudaEventRecordWithFlags(c->ev[cur][k][1], c->stream, cudaEventRecordExternal);
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
    if (c->o.precond == FM_PC_IC0) {
        e = run_ic<T>(c, c->d, c->g[cur], c->p, c->g[cur], c->g[nxt], cur);
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
        Mark m(c, cur, FM_K_DIR);
        e = launch_dir<T>(a, c->grid_data, c->stream);
    }
    if (e != cudaSuccess) return e;
    if (c->o.nls > 1) {
        Mark m(c, cur, FM_K_LS);
        e = launch_ls<T>(a, c->grid_ls, c->stream);
    }
    return e;
}

template <typename T>
int solve_t(fm_ctx* c, void* omega, int init, int niter, double* cost_hist) {
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
    }
    const size_t vb = (size_t)c->nv * c->ts;
    cudaStream_t s = c->stream;
    FM_CK(cudaMemsetAsync(c->istate + I_ERR, 0, sizeof(int), s), "reset");
    // the kernels write mask voxels only: every entry outside the mask starts (and stays) 0
    if (init) {
        FM_CK(cudaMemcpyAsync(c->w[0], c->w0, vb, cudaMemcpyDeviceToDevice, s), "copy omega");
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
    const int cur = niter & 1;
    FM_CK(run_grad<T>(c, c->w[cur], c->z[cur], c->w[cur ^ 1], c->g[cur], c->d, c->hist_cost), "final update");
    FM_CK(cudaMemcpyAsync(omega, c->w[cur ^ 1], vb, cudaMemcpyDeviceToDevice, s), "copy omega out");
    if (cost_hist)
        FM_CK(cudaMemcpyAsync(cost_hist, c->hist_cost, (niter + 1) * sizeof(double), cudaMemcpyDeviceToHost, s),
              "copy cost history");
    c->last_niter = niter;
    return check_dev(c);
}

bool valid_opts(const fm_opts& o) {
    return (o.precision == FM_FP32 || o.precision == FM_FP64) && o.nls >= 1 && o.nls <= 1000 &&
           (o.precond == FM_PC_IC0 || o.precond == FM_PC_DIAG || o.precond == FM_PC_NONE) &&
           (o.curvature == FM_CURV_LITERAL || o.curvature == FM_CURV_COMBINED) && o.spin_limit >= 1;
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
    {
        DataArgs probe{};
        probe.nc = ncoil;
        probe.literal = c->literal;
        const int occ = o.precision == FM_FP64 ? ls_max_blocks_per_sm<double>(probe) : ls_max_blocks_per_sm<float>(probe);
        if (occ < 1) return bail(FM_ERR_CUDA);
        c->grid_ls = (int)std::max(1LL, std::min<long long>(nblk, (long long)occ * c->nsm));
    }
    c->ntx = (nx + kTileX - 1) / kTileX;
    c->nty = (ny + kTileY - 1) / kTileY;
    const int tz = o.precision == FM_FP64 ? ic_tz<double>() : ic_tz<float>();
    c->ntz = (nz + tz - 1) / tz;
    c->ntiles = c->ntx * c->nty * c->ntz;
    {
        const int occ = o.precision == FM_FP64 ? ic_max_blocks_per_sm<double>() : ic_max_blocks_per_sm<float>();
        if (occ < 1) return bail(FM_ERR_CUDA);
        c->grid_ic = std::max(1, std::min(c->ntiles, occ * c->nsm));
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
    A(&c->d, vb); A(&c->p, vb); A(&c->v, vb); A(&c->ip, vb);
    A(&c->scal, S_NSCAL * sizeof(double));
    A(&c->partials, std::max<size_t>(8 * (size_t)std::max(c->grid_data, c->grid_ls), nchunks) * sizeof(double));
    A(&c->face, (size_t)c->ntiles *
                    (o.precision == FM_FP64 ? ic_face_bytes_per_tile<double>() : ic_face_bytes_per_tile<float>()));
    A(&c->tile_part, 2 * (size_t)c->ntiles * sizeof(double));
    A(&c->istate, I_NISTATE * sizeof(int));
    A(&c->icint, (4 + 2 * (size_t)c->ntiles) * sizeof(int));
    A(&c->order, (size_t)c->ntiles * sizeof(int));
    if (!ok) { cudaGetLastError(); return bail(FM_ERR_OOM); }
    // tiles in order of their tile hyperplane X + Y + Z (ties: z, y, x), a topological order
    std::vector<int> ord(c->ntiles);
    for (int t = 0; t < c->ntiles; ++t) ord[t] = t;
    const int ntx = c->ntx, nty = c->nty;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
        const int ha = a % ntx + (a / ntx) % nty + a / (ntx * nty);
        const int hb = b % ntx + (b / ntx) % nty + b / (ntx * nty);
        return ha != hb ? ha < hb : a < b;
    });
    if (cudaMemcpy(c->order, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->scal, 0, S_NSCAL * sizeof(double)) != cudaSuccess ||
        cudaMemset(c->istate, 0, I_NISTATE * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->nb, 0, (size_t)c->nv) != cudaSuccess)
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
    c->beta = beta;
    for (int l = 0; l < c->L; ++l) c->te[l] = te[l];
    Pairs pr{};
    for (int m = 0; m < c->L; ++m)
        for (int n = m + 1; n < c->L; ++n) {
            pr.m[pr.P] = m;
            pr.n[pr.P] = n;
            pr.dt[pr.P] = te[m] - te[n];
            ++pr.P;
        }
    c->pr = pr;
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }  // beta / dt are graph arguments
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

int fm_ic_factor(fm_ctx* c, const void* omega, void* inv_pivot) {
    if (!c) return FM_ERR_ARG;
    if (!omega) return fail(c, FM_ERR_ARG, "omega is required");
    if (!c->have_data) return fail(c, FM_ERR_STATE, "fm_set_data first");
    DevGuard guard(c->device);
    const bool f64 = c->o.precision == FM_FP64;
    cudaError_t e = f64 ? run_grad<double>(c, omega, nullptr, c->w[0], c->g[0], c->d, nullptr)
                        : run_grad<float>(c, omega, nullptr, c->w[0], c->g[0], c->d, nullptr);
    if (e != cudaSuccess) return cuda_fail(c, e, "gradient kernel");
    e = f64 ? run_ic<double>(c, c->d, c->g[0], c->p, nullptr, nullptr)
            : run_ic<float>(c, c->d, c->g[0], c->p, nullptr, nullptr);
    if (e != cudaSuccess) return cuda_fail(c, e, "IC(0) kernels");
    if (inv_pivot)
        FM_CK(cudaMemcpyAsync(inv_pivot, c->ip, (size_t)c->nv * c->ts, cudaMemcpyDeviceToDevice, c->stream), "copy");
    c->have_factor = true;
    return FM_OK;
}

int fm_ic_apply(fm_ctx* c, const void* g, void* p) {
    if (!c) return FM_ERR_ARG;
    if (!g || !p || g == p) return fail(c, FM_ERR_ARG, "g and p must be distinct device arrays");
    if (!c->have_factor) return fail(c, FM_ERR_STATE, "fm_ic_factor first");
    DevGuard guard(c->device);
    cudaError_t e = c->o.precision == FM_FP64 ? run_ic<double>(c, nullptr, g, p, nullptr, nullptr)
                                              : run_ic<float>(c, nullptr, g, p, nullptr, nullptr);
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
