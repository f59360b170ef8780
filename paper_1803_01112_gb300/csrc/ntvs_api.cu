// Host runtime and C ABI of the NTVS library (declared in include/ntvs.h).
//
// The outer loop of NTVS (arXiv 1803.01112, Appendix C) runs here on the host: it
// draws ell_k = rand(k, ell_{k-1}) (Sec. III-B item 4), forms beta = beta0 * alpha^ell
// (Appendix A) and queues the kernels of one cycle on the context's stream: N TV
// perturbation steps, then one block-DROP sweep P_T (Sec. III-D), then phi(x) in FP64.
// Without the TV check nothing waits on the device; with it the host reads each
// accept decision (one small device-to-host copy per try).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ntvs.h"
#include "ntvs_internal.h"
#include "step_rule.h"

using namespace ntvs;

namespace {

thread_local std::string g_err;

constexpr uint64_t kDefaultWaitNs = 2000000000ull;   // 2 s per bounded device wait
constexpr int kBetaTab = 4096;                        // step sizes tabulated on the host

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

std::string cuda_msg(const char* what, cudaError_t e) { return std::string(what) + ": " + cudaGetErrorString(e); }

#define CUDA_TRY(expr)                                                                                      \
    do {                                                                                                    \
        cudaError_t e_ = (expr);                                                                            \
        if (e_ != cudaSuccess)                                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? NTVS_ERR_OOM : NTVS_ERR_CUDA, cuda_msg(#expr, e_)); \
    } while (0)

#define TRY(expr)                   \
    do {                            \
        int r_ = (expr);            \
        if (r_ != NTVS_OK) return r_; \
    } while (0)

template <typename T>
int dev_alloc(T** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? NTVS_ERR_OOM : NTVS_ERR_CUDA,
                    std::string("device allocation of ") + what + " (" + std::to_string(bytes) + " bytes): " +
                        cudaGetErrorString(e));
    }
    return NTVS_OK;
}

template <typename T>
void dev_free(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

}  // namespace

void ntvs::set_last_error(const std::string& msg) { g_err = msg; }

struct ntvs_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t copy_stream = nullptr;   // load: host-to-device copies overlapped with preparation
    cudaStream_t copy_stream2 = nullptr;  // (columns on one, values on the other: two copies in flight)
    int sms = 1;

    // system
    bool loaded = false;
    int nx = 0, ny = 0, nz = 0;
    int64_t V = 0, M = 0, nnz = 0;
    int B = 0;
    // internal voxel order of x32, delta, inv_s and the stored columns (FP32 path)
    VoxMap vm{};
    int tile_req_x = 4, tile_req_y = 4;   // applied at the next load
    int compute_req = F32;                // arithmetic of FP32-stored systems, applied at the next load
    int vdt = F32, cdt = F32, storage = NTVS_CSR32;
    std::vector<int64_t> block_ptr;
    std::vector<int64_t> block_maxrow;   // longest row of each block
    int64_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    void* val = nullptr;
    void* b = nullptr;
    bool own_row_ptr = false, own_col = false, own_val = false, own_b = false;
    // CSR32 storage with FP32 values: [nnz] {column, value bits} pairs packed at load (the
    // DROP, projection and pipelined kernels read one 8-byte pair per entry); col and val
    // are released once the schedule is planned
    int32_t* ent = nullptr;
    // the column array the DROP kernels take: the packed pairs when there are any
    const int32_t* drop_cols() const { return ent ? ent : col; }
    void* inv_norm2 = nullptr;
    void* inv_s = nullptr;
    int lpr = 32;
    int drop_grid = 1;
    int apply_grid = 1;
    bool vector4 = false;
    int schedule = NTVS_SCHED_PLAIN;
    DropSegment* segs = nullptr;       // windowed schedule: all blocks' segments
    int32_t* seg_begin = nullptr;      // [B][win_grid + 1]
    DropStage* stages = nullptr;       // pipelined schedule: all blocks' stages
    int32_t* stage_begin = nullptr;    // [B][win_grid + 1]
    int win_grid = 0;
    float* wstat = nullptr;            // FP32 window scale per block: lmax [B], bound [B], observed [B],
                                       // then per block the seed bound and max |a| [2B]
    int* derr = nullptr;               // device error word (bounded waits that ran out)
    // DELTA16 index storage (packed at load from the int32 columns)
    uint16_t* d16off = nullptr;        // [nnz] column - chunk base
    int32_t* d16base = nullptr;        // [ceil(nnz/32)] chunk bases (negative: escaped chunk)
    int32_t* d16exc = nullptr;         // [escaped chunks][32] full columns
    uint8_t* d16rowesc = nullptr;      // [M] rows touching an escaped chunk
    uint32_t* d16word = nullptr;       // [nnz] 16-bit values: offset | value bits << 16 (replaces d16off, val)
    int64_t n_escaped = 0;             // escaped chunks
    // on-the-fly rows (ntvs_load_paths): path records and b, traced every sweep
    bool paths_mode = false;
    float* paths = nullptr;
    bool own_paths = false;
    OtfArgs otf{};
    Delta16 d16() const { return Delta16{d16off, d16base, d16exc, d16rowesc, d16word}; }

    // image and scratch: x is the FP64 master image; x32 its FP32 copy gathered by the
    // FP32-path DROP kernels (null on the FP64 path)
    double* x = nullptr;
    float* x32 = nullptr;
    float* xh = nullptr;   // FP32 path: fl32(x) and fl32(x - xh), canonical order (TV stencil)
    float* xl = nullptr;
    void* delta = nullptr;
    void* g = nullptr;
    RedScratch red{nullptr, nullptr, 1};
    double* dscal = nullptr;   // [0] ||g||^2, [1] phi(x), [2] phi(z), [3] phi for ntvs_get_tv
    int* daccept = nullptr;
    int* dflags = nullptr;
    double* resid = nullptr;   // [B]
    double* tvhist = nullptr;  // [tvcap]
    int64_t tvcap = 0;
    double* hscal = nullptr;   // pinned [8]
    int* hint = nullptr;       // pinned [4]
    int64_t* hll = nullptr;    // pinned [4]

    // TV check decided on the device: ell and the traces stay on the device while runs are
    // queued; the host pulls them (one synchronization) when it needs them
    CheckState* cstate = nullptr;
    int64_t* dev_ell_tr = nullptr;    // ell_k per cycle, indexed like ell_trace
    int32_t* dev_tries = nullptr;     // per step, indexed like tries_trace
    int32_t* dev_acc = nullptr;
    int64_t dtr_cap_k = 0, dtr_cap_s = 0;
    bool dev_pending = false;         // cycles [pend_k0, ell_trace.size()) still on the device
    int64_t pend_k0 = 0, pend_s0 = 0;
    bool dstate_valid = false;        // device ell == ell_prev
    double* beta_tab = nullptr;       // beta0 * alpha^ell, ell < kBetaTab (host-computed)
    double tab_beta0 = -1.0, tab_alpha = -1.0;
    int check_grid = 0;               // co-resident grid of the retry loop (0: host decisions)

    // row-sharded reconstruction: every DROP block's delta is summed over ranks by this
    // callback before it is applied (null: this context holds every row)
    ntvs_allreduce_fn ar_fn = nullptr;
    void* ar_user = nullptr;
    void* ext = nullptr;              // staging of host-side deltas and hit counts (V x 8 bytes)

    // bounded device waits: budget per wait and the test hook that starves a wait
    uint64_t wait_ns = kDefaultWaitNs;
    int hook_flags = 0;

    // parameters and state
    ntvs_params p{};
    int64_t k = 0, ell_prev = 0;
    std::vector<int64_t> ell_trace;
    std::vector<int32_t> tries_trace, acc_trace;
    std::vector<int64_t> override_ell;
    size_t override_pos = 0;
    int64_t n_steps = 0, n_accepted = 0, n_tries = 0;
    int64_t n_launches = 0;

    // per-launch event timing (profiling on): pairs recorded around each launch
    bool profiling = false;
    struct Timed { int kind; cudaEvent_t a, b; };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> event_pool;
    double prof_ms[3] = {0, 0, 0};
    int64_t prof_n[3] = {0, 0, 0};

    size_t csz() const { return dt_size(cdt); }
    // with_split = false leaves xh/xl stale (split_stale), to be refreshed before the next
    // gradient: DROP blocks other than the last of a sweep skip them
    ImgCopies copies(bool with_split = true) const {
        return ImgCopies{x32, with_split ? xh : nullptr, with_split ? xl : nullptr, vm};
    }
    bool split_stale = false;

    void free_system() {
        if (copy_stream) cudaStreamSynchronize(copy_stream);   // no copy may still target a buffer
        if (copy_stream2) cudaStreamSynchronize(copy_stream2);
        if (own_row_ptr) dev_free(row_ptr);
        if (own_col) dev_free(col);
        if (own_val) dev_free(val);
        if (own_b) dev_free(b);
        row_ptr = nullptr; col = nullptr; val = nullptr; b = nullptr;
        own_row_ptr = own_col = own_val = own_b = false;
        dev_free(ent);
        dev_free(inv_norm2);
        dev_free(inv_s);
        dev_free(segs);
        dev_free(seg_begin);
        dev_free(wstat);
        dev_free(stages);
        dev_free(stage_begin);
        dev_free(d16off);
        dev_free(d16base);
        dev_free(d16exc);
        dev_free(d16rowesc);
        dev_free(d16word);
        n_escaped = 0;
        if (own_paths) dev_free(paths);
        paths = nullptr;
        own_paths = false;
        paths_mode = false;
        schedule = NTVS_SCHED_PLAIN;
        dev_free(x);
        dev_free(x32);
        dev_free(xh);
        dev_free(xl);
        dev_free(delta);
        dev_free(g);
        dev_free(resid);
        loaded = false;
    }
};

namespace {

int use_device(ntvs_ctx* c) {
    if (!c) return fail(NTVS_ERR_ARG, "null context");
    CUDA_TRY(cudaSetDevice(c->device));
    return NTVS_OK;
}

int need_system(ntvs_ctx* c) {
    if (!c->loaded) return fail(NTVS_ERR_STATE, "no system loaded");
    return NTVS_OK;
}

enum { KIND_DROP = 0, KIND_APPLY = 1, KIND_TV = 2 };

cudaEvent_t take_event(ntvs_ctx* c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Folds finished timings into the totals (after a stream sync).
void harvest_timing(ntvs_ctx* c) {
    for (auto& t : c->timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            c->prof_ms[t.kind] += ms;
            c->prof_n[t.kind] += 1;
        }
        c->event_pool.push_back(t.a);
        c->event_pool.push_back(t.b);
    }
    c->timed.clear();
}

// Runs launch() on the context's stream, counted and (when profiling) bracketed by events.
template <typename F>
cudaError_t timed_launch(ntvs_ctx* c, int kind, F launch) {
    c->n_launches += 1;
    if (!c->profiling) return launch();
    if (c->timed.size() > 4096) {   // bound the outstanding events
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return e;
        harvest_timing(c);
    }
    cudaEvent_t a = take_event(c), b = take_event(c);
    cudaEventRecord(a, c->stream);
    cudaError_t e = launch();
    cudaEventRecord(b, c->stream);
    c->timed.push_back({kind, a, b});
    return e;
}

// Reads (and clears) the device error word after the stream has drained: a bounded
// device-side wait that ran out leaves a nonzero code there.
int check_device_error(ntvs_ctx* c) {
    CUDA_TRY(cudaMemcpyAsync(c->hint + 1, c->derr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    const int code = c->hint[1];
    if (code) {
        CUDA_TRY(cudaMemsetAsync(c->derr, 0, sizeof(int), c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        return fail(NTVS_ERR_TIMEOUT, std::string("a bounded device wait ran out (") +
                                          (code == kErrCheckBarrier ? "TV-check loop barrier" : "pipelined DROP kernel") +
                                          ", code " + std::to_string(code) + "); the image of this run is invalid");
    }
    return NTVS_OK;
}

int copy_in(void** dst, bool* own, const void* src, size_t bytes, int mem_kind, cudaStream_t s, const char* what) {
    if (mem_kind == NTVS_MEM_DEVICE) {
        *dst = const_cast<void*>(src);
        *own = false;
        return NTVS_OK;
    }
    TRY(dev_alloc(dst, bytes, what));
    *own = true;
    if (bytes) CUDA_TRY(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s));
    return NTVS_OK;
}

int ensure_tvhist(ntvs_ctx* c, int64_t need) {
    if (need <= c->tvcap) return NTVS_OK;
    int64_t cap = c->tvcap ? c->tvcap : 1024;
    while (cap < need) cap *= 2;
    double* nb = nullptr;
    TRY(dev_alloc(&nb, (size_t)cap * sizeof(double), "tv history"));
    if (c->tvhist) {
        CUDA_TRY(cudaMemcpyAsync(nb, c->tvhist, (size_t)c->tvcap * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        dev_free(c->tvhist);
    }
    c->tvhist = nb;
    c->tvcap = cap;
    return NTVS_OK;
}

// ---- one TV perturbation step (Appendix C inner loop) --------------------------------
int launch_grad(ntvs_ctx* c, bool with_phi) {
    if (c->xh && c->split_stale) {
        CUDA_TRY(timed_launch(c, KIND_TV, [&] {
            return k_x32_from_x64(c->x, ImgCopies{nullptr, c->xh, c->xl, c->vm}, c->stream);
        }));
        c->split_stale = false;
    }
    CUDA_TRY(timed_launch(c, KIND_TV, [&] {
        return k_tv_grad(c->cdt, c->x, c->xh, c->xl, c->g, c->nx, c->ny, c->nz, c->p.eps_tv, c->red, c->dscal + 0,
                         with_phi ? c->dscal + 1 : nullptr, c->stream);
    }));
    return NTVS_OK;
}

// one check-mode try with step beta: returns accept in *acc (host), x updated when accepted
int checked_try(ntvs_ctx* c, double beta, int* acc) {
    CUDA_TRY(timed_launch(c, KIND_TV, [&] {
        return k_tv_value(c->cdt, c->x, c->g, c->dscal + 0, beta, c->nx, c->ny, c->nz, c->red, c->dscal + 2,
                          c->dscal + 1, c->daccept, c->stream);
    }));
    CUDA_TRY(timed_launch(c, KIND_TV, [&] {
        return k_tv_apply(c->cdt, c->x, c->copies(), c->g, c->dscal + 0, beta, c->daccept, c->V, c->stream);
    }));
    CUDA_TRY(cudaMemcpyAsync(c->hint, c->daccept, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    *acc = c->hint[0];
    return NTVS_OK;
}

// Brings the traces, counters and ell of device-decided cycles to the host (one stream
// synchronization); a no-op when nothing is pending.
int pull_device_trace(ntvs_ctx* c) {
    if (!c->dev_pending) return NTVS_OK;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->dev_pending = false;
    const int rc = check_device_error(c);
    if (rc != NTVS_OK) {   // the traces of the failed run stay zero; the host's ell is kept
        c->dstate_valid = false;
        return rc;
    }
    const int64_t nk = (int64_t)c->ell_trace.size() - c->pend_k0;
    const int64_t ns = (int64_t)c->tries_trace.size() - c->pend_s0;
    if (nk > 0)
        CUDA_TRY(cudaMemcpy(c->ell_trace.data() + c->pend_k0, c->dev_ell_tr + c->pend_k0, sizeof(int64_t) * nk,
                            cudaMemcpyDeviceToHost));
    if (ns > 0) {
        CUDA_TRY(cudaMemcpy(c->tries_trace.data() + c->pend_s0, c->dev_tries + c->pend_s0, sizeof(int32_t) * ns,
                            cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(c->acc_trace.data() + c->pend_s0, c->dev_acc + c->pend_s0, sizeof(int32_t) * ns,
                            cudaMemcpyDeviceToHost));
    }
    for (int64_t q = c->pend_s0; q < (int64_t)c->tries_trace.size(); ++q) {
        c->n_tries += c->tries_trace[q];
        c->n_accepted += c->acc_trace[q];
    }
    CUDA_TRY(cudaMemcpy(c->hll, &c->cstate->ell, sizeof(int64_t), cudaMemcpyDeviceToHost));
    c->ell_prev = c->hll[0];
    c->dstate_valid = true;
    return NTVS_OK;
}

// Device-side set-up before k_iters checked cycles: trace capacity, the step-size table of
// the current (beta0, alpha), and the device ell when the host holds the current one.
int prepare_device_check(ntvs_ctx* c, int k_iters) {
    const int64_t need_k = (int64_t)c->ell_trace.size() + k_iters;
    const int64_t need_s = (int64_t)c->tries_trace.size() + (int64_t)k_iters * c->p.N;
    if (need_k > c->dtr_cap_k || need_s > c->dtr_cap_s) {
        TRY(pull_device_trace(c));   // nothing pending: the old buffers need no copy
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        int64_t ck = std::max<int64_t>(c->dtr_cap_k, 1024), cs = std::max<int64_t>(c->dtr_cap_s, 4096);
        while (ck < need_k) ck *= 2;
        while (cs < need_s) cs *= 2;
        dev_free(c->dev_ell_tr);
        dev_free(c->dev_tries);
        dev_free(c->dev_acc);
        c->dtr_cap_k = c->dtr_cap_s = 0;
        TRY(dev_alloc(&c->dev_ell_tr, sizeof(int64_t) * (size_t)ck, "ell trace"));
        TRY(dev_alloc(&c->dev_tries, sizeof(int32_t) * (size_t)cs, "tries trace"));
        TRY(dev_alloc(&c->dev_acc, sizeof(int32_t) * (size_t)cs, "accept trace"));
        c->dtr_cap_k = ck;
        c->dtr_cap_s = cs;
    }
    if (c->tab_beta0 != c->p.beta0 || c->tab_alpha != c->p.alpha) {
        CUDA_TRY(cudaStreamSynchronize(c->stream));   // the table may still be read by queued work
        std::vector<double> tab(kBetaTab);
        for (int l = 0; l < kBetaTab; ++l) tab[l] = step_beta(c->p, 0, 0, l);
        CUDA_TRY(cudaMemcpy(c->beta_tab, tab.data(), sizeof(double) * kBetaTab, cudaMemcpyHostToDevice));
        c->tab_beta0 = c->p.beta0;
        c->tab_alpha = c->p.alpha;
    }
    if (!c->dstate_valid) {
        c->hll[0] = c->ell_prev;
        CUDA_TRY(cudaMemcpyAsync(&c->cstate->ell, c->hll, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        c->dstate_valid = true;
    }
    if (!c->dev_pending) {
        c->pend_k0 = (int64_t)c->ell_trace.size();
        c->pend_s0 = (int64_t)c->tries_trace.size();
        c->dev_pending = true;
    }
    return NTVS_OK;
}

// N checked steps of cycle k with every decision on the device (ell drawn at cycle start
// by the caller): per step the gradient pass and one cooperative retry loop.
int perturb_steps_device(ntvs_ctx* c) {
    for (int n = 0; n < c->p.N; ++n) {
        TRY(launch_grad(c, true));
        const int64_t sidx = (int64_t)c->tries_trace.size();
        CheckLoopArgs a;
        a.cdt = c->cdt;
        a.x = c->x;
        a.copies = c->copies();
        a.g = c->g;
        a.gnorm2 = c->dscal + 0;
        a.phi_x = c->dscal + 1;
        a.st = c->cstate;
        a.beta_tab = c->beta_tab;
        a.tab_len = kBetaTab;
        a.beta0 = c->p.beta0;
        a.alpha = c->p.alpha;
        a.max_retries = c->p.max_retries;
        a.partials = c->red.partials;
        a.grid = std::max(1, std::min(c->red.grid, c->check_grid));
        a.err = c->derr;
        a.wait_ns = c->wait_ns;
        a.starve = (c->hook_flags & NTVS_HOOK_STARVE_CHECK) ? 1 : 0;
        a.tries_out = c->dev_tries + sidx;
        a.acc_out = c->dev_acc + sidx;
        a.nx = c->nx;
        a.ny = c->ny;
        a.nz = c->nz;
        CUDA_TRY(timed_launch(c, KIND_TV, [&] { return k_tv_check_loop(a, c->stream); }));
        c->tries_trace.push_back(0);   // filled by pull_device_trace
        c->acc_trace.push_back(0);
        c->n_steps += 1;
    }
    return NTVS_OK;
}

int perturb_steps(ntvs_ctx* c, int64_t* ell_io) {
    int64_t ell = *ell_io;
    const int N = c->p.N;
    const int64_t adv = ell_advances(c->p) ? 1 : 0;
    for (int n = 0; n < N; ++n) {
        double beta = step_beta(c->p, c->k, n, ell);
        int tries = 0, acc = 0;
        if (!c->p.tv_check) {
            TRY(launch_grad(c, false));
            CUDA_TRY(timed_launch(c, KIND_TV, [&] {
                return k_tv_apply(c->cdt, c->x, c->copies(), c->g, c->dscal + 0, beta, nullptr, c->V, c->stream);
            }));
            ell += adv;
            tries = 1;
            acc = 1;
        } else {
            TRY(launch_grad(c, true));
            for (;;) {
                int a = 0;
                TRY(checked_try(c, beta, &a));
                ell += adv;
                tries += 1;
                if (a) { acc = 1; break; }
                if (tries >= c->p.max_retries) break;
                beta = step_beta(c->p, c->k, n, ell);
            }
        }
        c->tries_trace.push_back(tries);
        c->acc_trace.push_back(acc);
        c->n_steps += 1;
        c->n_tries += tries;
        c->n_accepted += acc;
    }
    *ell_io = ell;
    return NTVS_OK;
}

// ---- block-DROP ------------------------------------------------------------------------
// Launches the DROP gather + scatter kernel of rows [r0, r1) of block t into delta
// (nothing applied), its residual sum of squares into *resid.  The whole block runs the
// context's schedule; a proper sub-range of it runs the plain schedule (the windowed and
// pipelined plans cover whole blocks).  *wb / *wo receive the block's window-scale slots
// for the apply kernel (null when the schedule has none).
int launch_drop_kernel(ntvs_ctx* c, int t, int64_t r0, int64_t r1, double* resid, float** wb, float** wo) {
    *wb = *wo = nullptr;
    if (r1 <= r0) return NTVS_OK;
    const bool whole = r0 == c->block_ptr[t] && r1 == c->block_ptr[t + 1];
    if (c->paths_mode) {
        CUDA_TRY(timed_launch(c, KIND_DROP, [&] {
            return k_otf_drop(c->otf, r0, r1, (const float*)c->inv_norm2, c->x32, (float*)c->delta, c->p.lambda,
                              resid, c->stream);
        }));
        return NTVS_OK;
    }
    DropArgs a;
    a.row_ptr = c->row_ptr;
    a.col = c->drop_cols();
    a.val = c->val;
    a.b = c->b;
    a.inv_norm2 = c->inv_norm2;
    a.r0 = r0;
    a.r1 = r1;
    a.x = (c->cdt == F64) ? (const void*)c->x : (const void*)c->x32;
    a.delta = c->delta;
    a.lambda = c->p.lambda;
    a.resid_ss = resid;
    a.vdt = c->vdt;
    a.cdt = c->cdt;
    a.lanes_per_row = c->lpr;
    a.grid = c->drop_grid;
    a.vector4 = c->vector4;
    a.use_d16 = c->storage == NTVS_DELTA16;
    a.d16 = c->d16();
    a.segs = nullptr;
    a.seg_begin = nullptr;
    a.slice = c->vm.slice_p;
    a.wlmax = nullptr;
    a.wbound = nullptr;
    a.wobs = nullptr;
    a.wamax = nullptr;
    a.max_row = t < (int)c->block_maxrow.size() ? c->block_maxrow[t] : (int64_t)1 << 40;
    if (whole && c->schedule == NTVS_SCHED_WINDOW) {
        a.segs = c->segs;
        a.seg_begin = c->seg_begin + (size_t)t * (c->win_grid + 1);
        a.grid = c->win_grid;
        if (c->wstat) {
            a.wlmax = c->wstat + t;
            a.wbound = *wb = c->wstat + c->B + t;
            a.wobs = *wo = c->wstat + 2 * c->B + t;
            a.wamax = c->wstat + 3 * c->B + 2 * t + 1;
        }
    }
    if (whole && c->schedule == NTVS_SCHED_PIPELINE) {
        DropPipeArgs pa;
        pa.row_ptr = c->row_ptr;
        pa.col = c->drop_cols();
        pa.val = c->val;
        pa.b = c->b;
        pa.inv_norm2 = c->inv_norm2;
        pa.stages = c->stages;
        pa.stage_begin = c->stage_begin + (size_t)t * (c->win_grid + 1);
        pa.slice = c->vm.slice_p;
        pa.x = a.x;
        pa.delta = c->delta;
        pa.lambda = c->p.lambda;
        pa.resid_ss = resid;
        pa.err = c->derr;
        pa.wait_ns = c->wait_ns;
        pa.starve = (c->hook_flags & NTVS_HOOK_STARVE_PIPE) ? 1 : 0;
        pa.vdt = c->vdt;
        pa.cdt = c->cdt;
        pa.grid = c->win_grid;
        pa.use_d16 = c->storage == NTVS_DELTA16;
        pa.d16 = c->d16();
        CUDA_TRY(timed_launch(c, KIND_DROP, [&] { return k_drop_pipe(pa, c->stream); }));
    } else {
        CUDA_TRY(timed_launch(c, KIND_DROP, [&] { return k_drop_block(a, c->stream); }));
    }
    return NTVS_OK;
}

// One block-DROP step: this context's rows of block t into delta, the sum over ranks
// through the all-reduce callback when one is set (row-sharded reconstruction), then
// x += delta / s^t.
int drop_block(ntvs_ctx* c, int t) {
    const int64_t r0 = c->block_ptr[t], r1 = c->block_ptr[t + 1];
    // the split copies of x are written by the last block of a sweep only (the TV gradient
    // reads them next); after any other block they are marked stale
    const bool split = t == c->B - 1;
    CUDA_TRY(cudaMemsetAsync(c->resid + t, 0, sizeof(double), c->stream));
    if (r1 <= r0 && !c->ar_fn) return NTVS_OK;
    float* wb = nullptr;
    float* wo = nullptr;
    TRY(launch_drop_kernel(c, t, r0, r1, c->resid + t, &wb, &wo));
    if (c->ar_fn) {
        int rc = c->ar_fn(c->delta, c->vm.vint, c->cdt, (void*)c->stream, c->ar_user);
        if (rc == 0) rc = c->ar_fn(c->resid + t, 1, NTVS_F64, (void*)c->stream, c->ar_user);
        if (rc != 0)
            return fail(NTVS_ERR_CUDA, "the all-reduce callback failed on block " + std::to_string(t) + " (returned " +
                                           std::to_string(rc) + ")");
    }
    CUDA_TRY(timed_launch(c, KIND_APPLY, [&] {
        return k_drop_apply(c->cdt, c->x, c->copies(split), c->delta,
                            (const char*)c->inv_s + (size_t)t * c->vm.vint * c->csz(), c->V, c->apply_grid, wb, wo,
                            c->stream);
    }));
    c->split_stale = !split;
    return NTVS_OK;
}

int drop_sweep(ntvs_ctx* c) {
    for (int t = 0; t < c->B; ++t) TRY(drop_block(c, t));
    return NTVS_OK;
}

// copy V values of device type sdt into `out` (dtype F64/F32, host or device)
int copy_image_out(ntvs_ctx* c, const void* src, int sdt, void* out, int dtype, int mem_kind) {
    if (dtype != NTVS_F64 && dtype != NTVS_F32) return fail(NTVS_ERR_ARG, "image dtype must be NTVS_F64 or NTVS_F32");
    if (!out && c->V) return fail(NTVS_ERR_ARG, "null output");
    if (mem_kind == NTVS_MEM_DEVICE) {
        CUDA_TRY(k_convert(src, sdt, out, dtype, c->V, c->stream));
        return NTVS_OK;
    }
    if (mem_kind != NTVS_MEM_HOST) return fail(NTVS_ERR_ARG, "bad mem_kind");
    if (dtype == sdt) {
        CUDA_TRY(cudaMemcpyAsync(out, src, (size_t)c->V * dt_size(sdt), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        return NTVS_OK;
    }
    std::vector<unsigned char> tmp((size_t)c->V * dt_size(sdt));
    CUDA_TRY(cudaMemcpyAsync(tmp.data(), src, tmp.size(), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (sdt == NTVS_F64) {
        const double* s = (const double*)tmp.data();
        float* d = (float*)out;
        for (int64_t j = 0; j < c->V; ++j) d[j] = (float)s[j];
    } else {
        const float* s = (const float*)tmp.data();
        double* d = (double*)out;
        for (int64_t j = 0; j < c->V; ++j) d[j] = (double)s[j];
    }
    return NTVS_OK;
}

}  // namespace

// ---- DELTA16 packing (load time) -----------------------------------------------------------
// Escaped chunks are counted on the device, then offsets, chunk bases, the escape table and
// the row flags are written (escape slots handed out by an atomic counter: their order does
// not matter); int32 columns that the context owns are released afterwards.
static int pack_delta16(ntvs_ctx* c) {
    const int64_t nnz = c->nnz, nch = delta16_slots(nnz, c->M);
    unsigned long long* ctr = nullptr;
    TRY(dev_alloc(&ctr, 2 * sizeof(unsigned long long), "DELTA16 counters"));
    struct Free {
        unsigned long long*& p;
        ~Free() { dev_free(p); }
    } guard{ctr};
    unsigned long long n_esc = 0;
    CUDA_TRY(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), c->stream));
    CUDA_TRY(k_delta16_count(c->row_ptr, c->col, c->M, ctr, c->stream));
    CUDA_TRY(cudaMemcpyAsync(&n_esc, ctr, sizeof(n_esc), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    TRY(dev_alloc(&c->d16off, sizeof(uint16_t) * (size_t)std::max<int64_t>(nnz, 8), "DELTA16 offsets"));
    TRY(dev_alloc(&c->d16base, sizeof(int32_t) * (size_t)std::max<int64_t>(nch, 1), "DELTA16 chunk bases"));
    TRY(dev_alloc(&c->d16exc, sizeof(int32_t) * 32 * (size_t)std::max<unsigned long long>(n_esc, 1),
                  "DELTA16 escaped chunks"));
    c->n_escaped = (int64_t)n_esc;
    TRY(dev_alloc(&c->d16rowesc, (size_t)std::max<int64_t>(c->M, 1), "DELTA16 row flags"));
    CUDA_TRY(k_delta16_fill(c->row_ptr, c->col, c->M, c->d16off, c->d16base, c->d16exc, c->d16rowesc, ctr + 1,
                            c->stream));
    if (dt_size(c->vdt) == 2) {   // 16-bit values: offset and value bits in one word per entry
        TRY(dev_alloc(&c->d16word, sizeof(uint32_t) * (size_t)std::max<int64_t>(nnz, 4), "DELTA16 words"));
        CUDA_TRY(k_pack_words(c->d16off, (const uint16_t*)c->val, nnz, c->d16word, c->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->own_col) {
        dev_free(c->col);
        c->own_col = false;
    }
    c->col = nullptr;
    if (c->d16word) {
        dev_free(c->d16off);
        if (c->own_val) dev_free(c->val);
        c->val = nullptr;
        c->own_val = false;
    }
    return NTVS_OK;
}

// ---- DROP schedule planning (load time) ------------------------------------------------
// Each block's rows are cut into chunks of kChunkRows consecutive rows; a chunk's home
// slice is the median of its rows' home slices (so a few rows that bend out of their
// slice do not break a run).  Per block, chunks are ordered by home slice and dealt to the
// win_grid CTAs in contiguous runs of about equal work; consecutive chunks of one CTA with
// the same home slice and adjacent rows merge into one segment.  A chunk's work is counted
// in the register steps its rows issue (k_chunk_cost): a row costs the depth of the body
// it runs, not its entry count, since every step of a body issues whether or not it holds
// entries (measured: the busiest SM's excess over the mean follows this count); a step
// past the row's end issues predicated off and counts a quarter of a live one.
constexpr int kChunkRows = 64;
constexpr double kMinMeanRun = 8.0;

static int plan_schedule(ntvs_ctx* c, int requested) {
    c->schedule = NTVS_SCHED_PLAIN;
    if (requested == NTVS_SCHED_PLAIN || c->M == 0) return NTVS_OK;
    const int64_t slice = c->vm.slice_p;
    int optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    // the window and the row stage plus the kernel's static shared memory (reductions)
    const int64_t need = k_window_smem_bytes(slice, c->csz(), c->storage == NTVS_DELTA16) + 9 * 1024;
    if (need > optin) {
        if (requested == NTVS_SCHED_WINDOW || requested == NTVS_SCHED_PIPELINE)
            return fail(NTVS_ERR_ARG, "windowed schedule: an nx*ny slice needs " + std::to_string(need) +
                                          " bytes of shared memory, the device allows " + std::to_string(optin));
        return NTVS_OK;
    }
    // home slice of every row, then on the device the median home of every chunk of
    // kChunkRows rows (chunks restart at each block) and the number of home changes
    // between consecutive rows; only the chunk medians come back to the host
    std::vector<int64_t> cstart;
    std::vector<int64_t> block_chunk(c->B + 1, 0);
    for (int t = 0; t < c->B; ++t) {
        block_chunk[t] = (int64_t)cstart.size();
        for (int64_t i = c->block_ptr[t]; i < c->block_ptr[t + 1]; i += kChunkRows) cstart.push_back(i);
    }
    block_chunk[c->B] = (int64_t)cstart.size();
    const int64_t nch = (int64_t)cstart.size();
    cstart.push_back(c->M);
    // the register depth of every chunk's block body (0: rows are counted instead)
    std::vector<int8_t> chunk_ch((size_t)std::max<int64_t>(nch, 1), 0);
    for (int t = 0; t < c->B; ++t) {
        const int64_t mr = t < (int)c->block_maxrow.size() ? c->block_maxrow[t] : 0;
        const int8_t d = (int8_t)window_register_steps(mr, c->cdt, c->vdt, c->lpr);
        for (int64_t q = block_chunk[t]; q < block_chunk[t + 1]; ++q) chunk_ch[(size_t)q] = d;
    }
    // the planning's device temporaries in one allocation (each free synchronizes the device)
    const size_t nchp = (size_t)std::max<int64_t>(nch, 1);
    auto up256 = [](size_t n) { return (n + 255) & ~(size_t)255; };
    const size_t o_home = 0, o_chunk = o_home + up256(sizeof(int32_t) * (size_t)c->M);
    const size_t o_start = o_chunk + up256(sizeof(int32_t) * nchp);
    const size_t o_changes = o_start + up256(sizeof(int64_t) * cstart.size());
    const size_t o_ch = o_changes + up256(sizeof(unsigned long long));
    const size_t o_cost = o_ch + up256(chunk_ch.size());
    const size_t scratch_bytes = o_cost + up256(sizeof(int64_t) * nchp);
    char* scratch = nullptr;
    TRY(dev_alloc(&scratch, scratch_bytes, "schedule planning scratch"));
    struct FreeScratch {
        char*& p;
        ~FreeScratch() { dev_free(p); }
    } scratch_guard{scratch};
    int32_t* dhome = reinterpret_cast<int32_t*>(scratch + o_home);
    int32_t* dchunk = reinterpret_cast<int32_t*>(scratch + o_chunk);
    int64_t* dstart = reinterpret_cast<int64_t*>(scratch + o_start);
    unsigned long long* dchanges = reinterpret_cast<unsigned long long*>(scratch + o_changes);
    int8_t* dch = reinterpret_cast<int8_t*>(scratch + o_ch);
    int64_t* dcost = reinterpret_cast<int64_t*>(scratch + o_cost);
    std::vector<int32_t> chome((size_t)nch);
    std::vector<int64_t> ccost((size_t)nch);
    unsigned long long changes = 0;
    cudaError_t e = cudaMemcpyAsync(dstart, cstart.data(), sizeof(int64_t) * cstart.size(), cudaMemcpyHostToDevice,
                                    c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dch, chunk_ch.data(), chunk_ch.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dchanges, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess)   // the columns of the packed pairs when there are any (col may be gone)
        e = k_row_home(c->row_ptr, c->ent ? c->ent : c->col, c->ent ? 2 : 1, c->M, slice, dhome, c->sms * 8, c->stream);
    if (e == cudaSuccess) e = k_chunk_home(dhome, dstart, nch, dchunk, dchanges, c->sms * 8, c->stream);
    // the middle body: every CSR32 row, and the narrow DELTA16 rows (90 % of the benchmark's;
    // the others run the block's depth, which the count slightly underestimates)
    const int mid_body = kMidBody;
    if (e == cudaSuccess) e = k_chunk_cost(c->row_ptr, dstart, dch, mid_body, nch, dcost, c->sms * 8, c->stream);
    if (e == cudaSuccess && nch > 0)
        e = cudaMemcpyAsync(chome.data(), dchunk, sizeof(int32_t) * (size_t)nch, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && nch > 0)
        e = cudaMemcpyAsync(ccost.data(), dcost, sizeof(int64_t) * (size_t)nch, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&changes, dchanges, sizeof(changes), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(NTVS_ERR_CUDA, cuda_msg("row home slices", e));
    int32_t last = 0;
    for (auto& h : chome) {   // chunks of empty rows join their predecessor's run
        if (h < 0) h = last;
        last = h;
    }
    // mean run length of equal home slices in stored order
    const double mean_run = (double)c->M / (double)(changes + 1);
    if (requested == NTVS_SCHED_AUTO && mean_run < kMinMeanRun) return NTVS_OK;

    const int G = c->sms;
    struct Chunk { int64_t r0, r1; int32_t home; int64_t cost; };
    std::vector<DropSegment> segs;
    std::vector<int32_t> begin((size_t)c->B * (G + 1), 0);
    std::vector<Chunk> ch;
    for (int t = 0; t < c->B; ++t) {
        ch.clear();
        int64_t total = 0;   // the block's work (at least one unit per row, as a guard)
        for (int64_t q = block_chunk[t]; q < block_chunk[t + 1]; ++q) {
            const int64_t w = std::max<int64_t>(ccost[(size_t)q], cstart[q + 1] - cstart[q]);
            ch.push_back({cstart[q], cstart[q + 1], chome[q], w});
            total += w;
        }
        std::stable_sort(ch.begin(), ch.end(), [](const Chunk& a, const Chunk& b) { return a.home < b.home; });
        int32_t* bg = begin.data() + (size_t)t * (G + 1);
        int cta = 0;
        bg[0] = (int32_t)segs.size();
        int64_t cum = 0;
        for (const Chunk& k : ch) {
            const int owner = total > 0 ? (int)std::min<int64_t>(G - 1, (cum * G) / total) : 0;
            while (cta < owner) bg[++cta] = (int32_t)segs.size();
            const bool own_last = (int64_t)segs.size() > bg[cta];
            if (own_last && segs.back().home == k.home && segs.back().r1 == k.r0) segs.back().r1 = k.r1;
            else segs.push_back({k.r0, k.r1, k.home, 0});
            cum += k.cost;
        }
        while (cta < G) bg[++cta] = (int32_t)segs.size();
    }
    if (segs.size() > (size_t)INT32_MAX) return NTVS_OK;
    c->win_grid = G;

    // pipelined schedule: cut every segment into ring-slot stages of whole rows
    const bool d16 = c->storage == NTVS_DELTA16;
    const int64_t vsz = (int64_t)dt_size(c->vdt);
    // one array per entry (packed pairs, DELTA16 words) or an index array beside the values
    const bool packed = !d16 && c->vdt == F32, words = d16 && vsz == 2;
    const int64_t idx_bytes = packed ? 8 : words ? 4 : d16 ? 2 : 4;
    const int ring_bytes = (int)((packed || words) ? idx_bytes : idx_bytes + vsz);
    // DELTA16 columns, words and packed pairs are buffers of our own (aligned); the int32
    // columns and the values may be borrowed
    const bool aligned = packed || words || ((d16 || (uintptr_t)c->col % 16 == 0) && ((uintptr_t)c->val % 16 == 0));
    const bool pipe_fits = (int64_t)pipe_smem_bytes(c->cdt, ring_bytes, slice) + 1024 <= optin;
    // AUTO takes the windowed kernel (measured faster than the pipelined one on the
    // 200x200x16 workload); the pipelined one only on request
    const bool want_pipe = requested == NTVS_SCHED_PIPELINE;
    if (want_pipe) {
        if (c->nz > 32767) return fail(NTVS_ERR_ARG, "pipelined schedule: nz > 32767");
        if (!aligned || !pipe_fits) {
            return fail(NTVS_ERR_ARG, !aligned ? "pipelined schedule: col and val must be 16-byte aligned"
                                               : "pipelined schedule: slice window + ring exceed shared memory");
        }
        std::vector<int64_t> rp((size_t)c->M + 1);
        CUDA_TRY(cudaMemcpyAsync(rp.data(), c->row_ptr, sizeof(int64_t) * rp.size(), cudaMemcpyDeviceToHost,
                                 c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        const int64_t S = pipe_stage_entries(ring_bytes);
        const int64_t nnz_all = rp[c->M];
        // entries per 16 bytes of the single array, or of both the index and the value arrays
        const int64_t A = (packed || words) ? 16 / idx_bytes : 16 / std::min<int64_t>(idx_bytes, vsz);
        auto down = [&](int64_t e) { return (e / A) * A; };
        auto up = [&](int64_t e) { return ((e + A - 1) / A) * A; };
        std::vector<DropStage> stages;
        std::vector<int32_t> sbeg((size_t)c->B * (G + 1), 0);
        for (int t = 0; t < c->B; ++t) {
            const int32_t* bg = begin.data() + (size_t)t * (G + 1);
            int32_t* sb = sbeg.data() + (size_t)t * (G + 1);
            for (int cta = 0; cta < G; ++cta) {
                sb[cta] = (int32_t)stages.size();
                for (int32_t q = bg[cta]; q < bg[cta + 1]; ++q) {
                    const DropSegment& sg = segs[q];
                    for (int64_t i = sg.r0; i < sg.r1;) {
                        DropStage st;
                        std::memset(&st, 0, sizeof(st));
                        st.r0 = i;
                        st.home = (int16_t)sg.home;
                        const int64_t e0 = down(rp[i]);
                        int64_t j = i;
                        // a stage's aligned copy never reaches past the last entry (the arrays
                        // may be the caller's, sized exactly): a row that would is read from
                        // global memory by the consumers
                        while (j < sg.r1 && j - i < kStageRows && up(rp[j + 1]) - e0 <= S && up(rp[j + 1]) <= nnz_all)
                            ++j;
                        if (j == i) {   // one row longer than a slot: consumers read it from global memory
                            st.e0 = rp[i];
                            st.nent = 0;
                            st.nrows = 1;
                            i += 1;
                        } else {
                            st.e0 = e0;
                            st.nent = (int32_t)(up(rp[j]) - e0);
                            st.nrows = (int16_t)(j - i);
                            for (int64_t k = 0; k <= j - i; ++k) st.off[k] = (uint16_t)(rp[i + k] - e0);
                            i = j;
                        }
                        stages.push_back(st);
                    }
                }
            }
            sb[G] = (int32_t)stages.size();
        }
        if (stages.size() > (size_t)INT32_MAX) return fail(NTVS_ERR_ARG, "too many pipeline stages");
        for (const DropStage& st : stages)
            if (st.nent > 0 && st.e0 + st.nent > nnz_all)
                return fail(NTVS_ERR_ARG, "pipelined schedule: a stage reaches past the last entry");
        TRY(dev_alloc(&c->stages, sizeof(DropStage) * std::max<size_t>(stages.size(), 1), "DROP stages"));
        TRY(dev_alloc(&c->stage_begin, sizeof(int32_t) * sbeg.size(), "DROP stage index"));
        CUDA_TRY(cudaMemcpyAsync(c->stages, stages.data(), sizeof(DropStage) * stages.size(), cudaMemcpyHostToDevice,
                                 c->stream));
        CUDA_TRY(cudaMemcpyAsync(c->stage_begin, sbeg.data(), sizeof(int32_t) * sbeg.size(), cudaMemcpyHostToDevice,
                                 c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        c->schedule = NTVS_SCHED_PIPELINE;
        return NTVS_OK;
    }

    TRY(dev_alloc(&c->segs, sizeof(DropSegment) * std::max<size_t>(segs.size(), 1), "DROP segments"));
    TRY(dev_alloc(&c->seg_begin, sizeof(int32_t) * begin.size(), "DROP segment index"));
    CUDA_TRY(cudaMemcpyAsync(c->segs, segs.data(), sizeof(DropSegment) * segs.size(), cudaMemcpyHostToDevice,
                             c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->seg_begin, begin.data(), sizeof(int32_t) * begin.size(), cudaMemcpyHostToDevice,
                             c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->schedule = NTVS_SCHED_WINDOW;
    return NTVS_OK;
}

// =========================================================================== C ABI
extern "C" {

const char* ntvs_version(void) { return "ntvs-gb300 0.1 (sm_103a)"; }

const char* ntvs_last_error(void) { return g_err.c_str(); }

int ntvs_create(ntvs_ctx** out, int device, void* cuda_stream) {
    if (!out) return fail(NTVS_ERR_ARG, "null output pointer");
    *out = nullptr;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(NTVS_ERR_ARG, "device index out of range");
    CUDA_TRY(cudaSetDevice(device));
    ntvs_ctx* c = new ntvs_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    if (c->sms < 1) c->sms = 1;
    int rc = NTVS_OK;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; return fail(NTVS_ERR_CUDA, cuda_msg("cudaStreamCreate", e)); }
        c->own_stream = true;
    }
    {
        cudaError_t e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) c->copy_stream = nullptr;
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->copy_stream2, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            c->copy_stream2 = nullptr;
            ntvs_destroy(c);
            return fail(NTVS_ERR_CUDA, cuda_msg("cudaStreamCreate", e));
        }
    }
    const int maxgrid = c->sms * 8;
    c->red.grid = 1;
    if ((rc = dev_alloc(&c->red.partials, sizeof(double) * 2 * (size_t)maxgrid, "reduction partials")) ||
        (rc = dev_alloc(&c->red.ticket, sizeof(unsigned), "reduction ticket")) ||
        (rc = dev_alloc(&c->dscal, sizeof(double) * 8, "scalars")) ||
        (rc = dev_alloc(&c->daccept, sizeof(int) * 4, "accept flag")) ||
        (rc = dev_alloc(&c->dflags, sizeof(int) * 4, "flags")) ||
        (rc = dev_alloc(&c->derr, sizeof(int), "error word")) ||
        (rc = dev_alloc(&c->cstate, sizeof(CheckState), "check state")) ||
        (rc = dev_alloc(&c->beta_tab, sizeof(double) * kBetaTab, "step-size table"))) {
        ntvs_destroy(c);
        return rc;
    }
    cudaError_t e1 = cudaMemsetAsync(c->red.ticket, 0, sizeof(unsigned), c->stream);
    cudaError_t e2 = cudaMemsetAsync(c->dscal, 0, sizeof(double) * 8, c->stream);
    if (e2 == cudaSuccess) e2 = cudaMemsetAsync(c->derr, 0, sizeof(int), c->stream);
    cudaError_t e3 = cudaHostAlloc((void**)&c->hscal, sizeof(double) * 8, cudaHostAllocDefault);
    cudaError_t e4 = cudaHostAlloc((void**)&c->hint, sizeof(int) * 4, cudaHostAllocDefault);
    if (e4 == cudaSuccess) e4 = cudaHostAlloc((void**)&c->hll, sizeof(int64_t) * 4, cudaHostAllocDefault);
    if (e4 == cudaSuccess) e4 = cudaMemsetAsync(c->cstate, 0, sizeof(CheckState), c->stream);
    cudaError_t e5 = cudaStreamSynchronize(c->stream);
    if (e1 || e2 || e3 || e4 || e5) {
        ntvs_destroy(c);
        return fail(NTVS_ERR_CUDA, "context set-up failed");
    }
    c->p.lambda = 1e-4;
    c->p.alpha = 0.75;
    c->p.beta0 = 1.0;
    c->p.eps_tv = 1e-8;
    c->p.N = 0;
    c->p.tv_check = 0;
    c->p.max_retries = 64;
    c->p.seed = 0;
    *out = c;
    return NTVS_OK;
}

int ntvs_destroy(ntvs_ctx* c) {
    if (!c) return NTVS_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    c->free_system();
    dev_free(c->red.partials);
    dev_free(c->red.ticket);
    dev_free(c->dscal);
    dev_free(c->daccept);
    dev_free(c->dflags);
    dev_free(c->derr);
    dev_free(c->tvhist);
    dev_free(c->cstate);
    dev_free(c->beta_tab);
    dev_free(c->dev_ell_tr);
    dev_free(c->dev_tries);
    dev_free(c->dev_acc);
    dev_free(c->ext);
    if (c->hll) cudaFreeHost(c->hll);
    for (auto& t : c->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->hscal) cudaFreeHost(c->hscal);
    if (c->hint) cudaFreeHost(c->hint);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->copy_stream2) cudaStreamDestroy(c->copy_stream2);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return NTVS_OK;
}

int ntvs_load_system(ntvs_ctx* c, const ntvs_system* s) {
    TRY(use_device(c));
    if (!s) return fail(NTVS_ERR_ARG, "null system");
    if (s->nx < 1 || s->ny < 1 || s->nz < 1) return fail(NTVS_ERR_ARG, "grid sizes must be >= 1");
    const int64_t V = (int64_t)s->nx * s->ny * s->nz;
    if (V > 0x7fffffffLL) return fail(NTVS_ERR_ARG, "V exceeds the int32 column range");
    if (s->n_rows < 0) return fail(NTVS_ERR_ARG, "n_rows < 0");
    if (s->val_dtype < NTVS_F64 || s->val_dtype > NTVS_BF16) return fail(NTVS_ERR_ARG, "bad val_dtype");
    if (s->mem_kind != NTVS_MEM_HOST && s->mem_kind != NTVS_MEM_DEVICE) return fail(NTVS_ERR_ARG, "bad mem_kind");
    if (s->storage != NTVS_CSR32 && s->storage != NTVS_DELTA16) return fail(NTVS_ERR_ARG, "bad storage");
    if (s->schedule < NTVS_SCHED_AUTO || s->schedule > NTVS_SCHED_PIPELINE) return fail(NTVS_ERR_ARG, "bad schedule");
    if (!s->row_ptr) return fail(NTVS_ERR_ARG, "null row_ptr");
    const int64_t M = s->n_rows;
    if (M > 0 && (!s->b)) return fail(NTVS_ERR_ARG, "null b");
    // block partition (host)
    std::vector<int64_t> bp;
    if (s->block_ptr) {
        if (s->n_blocks < 1) return fail(NTVS_ERR_ARG, "n_blocks must be >= 1 with block_ptr");
        bp.assign(s->block_ptr, s->block_ptr + s->n_blocks + 1);
        if (bp.front() != 0 || bp.back() != M) return fail(NTVS_ERR_ARG, "block_ptr must run from 0 to n_rows");
        for (int t = 0; t < s->n_blocks; ++t)
            if (bp[t] > bp[t + 1]) return fail(NTVS_ERR_ARG, "block_ptr decreases");
    } else {
        if (s->n_blocks < 1) return fail(NTVS_ERR_ARG, "n_blocks must be >= 1");
        const int64_t per = (M + s->n_blocks - 1) / s->n_blocks;
        bp.resize((size_t)s->n_blocks + 1);
        for (int t = 0; t <= s->n_blocks; ++t) bp[t] = std::min<int64_t>((int64_t)t * per, M);
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->free_system();
    c->nx = s->nx; c->ny = s->ny; c->nz = s->nz;
    c->V = V;
    c->M = M;
    c->B = (int)bp.size() - 1;
    c->block_ptr = bp;
    c->vdt = s->val_dtype;
    c->cdt = (s->val_dtype == NTVS_F64 || (s->val_dtype == NTVS_F32 && c->compute_req == F64)) ? F64 : F32;
    c->storage = s->storage;
    // the FP64 path gathers the canonical master image: no internal order there; the FP32
    // path's order carries the slice windows' slot swizzle
    if (c->cdt == F32) {
        c->vm = make_voxmap(s->nx, s->ny, s->nz, c->tile_req_x, c->tile_req_y, true);
        if (c->vm.vint > 0x7fffffffLL) c->vm = make_voxmap(s->nx, s->ny, s->nz, 1, 1, true);
    } else {
        c->vm = make_voxmap(s->nx, s->ny, s->nz, 1, 1);
    }
    if (c->vm.vint > 0x7fffffffLL) c->vm = make_voxmap(s->nx, s->ny, s->nz, 1, 1);
    const bool reordered = voxmap_reorders(c->vm);
    const int64_t VI = c->vm.vint;
    cudaStream_t st = c->stream;

    // row_ptr and nnz
    int64_t nnz = 0;
    if (s->mem_kind == NTVS_MEM_HOST) {
        nnz = s->row_ptr[M];
    } else {
        CUDA_TRY(cudaMemcpyAsync(c->hscal, s->row_ptr + M, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        std::memcpy(&nnz, c->hscal, sizeof(int64_t));
    }
    if (nnz < 0) return fail(NTVS_ERR_CSR, "row_ptr[n_rows] < 0");
    if (nnz > 0 && (!s->col || !s->val)) return fail(NTVS_ERR_ARG, "null col or val");
    c->nnz = nnz;
    const size_t vsz = dt_size(c->vdt), csz = c->csz();
    TRY(copy_in((void**)&c->row_ptr, &c->own_row_ptr, s->row_ptr, sizeof(int64_t) * (size_t)(M + 1), s->mem_kind, st,
                "row_ptr"));
    if (dt_size(c->vdt) == csz || c->vdt != NTVS_F32) {
        TRY(copy_in(&c->b, &c->own_b, s->b, csz * (size_t)M, s->mem_kind, st, "b"));
    } else {   // FP64 arithmetic on FP32 storage: b arrives as float and is widened once
        TRY(dev_alloc(&c->b, sizeof(double) * (size_t)M, "b (FP64)"));
        c->own_b = true;
        if (M > 0 && s->mem_kind == NTVS_MEM_DEVICE) {
            CUDA_TRY(k_convert(s->b, F32, c->b, F64, M, st));
        } else if (M > 0) {
            std::vector<double> tmp((size_t)M);
            const float* bf = (const float*)s->b;
            for (int64_t i = 0; i < M; ++i) tmp[(size_t)i] = (double)bf[i];
            CUDA_TRY(cudaMemcpyAsync(c->b, tmp.data(), sizeof(double) * (size_t)M, cudaMemcpyHostToDevice, st));
            CUDA_TRY(cudaStreamSynchronize(st));
        }
    }
    // Host arrays: col and val are copied block by block on the copy stream, and each
    // block's preparation (on the context's stream) starts once its entries have arrived,
    // so the preparation hides behind the host-to-device copy.  Block t's entry range
    // comes from the host row_ptr, clamped to [0, nnz); a row_ptr that is not
    // non-decreasing is rejected below before any block is prepared.
    const bool piped = s->mem_kind == NTVS_MEM_HOST && nnz > 0 && c->copy_stream && c->copy_stream2;
    // CSR32 storage with FP32 values from host arrays: the blocks pass through a ring of
    // kLoadRing block-sized device slots on their way into the packed pairs, so that the
    // separate column and value arrays are neither allocated nor freed (the copy of block
    // t + kLoadRing waits until block t has been prepared and packed)
    const bool ring = piped && c->storage == NTVS_CSR32 && c->vdt == F32;
    constexpr int kLoadRing = 3;
    std::vector<cudaEvent_t> arrived, freed;
    std::vector<int64_t> eb;   // [B+1] entry range of each block (piped)
    struct EventGuard {
        std::vector<cudaEvent_t>& v;
        ~EventGuard() { for (auto e : v) cudaEventDestroy(e); }
    } guard{arrived}, guard_freed{freed};
    int32_t* slot_c = nullptr;
    char* slot_v = nullptr;
    int64_t slot_cap = 0;
    int nslots = 0;
    struct SlotGuard {   // released once no copy or kernel can still touch the slots
        ntvs_ctx* c;
        int32_t*& sc;
        char*& sv;
        ~SlotGuard() {
            if (!sc && !sv) return;
            for (cudaStream_t q : {c->copy_stream, c->copy_stream2, c->stream})
                if (q) cudaStreamSynchronize(q);
            dev_free(sc);
            dev_free(sv);
        }
    } slot_guard{c, slot_c, slot_v};
    // block t's columns and values on the device: its slot, or its part of the whole arrays
    auto block_col = [&](int t) -> int32_t* {
        return ring ? slot_c + (size_t)(t % nslots) * (size_t)slot_cap : c->col + eb[t];
    };
    auto block_val = [&](int t) -> char* {
        return ring ? slot_v + (size_t)(t % nslots) * (size_t)slot_cap * vsz : (char*)c->val + vsz * (size_t)eb[t];
    };
    auto issue_copy = [&](int t) -> int {
        const int64_t n = eb[t + 1] - eb[t];
        if (ring && t >= nslots)
            for (cudaStream_t cs : {c->copy_stream, c->copy_stream2})
                CUDA_TRY(cudaStreamWaitEvent(cs, freed[(size_t)(t - nslots)], 0));
        if (n > 0) {
            CUDA_TRY(cudaMemcpyAsync(block_col(t), s->col + eb[t], sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice,
                                     c->copy_stream));
            CUDA_TRY(cudaMemcpyAsync(block_val(t), (const char*)s->val + vsz * (size_t)eb[t], vsz * (size_t)n,
                                     cudaMemcpyHostToDevice, c->copy_stream2));
        }
        for (cudaStream_t cs : {c->copy_stream, c->copy_stream2}) {
            cudaEvent_t ev;
            CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            arrived.push_back(ev);
            CUDA_TRY(cudaEventRecord(ev, cs));
        }
        return NTVS_OK;
    };
    if (piped) {
        eb.resize((size_t)c->B + 1);
        for (int t = 0; t <= c->B; ++t) {
            int64_t e = s->row_ptr[bp[t]];
            e = e < 0 ? 0 : (e > nnz ? nnz : e);
            eb[t] = t > 0 && e < eb[t - 1] ? eb[t - 1] : e;
        }
        eb[c->B] = nnz;
        if (ring) {
            for (int t = 0; t < c->B; ++t) slot_cap = std::max<int64_t>(slot_cap, eb[t + 1] - eb[t]);
            slot_cap = std::max<int64_t>(slot_cap, 1);
            nslots = std::min(kLoadRing, c->B);
            TRY(dev_alloc(&slot_c, sizeof(int32_t) * (size_t)slot_cap * (size_t)nslots, "column staging"));
            TRY(dev_alloc(&slot_v, vsz * (size_t)slot_cap * (size_t)nslots, "value staging"));
            for (int t = 0; t < nslots; ++t) TRY(issue_copy(t));
        } else {
            TRY(dev_alloc(&c->col, sizeof(int32_t) * (size_t)nnz, "col"));
            c->own_col = true;
            TRY(dev_alloc(&c->val, vsz * (size_t)nnz, "val"));
            c->own_val = true;
            for (int t = 0; t < c->B; ++t) TRY(issue_copy(t));
        }
    } else {
        TRY(copy_in((void**)&c->col, &c->own_col, s->col, sizeof(int32_t) * (size_t)nnz, s->mem_kind, st, "col"));
        TRY(copy_in(&c->val, &c->own_val, s->val, vsz * (size_t)nnz, s->mem_kind, st, "val"));
    }

    // validation; columns of the internal order are rewritten into a buffer of the context's
    // own (caller memory is never modified)
    CUDA_TRY(cudaMemsetAsync(c->dflags, 0, sizeof(int), st));
    if (reordered && nnz > 0 && !piped) {
        if (!c->own_col) {
            int32_t* mine = nullptr;
            TRY(dev_alloc(&mine, sizeof(int32_t) * (size_t)nnz, "col (internal order)"));
            CUDA_TRY(k_remap_cols(c->col, mine, nnz, c->vm, c->dflags, st));
            c->col = mine;
            c->own_col = true;
        } else {
            CUDA_TRY(k_remap_cols(c->col, c->col, nnz, c->vm, c->dflags, st));
        }
    }
    CUDA_TRY(k_validate_rows(c->row_ptr, M, c->dflags, st));
    CUDA_TRY(cudaMemcpyAsync(c->hint, c->dflags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (c->hint[0] & 3) {
        c->free_system();
        return fail(NTVS_ERR_CSR, (c->hint[0] & 2) ? "row_ptr[0] != 0" : "row_ptr decreases");
    }
    // one pass per block: entry / rhs validation, FP64 row norms, per-block hit counts
    TRY(dev_alloc(&c->inv_norm2, csz * (size_t)M, "inv_norm2"));
    int32_t* cnt = nullptr;
    TRY(dev_alloc(&cnt, sizeof(int32_t) * (size_t)c->B * VI, "hit counts"));
    CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)c->B * VI, st));
    // FP32 path: per-block scale statistics of the fixed-point DROP window (lmax = the
    // largest column sum of |a_ij|, the bound seeded with max_i |b_i| / ||a_i||^2)
    float* colsum = nullptr;
    struct FreeColsum {
        float*& p;
        ~FreeColsum() { dev_free(p); }
    } colsum_guard{colsum};
    if (c->cdt == F32) {
        TRY(dev_alloc(&c->wstat, sizeof(float) * 5 * (size_t)c->B, "window scale statistics"));
        CUDA_TRY(cudaMemsetAsync(c->wstat, 0, sizeof(float) * 5 * (size_t)c->B, st));
        TRY(dev_alloc(&colsum, sizeof(float) * (size_t)VI, "column sums"));
    }
    // CSR32 storage with FP32 values: every block's entries are packed into {column, value}
    // pairs once they are validated and remapped (during the copy of the later blocks)
    if (c->storage == NTVS_CSR32 && c->vdt == F32)
        TRY(dev_alloc(&c->ent, sizeof(int32_t) * 2 * (size_t)std::max<int64_t>(nnz, 1), "packed entries"));
    if (ring && !c->ent) return fail(NTVS_ERR_STATE, "staged load without packed entries");
    for (int t = 0; t < c->B; ++t) {
        // block t's entries: from entry e0 on at bc / bv (the whole arrays when not piped)
        int32_t* bc = c->col;
        const void* bv = c->val;
        int64_t e0 = 0;
        if (piped) {
            CUDA_TRY(cudaStreamWaitEvent(st, arrived[2 * (size_t)t], 0));
            CUDA_TRY(cudaStreamWaitEvent(st, arrived[2 * (size_t)t + 1], 0));
            bc = block_col(t);
            bv = block_val(t);
            e0 = eb[t];
            if (reordered) CUDA_TRY(k_remap_cols(bc, bc, eb[t + 1] - eb[t], c->vm, c->dflags, st));
        }
        if (colsum) CUDA_TRY(cudaMemsetAsync(colsum, 0, sizeof(float) * (size_t)VI, st));
        CUDA_TRY(k_prep_block(c->row_ptr, bc, bv, e0, c->vdt, c->b, bp[t], bp[t + 1], VI, c->inv_norm2, c->cdt,
                              cnt + (size_t)t * VI, c->dflags, colsum, colsum ? c->wstat + 3 * c->B + 2 * t : nullptr,
                              st));
        if (colsum) CUDA_TRY(k_colmax(colsum, VI, c->wstat + t, st));
        if (c->ent && piped)
            CUDA_TRY(k_pack_entries(bc, (const float*)bv, eb[t + 1] - eb[t], c->ent + 2 * eb[t], st));
        if (ring) {   // the slot is free again: the block nslots on may be copied into it
            cudaEvent_t ev;
            CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            freed.push_back(ev);
            CUDA_TRY(cudaEventRecord(ev, st));
            if (t + nslots < c->B) TRY(issue_copy(t + nslots));
        }
    }
    if (c->ent && !piped) CUDA_TRY(k_pack_entries(c->col, (const float*)c->val, nnz, c->ent, st));
    {   // longest row of every block
        unsigned long long* dm = nullptr;
        TRY(dev_alloc(&dm, sizeof(unsigned long long) * (size_t)c->B, "row lengths"));
        std::vector<unsigned long long> hm((size_t)c->B, 0);
        cudaError_t e = cudaMemsetAsync(dm, 0, sizeof(unsigned long long) * (size_t)c->B, st);
        for (int t = 0; t < c->B && e == cudaSuccess; ++t) e = k_row_maxlen(c->row_ptr, bp[t], bp[t + 1], dm + t, c->sms * 4, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hm.data(), dm, sizeof(unsigned long long) * (size_t)c->B, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        dev_free(dm);
        if (e != cudaSuccess) return fail(NTVS_ERR_CUDA, cuda_msg("row lengths", e));
        c->block_maxrow.assign(hm.begin(), hm.end());
    }
    if (c->wstat) {   // the first sweep's bound: max |b_i| / ||a_i||^2 (the residual at x = 0)
        std::vector<float> ws((size_t)5 * c->B);
        CUDA_TRY(cudaMemcpyAsync(ws.data(), c->wstat, sizeof(float) * ws.size(), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        for (int t = 0; t < c->B; ++t) ws[(size_t)c->B + t] = ws[(size_t)3 * c->B + 2 * t];
        CUDA_TRY(cudaMemcpyAsync(c->wstat, ws.data(), sizeof(float) * ws.size(), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    CUDA_TRY(cudaMemcpyAsync(c->hint, c->dflags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (c->hint[0]) {
        const int f = c->hint[0];
        dev_free(cnt);
        c->free_system();
        return fail(NTVS_ERR_CSR, (f & 4) ? "column index outside [0, V)" : (f & 8) ? "non-finite matrix value"
                                                                                    : "non-finite right-hand side");
    }
    TRY(dev_alloc(&c->inv_s, csz * (size_t)c->B * VI, "inverse hit counts"));
    CUDA_TRY(k_inv_counts(cnt, c->inv_s, c->cdt, (int64_t)c->B * VI, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    dev_free(cnt);

    // image state (x and g canonical; x32 and delta in the internal order, padding zero)
    TRY(dev_alloc(&c->x, sizeof(double) * (size_t)V, "x"));
    if (c->cdt == F32) {
        TRY(dev_alloc(&c->x32, sizeof(float) * (size_t)VI, "x32"));
        TRY(dev_alloc(&c->xh, sizeof(float) * (size_t)V, "xh"));
        TRY(dev_alloc(&c->xl, sizeof(float) * (size_t)V, "xl"));
    }
    TRY(dev_alloc(&c->delta, csz * (size_t)VI, "delta"));
    TRY(dev_alloc(&c->g, csz * (size_t)V, "g"));
    TRY(dev_alloc(&c->resid, sizeof(double) * (size_t)c->B, "residuals"));
    CUDA_TRY(cudaMemsetAsync(c->x, 0, sizeof(double) * (size_t)V, st));
    if (c->x32) CUDA_TRY(cudaMemsetAsync(c->x32, 0, sizeof(float) * (size_t)VI, st));
    if (c->xh) CUDA_TRY(cudaMemsetAsync(c->xh, 0, sizeof(float) * (size_t)V, st));
    if (c->xl) CUDA_TRY(cudaMemsetAsync(c->xl, 0, sizeof(float) * (size_t)V, st));
    CUDA_TRY(cudaMemsetAsync(c->delta, 0, csz * (size_t)VI, st));
    CUDA_TRY(cudaMemsetAsync(c->g, 0, csz * (size_t)V, st));
    CUDA_TRY(cudaMemsetAsync(c->resid, 0, sizeof(double) * (size_t)c->B, st));

    // launch shapes: lanes per row from the mean row length
    const double mean = M ? (double)nnz / (double)M : 0.0;
    c->lpr = mean <= 12.0 ? 4 : mean <= 40.0 ? 8 : mean <= 120.0 ? 16 : 32;
    c->drop_grid = c->sms * 8;
    // 4-entry vector loads put entries 4 apart along a path into one scatter instruction,
    // which measured slower than one coalesced entry per lane (2-entry loads too: 0.312
    // against 0.281 ms per 500k-row block); kept off
    c->vector4 = false;
    TRY(plan_schedule(c, s->schedule));
    if (c->storage == NTVS_DELTA16) TRY(pack_delta16(c));
    if (c->ent) {   // the pairs replace the column and value arrays (which the planning read)
        CUDA_TRY(cudaStreamSynchronize(st));
        if (c->own_col) dev_free(c->col);
        if (c->own_val) dev_free(c->val);
        c->col = nullptr;
        c->val = nullptr;
        c->own_col = c->own_val = false;
    }
    {
        const int64_t need = (V + 255) / 256;
        c->apply_grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)c->sms * 8));
    }
    c->red.grid = red_grid(V, c->sms);

    c->k = 0;
    c->ell_prev = 0;
    c->ell_trace.clear();
    c->tries_trace.clear();
    c->acc_trace.clear();
    c->n_steps = c->n_accepted = c->n_tries = 0;
    c->dev_pending = false;
    c->dstate_valid = false;
    c->check_grid = check_loop_max_grid(c->cdt, c->sms);
    c->ar_fn = nullptr;   // a new system starts with its own (local) hit counts
    c->ar_user = nullptr;
    CUDA_TRY(cudaStreamSynchronize(st));
    c->split_stale = false;
    c->loaded = true;
    return NTVS_OK;
}

int ntvs_load_paths(ntvs_ctx* c, const ntvs_paths* s) {
    TRY(use_device(c));
    if (!s) return fail(NTVS_ERR_ARG, "null paths");
    if (s->nx < 1 || s->ny < 1 || s->nz < 1) return fail(NTVS_ERR_ARG, "grid sizes must be >= 1");
    const int64_t V = (int64_t)s->nx * s->ny * s->nz;
    if (V > 0x7fffffffLL) return fail(NTVS_ERR_ARG, "V exceeds the int32 voxel range");
    if (!(s->dx > 0 && s->dy > 0 && s->dz > 0)) return fail(NTVS_ERR_ARG, "voxel sizes must be > 0");
    if (s->n_seg < 1 || s->n_seg > 64) return fail(NTVS_ERR_ARG, "n_seg must be in [1, 64]");
    if (!(s->min_len >= 0)) return fail(NTVS_ERR_ARG, "min_len must be >= 0");
    if (s->n_rows < 0) return fail(NTVS_ERR_ARG, "n_rows < 0");
    if (s->mem_kind != NTVS_MEM_HOST && s->mem_kind != NTVS_MEM_DEVICE) return fail(NTVS_ERR_ARG, "bad mem_kind");
    const int64_t M = s->n_rows;
    if (M > 0 && (!s->paths || !s->b)) return fail(NTVS_ERR_ARG, "null paths or b");
    std::vector<int64_t> bp;
    if (s->block_ptr) {
        if (s->n_blocks < 1) return fail(NTVS_ERR_ARG, "n_blocks must be >= 1 with block_ptr");
        bp.assign(s->block_ptr, s->block_ptr + s->n_blocks + 1);
        if (bp.front() != 0 || bp.back() != M) return fail(NTVS_ERR_ARG, "block_ptr must run from 0 to n_rows");
        for (int t = 0; t < s->n_blocks; ++t)
            if (bp[t] > bp[t + 1]) return fail(NTVS_ERR_ARG, "block_ptr decreases");
    } else {
        if (s->n_blocks < 1) return fail(NTVS_ERR_ARG, "n_blocks must be >= 1");
        const int64_t per = (M + s->n_blocks - 1) / s->n_blocks;
        for (int t = 0; t <= s->n_blocks; ++t) bp.push_back(std::min<int64_t>((int64_t)t * per, M));
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->free_system();
    cudaStream_t st = c->stream;
    c->nx = s->nx; c->ny = s->ny; c->nz = s->nz;
    c->V = V;
    c->M = M;
    c->B = (int)bp.size() - 1;
    c->block_ptr = bp;
    c->vdt = F32;
    c->cdt = F32;
    c->storage = NTVS_CSR32;
    c->nnz = 0;
    c->vm = make_voxmap(s->nx, s->ny, s->nz, c->tile_req_x, c->tile_req_y);
    if (c->vm.vint > 0x7fffffffLL) c->vm = make_voxmap(s->nx, s->ny, s->nz, 1, 1);
    const int64_t VI = c->vm.vint;
    TRY(copy_in((void**)&c->paths, &c->own_paths, s->paths, sizeof(float) * 10 * (size_t)M, s->mem_kind, st, "paths"));
    TRY(copy_in(&c->b, &c->own_b, s->b, sizeof(float) * (size_t)M, s->mem_kind, st, "b"));
    c->paths_mode = true;
    OtfArgs& o = c->otf;
    o.paths = c->paths;
    o.b = (const float*)c->b;
    o.M = M;
    o.nx = s->nx; o.ny = s->ny; o.nz = s->nz;
    o.dx = s->dx; o.dy = s->dy; o.dz = s->dz;
    o.n_seg = s->n_seg;
    o.min_len = (float)s->min_len;
    o.grid = c->sms * 8;
    o.vm = c->vm;
    CUDA_TRY(cudaMemsetAsync(c->dflags, 0, sizeof(int), st));
    CUDA_TRY(k_otf_validate(o, c->dflags, st));
    CUDA_TRY(cudaMemcpyAsync(c->hint, c->dflags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (c->hint[0]) {
        const int f = c->hint[0];
        c->free_system();
        return fail(NTVS_ERR_CSR, (f & 32) ? "non-finite path record" : "non-finite right-hand side");
    }
    TRY(dev_alloc(&c->inv_norm2, sizeof(float) * (size_t)std::max<int64_t>(M, 1), "inv_norm2"));
    int32_t* cnt = nullptr;
    TRY(dev_alloc(&cnt, sizeof(int32_t) * (size_t)c->B * VI, "hit counts"));
    CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)c->B * VI, st));
    for (int t = 0; t < c->B; ++t)
        CUDA_TRY(k_otf_prep(o, bp[t], bp[t + 1], (float*)c->inv_norm2, cnt + (size_t)t * VI, st));
    TRY(dev_alloc(&c->inv_s, sizeof(float) * (size_t)c->B * VI, "inverse hit counts"));
    CUDA_TRY(k_inv_counts(cnt, c->inv_s, F32, (int64_t)c->B * VI, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    dev_free(cnt);
    TRY(dev_alloc(&c->x, sizeof(double) * (size_t)V, "x"));
    TRY(dev_alloc(&c->x32, sizeof(float) * (size_t)VI, "x32"));
    TRY(dev_alloc(&c->xh, sizeof(float) * (size_t)V, "xh"));
    TRY(dev_alloc(&c->xl, sizeof(float) * (size_t)V, "xl"));
    TRY(dev_alloc(&c->delta, sizeof(float) * (size_t)VI, "delta"));
    TRY(dev_alloc(&c->g, sizeof(float) * (size_t)V, "g"));
    TRY(dev_alloc(&c->resid, sizeof(double) * (size_t)c->B, "residuals"));
    CUDA_TRY(cudaMemsetAsync(c->x, 0, sizeof(double) * (size_t)V, st));
    CUDA_TRY(cudaMemsetAsync(c->x32, 0, sizeof(float) * (size_t)VI, st));
    CUDA_TRY(cudaMemsetAsync(c->xh, 0, sizeof(float) * (size_t)V, st));
    CUDA_TRY(cudaMemsetAsync(c->xl, 0, sizeof(float) * (size_t)V, st));
    CUDA_TRY(cudaMemsetAsync(c->delta, 0, sizeof(float) * (size_t)VI, st));
    CUDA_TRY(cudaMemsetAsync(c->resid, 0, sizeof(double) * (size_t)c->B, st));
    c->lpr = 16;
    c->schedule = NTVS_SCHED_ONTHEFLY;
    {
        const int64_t need = (V + 255) / 256;
        c->apply_grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)c->sms * 8));
    }
    c->red.grid = red_grid(V, c->sms);
    c->k = 0;
    c->ell_prev = 0;
    c->ell_trace.clear();
    c->tries_trace.clear();
    c->acc_trace.clear();
    c->n_steps = c->n_accepted = c->n_tries = 0;
    c->dev_pending = false;
    c->dstate_valid = false;
    c->check_grid = check_loop_max_grid(c->cdt, c->sms);
    c->ar_fn = nullptr;   // a new system starts with its own (local) hit counts
    c->ar_user = nullptr;
    CUDA_TRY(cudaStreamSynchronize(st));
    c->split_stale = false;
    c->loaded = true;
    return NTVS_OK;
}

int ntvs_load_histories(ntvs_ctx* c, const ntvs_histories* h) {
    TRY(use_device(c));
    if (!h) return fail(NTVS_ERR_ARG, "null histories");
    if (h->n_rows < 0) return fail(NTVS_ERR_ARG, "n_rows < 0");
    if (h->mem_kind != NTVS_MEM_HOST && h->mem_kind != NTVS_MEM_DEVICE) return fail(NTVS_ERR_ARG, "bad mem_kind");
    const int64_t M = h->n_rows;
    if (M > 0 && (!h->hist || !h->b)) return fail(NTVS_ERR_ARG, "null hist or b");
    cudaStream_t st = c->stream;
    // device copies the context will own: the converted records and, for host input, b
    float* rec = nullptr;
    float* bdev = nullptr;
    float* hdev = nullptr;
    auto release = [&]() { dev_free(rec); dev_free(bdev); dev_free(hdev); };
    int rc = dev_alloc(&rec, sizeof(float) * 10 * (size_t)std::max<int64_t>(M, 1), "path records");
    const float* src = h->hist;
    const float* bsrc = h->b;
    if (rc == NTVS_OK && h->mem_kind == NTVS_MEM_HOST) {
        rc = dev_alloc(&hdev, sizeof(float) * 12 * (size_t)std::max<int64_t>(M, 1), "histories");
        if (rc == NTVS_OK) rc = dev_alloc(&bdev, sizeof(float) * (size_t)std::max<int64_t>(M, 1), "b");
        if (rc == NTVS_OK && M > 0) {
            cudaError_t e = cudaMemcpyAsync(hdev, h->hist, sizeof(float) * 12 * (size_t)M, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(bdev, h->b, sizeof(float) * (size_t)M, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) rc = fail(NTVS_ERR_CUDA, cuda_msg("history copy", e));
        }
        src = hdev;
        bsrc = bdev;
    }
    if (rc == NTVS_OK) {
        cudaError_t e = cudaMemsetAsync(c->dflags, 0, sizeof(int), st);
        if (e == cudaSuccess) e = k_hist_to_paths(src, M, rec, c->dflags, c->sms * 8, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->hint, c->dflags, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = fail(NTVS_ERR_CUDA, cuda_msg("history conversion", e));
        else if (c->hint[0]) rc = fail(NTVS_ERR_CSR, "non-finite history value");
    }
    dev_free(hdev);
    hdev = nullptr;
    if (rc != NTVS_OK) {
        release();
        return rc;
    }
    ntvs_paths p;
    p.nx = h->nx; p.ny = h->ny; p.nz = h->nz;
    p.n_blocks = h->n_blocks;
    p.dx = h->dx; p.dy = h->dy; p.dz = h->dz;
    p.n_rows = M;
    p.paths = rec;
    p.b = bsrc;
    p.block_ptr = h->block_ptr;
    p.n_seg = h->n_seg;
    p.mem_kind = NTVS_MEM_DEVICE;
    p.min_len = h->min_len;
    rc = ntvs_load_paths(c, &p);
    if (rc != NTVS_OK) {
        release();
        return rc;
    }
    c->own_paths = true;          // the records are the context's
    if (bdev) c->own_b = true;    // and so is the copy of host b
    return NTVS_OK;
}

int ntvs_set_params(ntvs_ctx* c, const ntvs_params* p) {
    if (!c || !p) return fail(NTVS_ERR_ARG, "null argument");
    if (p->N < 0) return fail(NTVS_ERR_ARG, "N must be >= 0");
    if (!(p->alpha > 0.0 && p->alpha < 1.0)) return fail(NTVS_ERR_ARG, "alpha must lie in (0, 1)");
    if (!(p->beta0 >= 0.0) || !std::isfinite(p->beta0)) return fail(NTVS_ERR_ARG, "beta0 must be finite and >= 0");
    if (!(p->eps_tv >= 0.0) || !std::isfinite(p->eps_tv)) return fail(NTVS_ERR_ARG, "eps_tv must be finite and >= 0");
    if (!std::isfinite(p->lambda)) return fail(NTVS_ERR_ARG, "lambda must be finite");
    if (p->tv_check && p->max_retries < 1) return fail(NTVS_ERR_ARG, "max_retries must be >= 1");
    if (p->step_rule < NTVS_STEP_NTVS || p->step_rule > NTVS_STEP_DECOUPLED)
        return fail(NTVS_ERR_ARG, "unknown step_rule");
    if (p->step_rule == NTVS_STEP_DECOUPLED) {
        if (!(p->gamma > 0.0 && p->gamma < 1.0)) return fail(NTVS_ERR_ARG, "gamma must lie in (0, 1)");
        if (p->tv_check) return fail(NTVS_ERR_ARG, "the decoupled step rule is defined without the TV check");
    }
    c->p = *p;
    return NTVS_OK;
}

int ntvs_set_image(ntvs_ctx* c, const void* x, int dtype, int mem_kind) {
    TRY(use_device(c));
    TRY(need_system(c));
    if (dtype != NTVS_F64 && dtype != NTVS_F32) return fail(NTVS_ERR_ARG, "image dtype must be NTVS_F64 or NTVS_F32");
    if (!x) return fail(NTVS_ERR_ARG, "null image");
    if (mem_kind == NTVS_MEM_DEVICE) {
        CUDA_TRY(k_convert(x, dtype, c->x, NTVS_F64, c->V, c->stream));
    } else if (mem_kind != NTVS_MEM_HOST) {
        return fail(NTVS_ERR_ARG, "bad mem_kind");
    } else if (dtype == NTVS_F64) {
        CUDA_TRY(cudaMemcpyAsync(c->x, x, (size_t)c->V * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    } else {
        std::vector<double> tmp((size_t)c->V);
        const float* s = (const float*)x;
        for (int64_t j = 0; j < c->V; ++j) tmp[j] = s[j];
        CUDA_TRY(cudaMemcpyAsync(c->x, tmp.data(), tmp.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    if (c->x32) CUDA_TRY(k_x32_from_x64(c->x, c->copies(), c->stream));
    c->split_stale = false;
    return NTVS_OK;
}

int ntvs_get_image(ntvs_ctx* c, void* out, int dtype, int mem_kind) {
    TRY(use_device(c));
    TRY(need_system(c));
    TRY(check_device_error(c));
    return copy_image_out(c, c->x, NTVS_F64, out, dtype, mem_kind);
}

int ntvs_run(ntvs_ctx* c, int k_iters) {
    TRY(use_device(c));
    TRY(need_system(c));
    if (k_iters < 0) return fail(NTVS_ERR_ARG, "k_iters < 0");
    TRY(ensure_tvhist(c, c->k + k_iters));
    // with the TV check every decision (and ell) stays on the device; without it the host
    // knows ell at every step and draws it itself
    const bool dev_check = c->p.tv_check && c->check_grid > 0 && c->p.step_rule != NTVS_STEP_DECOUPLED;
    if (dev_check) TRY(prepare_device_check(c, k_iters));
    else TRY(pull_device_trace(c));
    for (int kk = 0; kk < k_iters; ++kk) {
        if (dev_check) {
            const bool has = c->override_pos < c->override_ell.size();
            const int64_t ov = has ? c->override_ell[c->override_pos++] : 0;
            int64_t* slot = c->dev_ell_tr + (int64_t)c->ell_trace.size();
            CUDA_TRY(timed_launch(c, KIND_TV, [&] {
                return k_check_cycle_begin(c->cstate, c->p.step_rule, c->p.seed, c->k, has, ov, slot, c->stream);
            }));
            c->ell_trace.push_back(0);   // filled by pull_device_trace
            TRY(perturb_steps_device(c));
        } else {
            int64_t ell;
            if (c->override_pos < c->override_ell.size()) ell = c->override_ell[c->override_pos++];
            else ell = cycle_ell(c->p, c->k, c->ell_prev);
            c->ell_trace.push_back(ell);
            TRY(perturb_steps(c, &ell));
            if (ell_advances(c->p)) {
                c->ell_prev = ell;
                c->dstate_valid = false;
            }
        }
        TRY(drop_sweep(c));
        CUDA_TRY(timed_launch(c, KIND_TV, [&] {
            return k_tv_value(c->cdt, c->x, nullptr, c->dscal, 0.0, c->nx, c->ny, c->nz, c->red, c->tvhist + c->k,
                              nullptr, nullptr, c->stream);
        }));
        c->k += 1;
    }
    return NTVS_OK;
}

int ntvs_sync(ntvs_ctx* c) {
    TRY(use_device(c));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

int ntvs_get_tv(ntvs_ctx* c, double* tv) {
    TRY(use_device(c));
    TRY(need_system(c));
    if (!tv) return fail(NTVS_ERR_ARG, "null output");
    CUDA_TRY(timed_launch(c, KIND_TV, [&] {
        return k_tv_value(c->cdt, c->x, nullptr, c->dscal, 0.0, c->nx, c->ny, c->nz, c->red, c->dscal + 3, nullptr,
                          nullptr, c->stream);
    }));
    CUDA_TRY(cudaMemcpyAsync(c->hscal, c->dscal + 3, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    *tv = c->hscal[0];
    return check_device_error(c);
}

int ntvs_get_stats(ntvs_ctx* c, ntvs_stats* st) {
    TRY(use_device(c));
    if (!st) return fail(NTVS_ERR_ARG, "null output");
    TRY(pull_device_trace(c));
    std::memset(st, 0, sizeof(*st));
    st->k = c->k;
    st->ell_prev = c->ell_prev;
    st->n_steps = c->n_steps;
    st->n_accepted = c->n_accepted;
    st->n_tries = c->n_tries;
    st->nnz = c->nnz;
    st->n_rows = c->M;
    st->n_blocks = c->B;
    st->compute_dtype = c->cdt;
    st->last_tv = NAN;
    st->n_launches = c->n_launches;
    st->drop_schedule = c->schedule;
    st->lanes_per_row = c->lpr;
    st->n_escaped = c->n_escaped;
    st->voxel_tile_x = c->loaded ? c->vm.tx : 0;
    st->voxel_tile_y = c->loaded ? c->vm.ty : 0;
    if (c->k > 0 && c->tvhist) {
        CUDA_TRY(cudaMemcpyAsync(c->hscal, c->tvhist + (c->k - 1), sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        st->last_tv = c->hscal[0];
    } else {
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    return NTVS_OK;
}

int ntvs_get_block_resid(ntvs_ctx* c, double* out, int cap) {
    TRY(use_device(c));
    TRY(need_system(c));
    if (!out || cap < c->B) return fail(NTVS_ERR_ARG, "output too small");
    CUDA_TRY(cudaMemcpyAsync(out, c->resid, sizeof(double) * (size_t)c->B, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

int ntvs_get_trace(ntvs_ctx* c, int64_t* ell_k, int32_t* tries, int32_t* accepted, int64_t cap, int64_t* n_cycles) {
    TRY(use_device(c));
    TRY(pull_device_trace(c));
    const int64_t nk = (int64_t)c->ell_trace.size();
    const int64_t ns = (int64_t)c->tries_trace.size();
    if (ell_k) for (int64_t i = 0; i < nk && i < cap; ++i) ell_k[i] = c->ell_trace[i];
    if (tries) for (int64_t i = 0; i < ns && i < cap; ++i) tries[i] = c->tries_trace[i];
    if (accepted) for (int64_t i = 0; i < ns && i < cap; ++i) accepted[i] = c->acc_trace[i];
    if (n_cycles) *n_cycles = nk;
    return NTVS_OK;
}

int ntvs_get_state(ntvs_ctx* c, int64_t* k, int64_t* ell_prev) {
    TRY(use_device(c));
    TRY(pull_device_trace(c));
    if (k) *k = c->k;
    if (ell_prev) *ell_prev = c->ell_prev;
    return NTVS_OK;
}

int ntvs_set_state(ntvs_ctx* c, int64_t k, int64_t ell_prev) {
    TRY(use_device(c));
    if (k < 0 || ell_prev < 0) return fail(NTVS_ERR_ARG, "k and ell_prev must be >= 0");
    TRY(pull_device_trace(c));
    c->k = k;
    c->ell_prev = ell_prev;
    c->dstate_valid = false;
    return NTVS_OK;
}

int ntvs_set_profiling(ntvs_ctx* c, int on) {
    TRY(use_device(c));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    harvest_timing(c);
    c->profiling = on != 0;
    if (c->profiling) {
        for (int q = 0; q < 3; ++q) { c->prof_ms[q] = 0.0; c->prof_n[q] = 0; }
    }
    return NTVS_OK;
}

int ntvs_get_profile(ntvs_ctx* c, ntvs_profile* out) {
    TRY(use_device(c));
    if (!out) return fail(NTVS_ERR_ARG, "null output");
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    harvest_timing(c);
    out->drop_block_ms = c->prof_ms[KIND_DROP];
    out->drop_block_launches = c->prof_n[KIND_DROP];
    out->drop_apply_ms = c->prof_ms[KIND_APPLY];
    out->drop_apply_launches = c->prof_n[KIND_APPLY];
    out->tv_ms = c->prof_ms[KIND_TV];
    out->tv_launches = c->prof_n[KIND_TV];
    return NTVS_OK;
}

int ntvs_set_voxel_tile(ntvs_ctx* c, int tx, int ty) {
    if (!c) return fail(NTVS_ERR_ARG, "null context");
    auto ok = [](int v) { return v == 1 || v == 2 || v == 4 || v == 8 || v == 16; };
    if (!ok(tx) || !ok(ty)) return fail(NTVS_ERR_ARG, "tile sizes must be 1, 2, 4, 8 or 16");
    c->tile_req_x = tx;
    c->tile_req_y = ty;
    return NTVS_OK;
}

int ntvs_set_fault_hook(ntvs_ctx* c, int64_t wait_ns, int flags) {
    if (!c) return fail(NTVS_ERR_ARG, "null context");
    if (flags & ~(NTVS_HOOK_STARVE_PIPE | NTVS_HOOK_STARVE_CHECK)) return fail(NTVS_ERR_ARG, "unknown hook flag");
    c->wait_ns = wait_ns > 0 ? (uint64_t)wait_ns : kDefaultWaitNs;
    c->hook_flags = flags;
    return NTVS_OK;
}

int ntvs_set_compute_dtype(ntvs_ctx* c, int dtype) {
    if (!c) return fail(NTVS_ERR_ARG, "null context");
    if (dtype != NTVS_F32 && dtype != NTVS_F64) return fail(NTVS_ERR_ARG, "compute dtype must be NTVS_F32 or NTVS_F64");
    c->compute_req = dtype;
    return NTVS_OK;
}

int ntvs_set_ell_override(ntvs_ctx* c, const int64_t* ell_k, int64_t n) {
    if (!c) return fail(NTVS_ERR_ARG, "null context");
    c->override_ell.clear();
    c->override_pos = 0;
    if (ell_k && n > 0) c->override_ell.assign(ell_k, ell_k + n);
    return NTVS_OK;
}

int ntvs_tv_gradient(ntvs_ctx* c, void* g_out, int dtype, int mem_kind, double* gnorm) {
    TRY(use_device(c));
    TRY(need_system(c));
    TRY(launch_grad(c, false));
    if (g_out) TRY(copy_image_out(c, c->g, c->cdt, g_out, dtype, mem_kind));
    if (gnorm) {
        CUDA_TRY(cudaMemcpyAsync(c->hscal, c->dscal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        *gnorm = std::sqrt(c->hscal[0]);
    }
    return NTVS_OK;
}

int ntvs_perturb(ntvs_ctx* c, double beta) {
    TRY(use_device(c));
    TRY(need_system(c));
    TRY(launch_grad(c, false));
    CUDA_TRY(timed_launch(c, KIND_TV, [&] {
        return k_tv_apply(c->cdt, c->x, c->copies(), c->g, c->dscal + 0, beta, nullptr, c->V, c->stream);
    }));
    return NTVS_OK;
}

int ntvs_perturb_checked(ntvs_ctx* c, double beta, int* accepted, double* phi_x, double* phi_z) {
    TRY(use_device(c));
    TRY(need_system(c));
    TRY(launch_grad(c, true));
    int a = 0;
    TRY(checked_try(c, beta, &a));
    if (accepted) *accepted = a;
    if (phi_x || phi_z) {
        CUDA_TRY(cudaMemcpyAsync(c->hscal, c->dscal, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (phi_x) *phi_x = c->hscal[1];
        if (phi_z) *phi_z = c->hscal[2];
    }
    return NTVS_OK;
}

int ntvs_drop_block(ntvs_ctx* c, int t) {
    TRY(use_device(c));
    TRY(need_system(c));
    if (t < 0 || t >= c->B) return fail(NTVS_ERR_ARG, "block index out of range");
    return drop_block(c, t);
}

int ntvs_drop_sweep(ntvs_ctx* c) {
    TRY(use_device(c));
    TRY(need_system(c));
    return drop_sweep(c);
}

}  // extern "C"

namespace {

int ensure_ext(ntvs_ctx* c) {
    if (!c->ext) TRY(dev_alloc(&c->ext, sizeof(double) * (size_t)std::max<int64_t>(c->V, 1), "staging buffer"));
    return NTVS_OK;
}

int check_block_and_image(ntvs_ctx* c, int t, int dtype, int mem_kind) {
    if (t < 0 || t >= c->B) return fail(NTVS_ERR_ARG, "block index out of range");
    if (dtype != NTVS_F64 && dtype != NTVS_F32) return fail(NTVS_ERR_ARG, "dtype must be NTVS_F64 or NTVS_F32");
    if (mem_kind != NTVS_MEM_HOST && mem_kind != NTVS_MEM_DEVICE) return fail(NTVS_ERR_ARG, "bad mem_kind");
    return NTVS_OK;
}

const void* inv_s_of(ntvs_ctx* c, int t) { return (const char*)c->inv_s + (size_t)t * c->vm.vint * c->csz(); }

}  // namespace

extern "C" {

int ntvs_forward_project(ntvs_ctx* c, const void* x, int x_dtype, int x_mem, void* out, int out_dtype, int out_mem) {
    TRY(use_device(c));
    TRY(need_system(c));
    if (!x || (!out && c->M > 0)) return fail(NTVS_ERR_ARG, "null image or output");
    if ((x_dtype != NTVS_F64 && x_dtype != NTVS_F32) || (out_dtype != NTVS_F64 && out_dtype != NTVS_F32))
        return fail(NTVS_ERR_ARG, "dtypes must be NTVS_F64 or NTVS_F32");
    if ((x_mem != NTVS_MEM_HOST && x_mem != NTVS_MEM_DEVICE) || (out_mem != NTVS_MEM_HOST && out_mem != NTVS_MEM_DEVICE))
        return fail(NTVS_ERR_ARG, "bad mem_kind");
    double* x64 = nullptr;
    float* xg = nullptr;
    void* oc = nullptr;
    struct Free {
        double*& a;
        float*& b;
        void*& c;
        ~Free() { dev_free(a); dev_free(b); dev_free(c); }
    } guard{x64, xg, oc};
    cudaStream_t st = c->stream;
    // x as FP64 canonical, then in the gather order of the stored columns
    TRY(dev_alloc(&x64, sizeof(double) * (size_t)c->V, "projection image"));
    if (x_mem == NTVS_MEM_DEVICE) {
        CUDA_TRY(k_convert(x, x_dtype, x64, NTVS_F64, c->V, st));
    } else if (x_dtype == NTVS_F64) {
        CUDA_TRY(cudaMemcpyAsync(x64, x, sizeof(double) * (size_t)c->V, cudaMemcpyHostToDevice, st));
    } else {
        std::vector<double> tmp((size_t)c->V);
        const float* xf = (const float*)x;
        for (int64_t j = 0; j < c->V; ++j) tmp[(size_t)j] = xf[j];
        CUDA_TRY(cudaMemcpyAsync(x64, tmp.data(), sizeof(double) * (size_t)c->V, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    const void* xs = x64;
    if (c->cdt == F32) {
        TRY(dev_alloc(&xg, sizeof(float) * (size_t)c->vm.vint, "projection gather image"));
        CUDA_TRY(cudaMemsetAsync(xg, 0, sizeof(float) * (size_t)c->vm.vint, st));
        CUDA_TRY(k_x32_from_x64(x64, ImgCopies{xg, nullptr, nullptr, c->vm}, st));
        xs = xg;
    }
    TRY(dev_alloc(&oc, c->csz() * (size_t)std::max<int64_t>(c->M, 1), "projection"));
    if (c->paths_mode) {
        CUDA_TRY(k_otf_project(c->otf, (const float*)xs, (float*)oc, st));
    } else {
        DropArgs a;
        std::memset(&a, 0, sizeof(a));
        a.row_ptr = c->row_ptr;
        a.col = c->drop_cols();
        a.val = c->val;
        a.vdt = c->vdt;
        a.cdt = c->cdt;
        a.grid = c->drop_grid;
        a.use_d16 = c->storage == NTVS_DELTA16;
        a.d16 = c->d16();
        CUDA_TRY(k_project(a, c->M, xs, oc, st));
    }
    if (out_mem == NTVS_MEM_DEVICE) {
        CUDA_TRY(k_convert(oc, c->cdt, out, out_dtype, c->M, st));
        CUDA_TRY(cudaStreamSynchronize(st));   // the temporaries are released on return
        return NTVS_OK;
    }
    std::vector<unsigned char> h(c->csz() * (size_t)c->M);
    if (c->M > 0) CUDA_TRY(cudaMemcpyAsync(h.data(), oc, h.size(), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < c->M; ++i) {
        const double v = c->cdt == F64 ? ((const double*)h.data())[i] : (double)((const float*)h.data())[i];
        if (out_dtype == NTVS_F64) ((double*)out)[i] = v;
        else ((float*)out)[i] = (float)v;
    }
    return NTVS_OK;
}

int ntvs_drop_block_partial(ntvs_ctx* c, int t, int64_t r0, int64_t r1, void* delta_out, int dtype, int mem_kind,
                            double* resid_ss) {
    TRY(use_device(c));
    TRY(need_system(c));
    TRY(check_block_and_image(c, t, dtype, mem_kind));
    if (!delta_out) return fail(NTVS_ERR_ARG, "null delta_out");
    if (r0 < 0 && r1 < 0) {
        r0 = c->block_ptr[t];
        r1 = c->block_ptr[t + 1];
    }
    if (r0 < c->block_ptr[t] || r1 > c->block_ptr[t + 1] || r0 > r1)
        return fail(NTVS_ERR_ARG, "rows [r0, r1) must lie inside block t");
    CUDA_TRY(cudaMemsetAsync(c->dscal + 4, 0, sizeof(double), c->stream));
    float* wb = nullptr;
    float* wo = nullptr;
    TRY(launch_drop_kernel(c, t, r0, r1, c->dscal + 4, &wb, &wo));
    const size_t bytes = (size_t)c->V * dt_size(dtype);
    if (mem_kind == NTVS_MEM_DEVICE) {
        CUDA_TRY(k_delta_out(c->cdt, c->delta, c->vm, delta_out, dtype, c->stream));
    } else {
        TRY(ensure_ext(c));
        CUDA_TRY(k_delta_out(c->cdt, c->delta, c->vm, c->ext, dtype, c->stream));
        CUDA_TRY(cudaMemcpyAsync(delta_out, c->ext, bytes, cudaMemcpyDeviceToHost, c->stream));
    }
    if (resid_ss) CUDA_TRY(cudaMemcpyAsync(c->hscal + 4, c->dscal + 4, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (resid_ss || mem_kind == NTVS_MEM_HOST) {
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (resid_ss) *resid_ss = c->hscal[4];
    }
    return NTVS_OK;
}

int ntvs_apply_delta(ntvs_ctx* c, int t, const void* delta, int dtype, int mem_kind) {
    TRY(use_device(c));
    TRY(need_system(c));
    TRY(check_block_and_image(c, t, dtype, mem_kind));
    if (!delta) return fail(NTVS_ERR_ARG, "null delta");
    const void* src = delta;
    if (mem_kind == NTVS_MEM_HOST) {
        TRY(ensure_ext(c));
        CUDA_TRY(cudaMemcpyAsync(c->ext, delta, (size_t)c->V * dt_size(dtype), cudaMemcpyHostToDevice, c->stream));
        src = c->ext;
    }
    CUDA_TRY(timed_launch(c, KIND_APPLY, [&] {
        return k_apply_ext(c->cdt, c->x, c->copies(), src, dtype, inv_s_of(c, t), c->stream);
    }));
    c->split_stale = false;
    if (mem_kind == NTVS_MEM_HOST) CUDA_TRY(cudaStreamSynchronize(c->stream));
    return NTVS_OK;
}

int ntvs_get_hit_counts(ntvs_ctx* c, int t, int32_t* out, int mem_kind) {
    TRY(use_device(c));
    TRY(need_system(c));
    TRY(check_block_and_image(c, t, NTVS_F32, mem_kind));
    if (!out) return fail(NTVS_ERR_ARG, "null output");
    if (mem_kind == NTVS_MEM_DEVICE) {
        CUDA_TRY(k_counts_out(c->cdt, inv_s_of(c, t), c->vm, out, c->stream));
        return NTVS_OK;
    }
    TRY(ensure_ext(c));
    CUDA_TRY(k_counts_out(c->cdt, inv_s_of(c, t), c->vm, (int32_t*)c->ext, c->stream));
    CUDA_TRY(cudaMemcpyAsync(out, c->ext, sizeof(int32_t) * (size_t)c->V, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return NTVS_OK;
}

int ntvs_set_hit_counts(ntvs_ctx* c, int t, const int32_t* counts, int mem_kind) {
    TRY(use_device(c));
    TRY(need_system(c));
    TRY(check_block_and_image(c, t, NTVS_F32, mem_kind));
    if (!counts) return fail(NTVS_ERR_ARG, "null counts");
    const int32_t* src = counts;
    if (mem_kind == NTVS_MEM_HOST) {
        for (int64_t j = 0; j < c->V; ++j)
            if (counts[j] < 0) return fail(NTVS_ERR_ARG, "hit counts must be >= 0");
        TRY(ensure_ext(c));
        CUDA_TRY(cudaMemcpyAsync(c->ext, counts, sizeof(int32_t) * (size_t)c->V, cudaMemcpyHostToDevice, c->stream));
        src = (const int32_t*)c->ext;
    }
    CUDA_TRY(k_counts_in(c->cdt, src, c->vm, const_cast<void*>(inv_s_of(c, t)), c->stream));
    if (mem_kind == NTVS_MEM_HOST) CUDA_TRY(cudaStreamSynchronize(c->stream));
    return NTVS_OK;
}

int ntvs_set_allreduce(ntvs_ctx* c, ntvs_allreduce_fn fn, void* user) {
    TRY(use_device(c));
    TRY(need_system(c));
    if (!fn) {
        c->ar_fn = nullptr;
        c->ar_user = nullptr;
        return NTVS_OK;
    }
    if (c->ar_fn) return fail(NTVS_ERR_STATE, "an all-reduce callback is already set (the counts are global)");
    // global hit counts: this rank's counts of every block, summed over the ranks
    const int64_t n = (int64_t)c->B * c->vm.vint;
    int32_t* cnt = nullptr;
    TRY(dev_alloc(&cnt, sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1), "hit counts"));
    struct Free {
        int32_t*& p;
        ~Free() { dev_free(p); }
    } guard{cnt};
    CUDA_TRY(k_counts_from_inv(c->cdt, c->inv_s, cnt, n, c->stream));
    const int rc = fn(cnt, n, NTVS_I32, (void*)c->stream, user);
    if (rc != 0) return fail(NTVS_ERR_CUDA, "the all-reduce callback failed on the hit counts (returned " +
                                                std::to_string(rc) + ")");
    CUDA_TRY(k_inv_counts(cnt, c->inv_s, c->cdt, n, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->ar_fn = fn;
    c->ar_user = user;
    return NTVS_OK;
}

}  // extern "C"
