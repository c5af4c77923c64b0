// C ABI of the library: argument checks, workspace, the CG driver (CUDA-graph
// replay of the iteration) and the LML / gradient pipeline.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "batch.cuh"
#include "lgp_internal.cuh"

using namespace lgp;

namespace {

constexpr int kVersion = 10000;  // 1.0.0
constexpr int kRowPad = 256;     // workspace rows are padded to a multiple of this
constexpr int kChunk = 8;        // CG iterations per graph launch
constexpr long long kDefaultWaitBudget = 4000000000LL;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct lgp_ctx {
    int device = 0;
    int num_sms = 0;
    std::string err;
    long long wait_budget = kDefaultWaitBudget;
    cudaStream_t work = nullptr;  // internal stream (graph capture is not allowed on the legacy stream)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t ev_chunk[2] = {nullptr, nullptr};
    // workspace
    DevBuf xs, mv_partial, cg_vec, cg_partial, cg_state, cg_hist, scal, rhs, adj_b, adj_partial, vsplit, flags;
    DevBuf batch_meta, batch_part, pred_xs, pred_z, pred_q;
    DevBuf sr_x, sr_state, sr_hist, sr_tmp;  // single-column solves assembled into t columns
    DevBuf pc_l64, pc_l32, pc_d, pc_info, pc_part, pc_u, pc_cinv, pc_gram, pc_e, pc_rhs;
    int64_t ws_bytes = 0;
    // pinned host mirrors
    CgState *h_state = nullptr;
    int *h_done = nullptr;      // [2] per pipelined chunk
    double *h_scal = nullptr;   // [kMaxT * 4]
    int *h_flags = nullptr;     // [4]
    // cached CG graph
    cudaGraphExec_t cg_exec = nullptr;
    std::vector<unsigned char> cg_key;
    // autotuned column-split counts of the tensor-core product, keyed by (Np, t, fmt, D, kind)
    std::map<std::vector<int64_t>, int> tc_splits;
    // route of a batched problem shape, keyed by (Np, D, kind, t): 0 = the persistent batch launch,
    // 1 = its own solve with the tensor-core product (timed once per shape, batch_route)
    std::map<std::vector<int64_t>, int> batch_routes;
    std::map<std::vector<int64_t>, int> batch_splits;  // column splits of a persistent-batch problem, per shape
    // the last symmetric-tile product: its kind, padded rows and columns (for the distance-form query)
    int sym_kind = -1, sym_D = 0, sym_t = 0;
    int64_t sym_Np = 0;
    // prepare_x calls so far; the X-only operands of the tensor-core products in vsplit (transposed X,
    // with opnd_dot also the dot-form distance operands) belong to prepared X number opnd_version (built for
    // opnd_t columns at workspace address opnd_buf), 0 = none
    uint64_t prep_version = 0, opnd_version = 0;
    int opnd_t = 0;
    bool opnd_dot = false;
    void *opnd_buf = nullptr;
    size_t opnd_buf_bytes = 0;  // with opnd_buf: the workspace allocation the operands were written to
    int cg_dist_form = -1;      // distance form baked into the last CG graph (-1: both instances launch)
    int last_batch_tc = 0;      // problems of the last batched solve that took the tensor-core route
    // kernel timing (lgp_set_kernel_timing): events recorded around the product kernel's launch by
    // products outside stream capture; kev_set once a pair has been recorded
    bool kernel_timing = false, kev_set = false;
    cudaEvent_t kev[2] = {nullptr, nullptr};
};

namespace {

// NVTX range over the host-side part of a call (no-op unless a profiler is attached), so that a
// timeline shows the library's phases: entry points, input preparation, autotuning, the
// preconditioner build and the CG loop.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

lgp_status fail(lgp_ctx *c, lgp_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
lgp_status fail(lgp_ctx *c, lgp_status s, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define LGP_CUDA(call)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail(ctx, LGP_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                        __FILE__, __LINE__);                                                           \
    } while (0)

lgp_status ensure(lgp_ctx *ctx, DevBuf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return LGP_OK;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        ctx->ws_bytes -= (int64_t)b.bytes;
        b.p = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess) return fail(ctx, LGP_ERR_CUDA, "cudaFree: %s", cudaGetErrorString(e));
    }
    const size_t rounded = (bytes + (1u << 20) - 1) & ~((size_t)(1u << 20) - 1);
    cudaError_t e = cudaMalloc(&b.p, rounded);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        b.p = nullptr;
        return fail(ctx, LGP_ERR_WORKSPACE, "workspace allocation of %zu bytes failed: %s", rounded,
                    cudaGetErrorString(e));
    }
    b.bytes = rounded;
    ctx->ws_bytes += (int64_t)rounded;
    // any workspace move invalidates the cached CG graph
    if (ctx->cg_exec) {
        cudaGraphExecDestroy(ctx->cg_exec);
        ctx->cg_exec = nullptr;
        ctx->cg_key.clear();
    }
    return LGP_OK;
}

int64_t pad_rows(int64_t N) { return (N + kRowPad - 1) / kRowPad * kRowPad; }

lgp_status check_dev_ptr(lgp_ctx *ctx, const void *p, const char *name) {
    if (p == nullptr) return fail(ctx, LGP_ERR_INVALID_ARG, "%s is NULL", name);
    if (((uintptr_t)p) % 4 != 0) return fail(ctx, LGP_ERR_INVALID_ARG, "%s is not 4-byte aligned", name);
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ctx, LGP_ERR_INVALID_ARG, "%s is not a CUDA pointer (%s)", name, cudaGetErrorString(e));
    }
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return fail(ctx, LGP_ERR_INVALID_ARG, "%s is not device memory", name);
    if (attr.device != ctx->device)
        return fail(ctx, LGP_ERR_INVALID_ARG, "%s lives on device %d, context is on device %d", name, attr.device,
                    ctx->device);
    return LGP_OK;
}

lgp_status make_params(lgp_ctx *ctx, const lgp_hyper *h, KernelParams *kp) {
    if (!h) return fail(ctx, LGP_ERR_INVALID_ARG, "hyp is NULL");
    if (!kind_supported(h->kind))
        return fail(ctx, LGP_ERR_INVALID_ARG, "unknown kernel kind %d", h->kind);
    if (h->D < 1 || h->D > kMaxD) return fail(ctx, LGP_ERR_UNSUPPORTED, "D=%d outside 1..%d", h->D, kMaxD);
    if (!h->log_lengthscale) return fail(ctx, LGP_ERR_INVALID_ARG, "log_lengthscale is NULL");
    if (!std::isfinite(h->log_outputscale) || !std::isfinite(h->log_noise))
        return fail(ctx, LGP_ERR_NONFINITE, "non-finite outputscale or noise");
    std::memset(kp, 0, sizeof *kp);
    kp->kind = h->kind;
    kp->D = h->D;
    kp->dpad = dpad_of(h->D);
    const double c = prescale_of(h->kind);
    for (int d = 0; d < h->D; ++d) {
        const double ll = h->log_lengthscale[d];
        if (!std::isfinite(ll)) return fail(ctx, LGP_ERR_NONFINITE, "non-finite log_lengthscale[%d]", d);
        kp->scale[d] = (float)(c * std::exp(-ll));
        if (!(kp->scale[d] > 0.0f) || !std::isfinite(kp->scale[d]))
            return fail(ctx, LGP_ERR_UNSUPPORTED, "lengthscale[%d] out of float range", d);
    }
    kp->s2 = (float)std::exp((double)h->log_outputscale);
    kp->log2_s2 = (float)((double)h->log_outputscale / std::log(2.0));
    kp->noise = (float)std::exp((double)h->log_noise);
    if (!(kp->s2 > 0.0f) || !std::isfinite(kp->s2) || !(kp->noise >= 0.0f) || !std::isfinite(kp->noise))
        return fail(ctx, LGP_ERR_UNSUPPORTED, "outputscale or noise out of float range");
    return LGP_OK;
}

// Resolve the product arithmetic for t columns.
int resolve_prec(int t, int prec) {
    if (prec == LGP_PREC_FP32) return LGP_PREC_FP32;
    if (prec == LGP_PREC_SPLIT_BF16 || prec == LGP_PREC_SPLIT_F16)
        return tc_supported(t) ? prec : (int)LGP_ERR_UNSUPPORTED;
    if (prec == LGP_PREC_AUTO) return tc_supported(t) ? LGP_PREC_SPLIT_F16 : LGP_PREC_FP32;
    return LGP_ERR_INVALID_ARG;
}

// resolve_prec for the entry points that zero-pad the caller's columns (lgp_kernel_matvec, lgp_cg_solve): an
// explicit split precision with t not in {16, 32} runs with *tp = 16 (t < 16) or 32 (16 < t < 32) columns, the
// extra ones zero. AUTO is unchanged (split only at t in {16, 32}). *tp = t otherwise.
int resolve_prec_padded(int t, int prec, int *tp) {
    *tp = t;
    if ((prec == LGP_PREC_SPLIT_BF16 || prec == LGP_PREC_SPLIT_F16) && t != 16 && t != 32) {
        const int padded = t < 16 ? 16 : (t < 32 ? 32 : 0);
        if (padded == 0 || !tc_supported(padded)) return LGP_ERR_UNSUPPORTED;
        *tp = padded;
        return prec;
    }
    return resolve_prec(t, prec);
}

bool is_tc(int prec) { return prec == LGP_PREC_SPLIT_BF16 || prec == LGP_PREC_SPLIT_F16; }
int tc_fmt(int prec) { return prec == LGP_PREC_SPLIT_F16 ? 1 : 0; }

struct Prepared {
    KernelParams kp;
    int64_t N, Np;
    float *xs;
    uint64_t version;  // distinguishes successive preparations of the context's xs buffer
};

lgp_status prepare_x(lgp_ctx *ctx, const lgp_hyper *hyp, const float *X, int64_t N, cudaStream_t st, Prepared *pp) {
    NvtxRange nvtx_range("lgp.prepare_x");
    lgp_status s = make_params(ctx, hyp, &pp->kp);
    if (s != LGP_OK) return s;
    pp->N = N;
    pp->Np = pad_rows(N);
    s = ensure(ctx, ctx->xs, (size_t)pp->Np * pp->kp.dpad * sizeof(float));
    if (s != LGP_OK) return s;
    s = ensure(ctx, ctx->flags, 64);
    if (s != LGP_OK) return s;
    pp->xs = (float *)ctx->xs.p;
    pp->version = ++ctx->prep_version;
    launch_prep_x(X, N, pp->kp.D, pp->kp.dpad, pp->kp.scale, pp->xs, pp->Np, (int *)ctx->flags.p, st);
    LGP_CUDA(cudaGetLastError());
    return LGP_OK;
}

std::vector<int64_t> tc_key(const Prepared &pp, int t, int prec) {
    return {pp.Np, (int64_t)t, (int64_t)tc_fmt(prec), (int64_t)pp.kp.D, (int64_t)pp.kp.kind};
}

int tc_splits_for(const lgp_ctx *ctx, const Prepared &pp, int t, int prec) {
    auto it = ctx->tc_splits.find(tc_key(pp, t, prec));
    return it == ctx->tc_splits.end() ? 0 : it->second;
}

// Autotuner of the tensor-core product's kernel: on the first product of a shape, time the
// symmetric-tile kernel and the three most wave-efficient column-split counts of the row kernel
// on the caller's own inputs (one warm-up and two timed launches each, CUDA events on the
// stream) and keep the fastest for that shape. Never runs during a stream capture.
// LGP_AUTOTUNE=0 keeps the row kernel's wave-efficiency heuristic; LGP_TC_SYMMETRIC=1 forces the
// symmetric kernel (where the shape allows it), LGP_TC_SYMMETRIC=0 leaves it out.
// Persistent autotune cache (LGP_AUTOTUNE_CACHE=<file>): one text line per tuned shape,
// "<device name>|<SMs>|<Np>|<t>|<fmt>|<D>|<kind> <choice>", read before timing and appended after.
std::string tune_cache_key(const lgp_ctx *ctx, const std::vector<int64_t> &key) {
    cudaDeviceProp prop;
    std::string name = cudaGetDeviceProperties(&prop, ctx->device) == cudaSuccess ? prop.name : "unknown";
    for (char &c : name)
        if (c == '|' || c == ' ') c = '_';
    std::string k = name + "|" + std::to_string(ctx->num_sms);
    for (int64_t v : key) k += "|" + std::to_string(v);
    return k;
}

bool tune_cache_lookup(const char *path, const std::string &k, int *choice) {
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        char name[400];
        int v = 0;
        if (std::sscanf(line, "%399s %d", name, &v) == 2 && k == name) {
            *choice = v;  // the last entry for a key wins
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void tune_cache_store(const char *path, const std::string &k, int choice) {
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d\n", k.c_str(), choice);
    std::fclose(f);
}

lgp_status autotune_tc(lgp_ctx *ctx, const Prepared &pp, const float *V, int64_t ldv, float *out, int64_t ldo, int t,
                       int prec, cudaStream_t st) {
    NvtxRange nvtx_range("lgp.autotune");
    const std::vector<int64_t> key = tc_key(pp, t, prec);
    if (ctx->tc_splits.count(key)) return LGP_OK;
    const char *env = std::getenv("LGP_AUTOTUNE");
    const char *sym = std::getenv("LGP_TC_SYMMETRIC");
    int cand[4], n = 0;
    tc_split_candidates(pp.Np, ctx->num_sms, cand, &n);
    if (sym && sym[0] == '1' && tc_symmetric_ok(pp.Np)) {
        ctx->tc_splits[key] = kTcSymmetric;
        return LGP_OK;
    }
    if (sym && sym[0] == '0' && n > 0 && cand[0] == kTcSymmetric) {
        for (int k = 1; k < n; ++k) cand[k - 1] = cand[k];
        --n;
    }
    if ((env && env[0] == '0') || n <= 1) {
        ctx->tc_splits[key] = 0;
        return LGP_OK;
    }
    const char *cache_path = std::getenv("LGP_AUTOTUNE_CACHE");
    const std::string cache_key = cache_path ? tune_cache_key(ctx, key) : std::string();
    int cached = 0;
    if (cache_path && tune_cache_lookup(cache_path, cache_key, &cached)) {
        bool allowed = false;
        for (int k = 0; k < n; ++k) allowed |= cand[k] == cached;
        if (allowed) {
            ctx->tc_splits[key] = cached;
            return LGP_OK;
        }
    }
    int64_t need = 1;
    for (int k = 0; k < n; ++k) need = std::max(need, mv_tc_partial_floats(pp.Np, t, ctx->num_sms, cand[k]));
    lgp_status s;
    if ((s = ensure(ctx, ctx->mv_partial, (size_t)need * sizeof(float))) != LGP_OK) return s;
    if ((s = ensure(ctx, ctx->vsplit, (size_t)tc_vsplit_bytes(pp.Np, t))) != LGP_OK) return s;
    cudaEvent_t e0, e1;
    LGP_CUDA(cudaEventCreate(&e0));
    LGP_CUDA(cudaEventCreate(&e1));
    int best = 0;
    float best_ms = 1e30f;
    cudaError_t ce = cudaSuccess;
    for (int k = 0; k < n && ce == cudaSuccess; ++k) {
        float total = 0.0f;
        for (int rep = 0; rep < 3 && ce == cudaSuccess; ++rep) {
            ce = cudaEventRecord(e0, st);
            if (ce == cudaSuccess)
                ce = launch_mv_tc(pp.kp, pp.xs, pp.N, pp.Np, V, ldv, out, ldo, t, tc_fmt(prec), ctx->vsplit.p,
                                  (float *)ctx->mv_partial.p, (int64_t)(ctx->mv_partial.bytes / sizeof(float)), nullptr,
                                  (int *)ctx->flags.p + 1, ctx->wait_budget, ctx->num_sms, st, cand[k]);
            if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) total += ms;
        }
        if (ce == cudaSuccess && total < best_ms) {
            best_ms = total;
            best = cand[k];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ce != cudaSuccess) return fail(ctx, LGP_ERR_CUDA, "autotune launch failed: %s", cudaGetErrorString(ce));
    ctx->tc_splits[key] = best;
    if (cache_path) tune_cache_store(cache_path, cache_key, best);
    return LGP_OK;
}

// Whether the symmetric product of this shape may take the dot form (and so needs its operands).
bool needs_dot(const lgp_ctx *ctx, const Prepared &pp, int t, int prec) {
    return is_tc(prec) && tc_splits_for(ctx, pp, t, prec) == kTcSymmetric && dot_form_allowed(pp.kp.kind, pp.kp.D);
}

// Whether the X-only operands of prepared X (for a product of this shape) are in the context's V-split
// workspace for t columns.
bool tc_operands_valid(const lgp_ctx *ctx, const Prepared &pp, int t, int prec) {
    return ctx->opnd_version == pp.version && ctx->opnd_t == t && ctx->opnd_buf == ctx->vsplit.p &&
           ctx->opnd_buf_bytes == ctx->vsplit.bytes && (ctx->opnd_dot || !needs_dot(ctx, pp, t, prec));
}

// Builds the X-only operands of the tensor-core products of prepared X once (not inside the products of a
// solve, where X does not change): the transposed X and, for a symmetric product that may take the dot
// form, its distance operands.
lgp_status ensure_tc_operands(lgp_ctx *ctx, const Prepared &pp, int t, int prec, cudaStream_t st) {
    if (!is_tc(prec) || tc_operands_valid(ctx, pp, t, prec)) return LGP_OK;
    lgp_status s = ensure(ctx, ctx->vsplit, (size_t)tc_vsplit_bytes(pp.Np, t));
    if (s != LGP_OK) return s;
    const bool dot = needs_dot(ctx, pp, t, prec);
    LGP_CUDA(launch_tc_operands(pp.kp, pp.xs, pp.N, pp.Np, t, ctx->vsplit.p, dot, st));
    ctx->opnd_version = pp.version;
    ctx->opnd_t = t;
    ctx->opnd_dot = dot;
    ctx->opnd_buf = ctx->vsplit.p;
    ctx->opnd_buf_bytes = ctx->vsplit.bytes;
    return LGP_OK;
}

// K_y V for prepared X. V has row stride ldv; out has row stride ldo.
// dist_form: see launch_mv_tc (-1 unless the caller read the dot-form gate word of this X).
// Whether this product records the kernel-timing events: timing switched on and st not capturing.
bool kernel_timing_on(const lgp_ctx *ctx, cudaStream_t st) {
    if (!ctx->kernel_timing || !ctx->kev[0] || !ctx->kev[1]) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
}

lgp_status matvec_prepared(lgp_ctx *ctx, const Prepared &pp, const float *V, int64_t ldv, float *out, int64_t ldo,
                           int t, int prec, const int *skip, cudaStream_t st, int dist_form = -1) {
    if (is_tc(prec)) {
        lgp_status s = ensure(ctx, ctx->vsplit, (size_t)tc_vsplit_bytes(pp.Np, t));
        if (s != LGP_OK) return s;
        const int forced = tc_splits_for(ctx, pp, t, prec);
        const int64_t pf = mv_tc_partial_floats(pp.Np, t, ctx->num_sms, forced);
        s = ensure(ctx, ctx->mv_partial, (size_t)std::max<int64_t>(pf, 1) * sizeof(float));
        if (s != LGP_OK) return s;
        if ((s = ensure_tc_operands(ctx, pp, t, prec, st)) != LGP_OK) return s;
        const bool timed = kernel_timing_on(ctx, st);
        LGP_CUDA(launch_mv_tc(pp.kp, pp.xs, pp.N, pp.Np, V, ldv, out, ldo, t, tc_fmt(prec), ctx->vsplit.p,
                              (float *)ctx->mv_partial.p,
                              (int64_t)(ctx->mv_partial.bytes / sizeof(float)), skip, (int *)ctx->flags.p + 1,
                              ctx->wait_budget, ctx->num_sms, st, forced, tc_operands_valid(ctx, pp, t, prec),
                              dist_form, timed ? ctx->kev[0] : nullptr, timed ? ctx->kev[1] : nullptr));
        if (timed) ctx->kev_set = true;
        if (forced == kTcSymmetric) {
            ctx->sym_kind = pp.kp.kind;
            ctx->sym_D = pp.kp.D;
            ctx->sym_t = t;
            ctx->sym_Np = pp.Np;
        }
        return LGP_OK;
    }
    const int64_t pf = mv_simt_partial_floats(pp.N, pp.Np, t, ctx->num_sms);
    lgp_status s = ensure(ctx, ctx->mv_partial, (size_t)std::max<int64_t>(pf, 1) * sizeof(float));
    if (s != LGP_OK) return s;
    MvLaunch m;
    m.kp = &pp.kp;
    m.Xs = pp.xs;
    m.N = pp.N;
    m.Np = pp.Np;
    m.V = V;
    m.ldv = ldv;
    m.out = out;
    m.ldo = ldo;
    m.t = t;
    m.partial = (float *)ctx->mv_partial.p;
    m.partial_cap = (int64_t)(ctx->mv_partial.bytes / sizeof(float));
    m.skip = skip;
    m.num_sms = ctx->num_sms;
    const bool timed = kernel_timing_on(ctx, st);
    if (timed) cudaEventRecord(ctx->kev[0], st);
    LGP_CUDA(launch_mv_simt(m, st));
    if (timed) {
        cudaEventRecord(ctx->kev[1], st);
        ctx->kev_set = true;
    }
    return LGP_OK;
}

lgp_status check_opts(lgp_ctx *ctx, const lgp_options *o, bool need_probes) {
    if (!o) return fail(ctx, LGP_ERR_INVALID_ARG, "options is NULL");
    if (!(o->tol > 0.0) || !std::isfinite(o->tol)) return fail(ctx, LGP_ERR_INVALID_ARG, "tol must be > 0");
    if (o->max_iter < 1) return fail(ctx, LGP_ERR_INVALID_ARG, "max_iter must be >= 1");
    if (o->precond_rank < 0 || o->precond_rank > kMaxRank)
        return fail(ctx, LGP_ERR_UNSUPPORTED, "precond_rank=%d outside 0..%d", o->precond_rank, kMaxRank);
    if (need_probes) {
        if (o->n_probes < 1 || o->n_probes + 1 > kMaxT)
            return fail(ctx, LGP_ERR_UNSUPPORTED, "n_probes=%d outside 1..%d", o->n_probes, kMaxT - 1);
        if (o->lanczos_steps < 1 || o->lanczos_steps > kMaxLanczos)
            return fail(ctx, LGP_ERR_UNSUPPORTED, "lanczos_steps=%d outside 1..%d", o->lanczos_steps, kMaxLanczos);
    }
    return LGP_OK;
}

// Workspace layout of one CG run.
lgp_status cg_buffers(lgp_ctx *ctx, int64_t N, int64_t Np, int t, int hist_len, CgBuffers *b) {
    lgp_status s;
    if ((s = ensure(ctx, ctx->cg_vec, (size_t)5 * Np * t * sizeof(float))) != LGP_OK) return s;
    b->G = cg_num_blocks(N, t, ctx->num_sms);
    if ((s = ensure(ctx, ctx->cg_partial, (size_t)b->G * 3 * t * sizeof(double))) != LGP_OK) return s;
    if ((s = ensure(ctx, ctx->cg_state, sizeof(CgState))) != LGP_OK) return s;
    if ((s = ensure(ctx, ctx->cg_hist, (size_t)2 * std::max(hist_len, 1) * t * sizeof(double))) != LGP_OK) return s;
    float *v = (float *)ctx->cg_vec.p;
    b->x = v;
    b->r = v + Np * t;
    b->p = v + 2 * Np * t;
    b->Kp = v + 3 * Np * t;
    b->z = v + 4 * Np * t;
    b->pc = Precond();
    b->partial = (double *)ctx->cg_partial.p;
    b->state = (CgState *)ctx->cg_state.p;
    b->hist_alpha = (double *)ctx->cg_hist.p;
    b->hist_beta = b->hist_alpha + (size_t)std::max(hist_len, 1) * t;
    return LGP_OK;
}

// Cholesky factor of the symmetric positive definite n x n matrix A (row-major, in place, lower
// triangle); false if a pivot is not positive.
bool host_cholesky(std::vector<double> &A, int n) {
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int q = 0; q < j; ++q) d -= A[j * n + q] * A[j * n + q];
        if (!(d > 0.0)) return false;
        const double ljj = std::sqrt(d);
        A[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double v = A[i * n + j];
            for (int q = 0; q < j; ++q) v -= A[i * n + q] * A[j * n + q];
            A[i * n + j] = v / ljj;
        }
    }
    return true;
}

// Builds the rank-k pivoted-Cholesky preconditioner P = L L^T + sigma^2 I of K_y for solves with t
// columns (precond.cu): L from the raw X in float64, C = sigma^2 I + L^T L reduced on the device and
// factored on the host (float64), C^{-1} uploaded, log|P| = (N - k) log sigma^2 + log|C|.
// Synchronises the internal stream once.
lgp_status build_precond(lgp_ctx *ctx, const lgp_hyper *hyp, const float *X, const Prepared &pp, int k, int t,
                         Precond *out) {
    NvtxRange nvtx_range("lgp.build_precond");
    cudaStream_t st = ctx->work;
    const int64_t N = pp.N, Np = pp.Np;
    if (k < 1 || k > kMaxRank) return fail(ctx, LGP_ERR_UNSUPPORTED, "precond_rank=%d outside 1..%d", k, kMaxRank);
    if (t > 32 || k * t > 1024)
        return fail(ctx, LGP_ERR_UNSUPPORTED, "preconditioned solves take at most 32 columns (t=%d, rank %d)", t, k);
    const int G2 = std::max(1, std::min(2 * ctx->num_sms, (int)((N + 255) / 256)));
    lgp_status s;
    if ((s = ensure(ctx, ctx->pc_l64, (size_t)k * Np * sizeof(double))) != LGP_OK ||
        (s = ensure(ctx, ctx->pc_l32, (size_t)k * Np * sizeof(float))) != LGP_OK ||
        (s = ensure(ctx, ctx->pc_d, (size_t)Np * sizeof(double))) != LGP_OK ||
        (s = ensure(ctx, ctx->pc_info, pivinfo_bytes())) != LGP_OK ||
        (s = ensure(ctx, ctx->pc_part, (size_t)G2 * k * t * sizeof(double))) != LGP_OK ||
        (s = ensure(ctx, ctx->pc_u, (size_t)k * t * sizeof(double))) != LGP_OK ||
        (s = ensure(ctx, ctx->pc_cinv, (size_t)k * k * sizeof(double))) != LGP_OK ||
        (s = ensure(ctx, ctx->pc_gram, (size_t)G2 * k * k * sizeof(double))) != LGP_OK)
        return s;
    const int D = hyp->D;
    double inv_ls[kMaxD];
    for (int d = 0; d < D; ++d) inv_ls[d] = std::exp(-(double)hyp->log_lengthscale[d]);
    const double s2 = std::exp((double)hyp->log_outputscale);
    const double noise = std::exp((double)hyp->log_noise);
    double *L64 = (double *)ctx->pc_l64.p;
    launch_pivchol(X, N, Np, D, inv_ls, s2, hyp->kind, k, L64, (double *)ctx->pc_d.p, ctx->pc_info.p, st);
    launch_gram(L64, Np, N, k, (double *)ctx->pc_gram.p, G2, st);
    launch_to_f32(L64, (float *)ctx->pc_l32.p, (int64_t)k * Np, st);
    LGP_CUDA(cudaGetLastError());
    std::vector<double> part((size_t)G2 * k * k);
    LGP_CUDA(cudaMemcpyAsync(part.data(), ctx->pc_gram.p, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    LGP_CUDA(cudaStreamSynchronize(st));
    std::vector<double> C((size_t)k * k, 0.0);
    for (int b = 0; b < G2; ++b)
        for (int e = 0; e < k * k; ++e) C[e] += part[(size_t)b * k * k + e];
    for (int q = 0; q < k; ++q) C[q * k + q] += noise;
    for (double v : C)
        if (!std::isfinite(v)) return fail(ctx, LGP_ERR_NONFINITE, "non-finite value in the preconditioner factor");
    std::vector<double> Lc = C;
    if (!host_cholesky(Lc, k)) return fail(ctx, LGP_ERR_BREAKDOWN, "preconditioner core matrix not positive definite");
    double logdet_c = 0.0;
    for (int q = 0; q < k; ++q) logdet_c += 2.0 * std::log(Lc[q * k + q]);
    // C^{-1} column by column from the Cholesky factor (forward then backward substitution)
    std::vector<double> Cinv((size_t)k * k);
    std::vector<double> col(k);
    for (int j = 0; j < k; ++j) {
        for (int i = 0; i < k; ++i) {
            double v = i == j ? 1.0 : 0.0;
            for (int q = 0; q < i; ++q) v -= Lc[i * k + q] * col[q];
            col[i] = v / Lc[i * k + i];
        }
        for (int i = k - 1; i >= 0; --i) {
            double v = col[i];
            for (int q = i + 1; q < k; ++q) v -= Lc[q * k + i] * col[q];
            col[i] = v / Lc[i * k + i];
        }
        for (int i = 0; i < k; ++i) Cinv[i * k + j] = col[i];
    }
    LGP_CUDA(cudaMemcpy(ctx->pc_cinv.p, Cinv.data(), Cinv.size() * sizeof(double), cudaMemcpyHostToDevice));
    Precond pc;
    pc.k = k;
    pc.Np = Np;
    pc.L64 = L64;
    pc.L32 = (const float *)ctx->pc_l32.p;
    pc.Cinv = (const double *)ctx->pc_cinv.p;
    pc.part = (double *)ctx->pc_part.p;
    pc.U = (double *)ctx->pc_u.p;
    pc.G = G2;
    pc.noise = noise;
    pc.logdet = (double)(N - k) * std::log(noise) + logdet_c;
    *out = pc;
    return LGP_OK;
}

// Run CG on the internal stream: init, then replay a captured chunk of iterations until done.
int matvec_launches(const lgp_ctx *ctx, const Prepared &pp, int t, int prec, int dist_form = -1) {
    return is_tc(prec) ? mv_tc_launches(pp.Np, t, ctx->num_sms, tc_fmt(prec), tc_splits_for(ctx, pp, t, prec), pp.kp.kind,
                                        pp.kp.D, tc_operands_valid(ctx, pp, t, prec), dist_form)
                       : mv_simt_launches(pp.N, pp.Np, t, ctx->num_sms);
}

// Kernel launches of one CG iteration (the product plus the five vector/scalar kernels).
int cg_iteration_launches(const lgp_ctx *ctx, const Prepared &pp, int t, int prec, int dist_form = -1) {
    return matvec_launches(ctx, pp, t, prec, dist_form) + 5;
}

lgp_status run_cg(lgp_ctx *ctx, const Prepared &pp, const float *B, int64_t ldb, int t, const lgp_options *opt,
                  int hist_len, int prec, CgBuffers *bout, int *chunks_run = nullptr, const Precond *pc = nullptr,
                  const float *X0 = nullptr) {
    NvtxRange nvtx_range("lgp.cg");
    cudaStream_t st = ctx->work;
    CgBuffers b;
    lgp_status s = cg_buffers(ctx, pp.N, pp.Np, t, hist_len, &b);
    if (s != LGP_OK) return s;
    // the product's own workspace must exist before capture (no allocation inside a capture)
    if (is_tc(prec)) {
        // tune the product on this solve's right-hand sides (Kp is scratch here) before capture
        if ((s = autotune_tc(ctx, pp, B, ldb, b.Kp, t, t, prec, st)) != LGP_OK) return s;
        if ((s = ensure(ctx, ctx->vsplit, (size_t)tc_vsplit_bytes(pp.Np, t))) != LGP_OK) return s;
        const int64_t pf = mv_tc_partial_floats(pp.Np, t, ctx->num_sms, tc_splits_for(ctx, pp, t, prec));
        if ((s = ensure(ctx, ctx->mv_partial, (size_t)std::max<int64_t>(pf, 1) * sizeof(float))) != LGP_OK) return s;
    } else {
        const int64_t pf = mv_simt_partial_floats(pp.N, pp.Np, t, ctx->num_sms);
        if ((s = ensure(ctx, ctx->mv_partial, (size_t)std::max<int64_t>(pf, 1) * sizeof(float))) != LGP_OK) return s;
    }
    // the X-only operands of the products, once for the whole solve (outside the captured loop)
    if ((s = ensure_tc_operands(ctx, pp, t, prec, st)) != LGP_OK) return s;
    // the symmetric product's distance form, read once per solve from the gate word those operands hold,
    // so that only the instance of that form is launched in the loop
    int dist_form = -1;
    if (needs_dot(ctx, pp, t, prec) && tc_operands_valid(ctx, pp, t, prec)) {
        unsigned int bits = 0;
        LGP_CUDA(cudaMemcpyAsync(&bits, (const char *)ctx->vsplit.p + tc_dot_gate_offset(pp.Np, t), sizeof bits,
                                 cudaMemcpyDeviceToHost, st));
        LGP_CUDA(cudaStreamSynchronize(st));
        float amax;
        std::memcpy(&amax, &bits, sizeof amax);
        dist_form = amax <= dot_gate_limit(pp.kp.kind) ? 1 : 0;
    }
    ctx->cg_dist_form = dist_form;
    // cg_buffers/ensure may have moved memory: re-read pointers
    s = cg_buffers(ctx, pp.N, pp.Np, t, hist_len, &b);
    if (s != LGP_OK) return s;
    if (pc) b.pc = *pc;

    if (X0) {
        // warm start: r0 = b - K_y x0 needs one product first (into Kp)
        if ((s = matvec_prepared(ctx, pp, X0, t, b.Kp, t, t, prec, nullptr, st, dist_form)) != LGP_OK) return s;
    }
    launch_cg_init(B, ldb, pp.N, pp.Np, t, b, opt->tol, opt->max_iter, hist_len, st, X0, t);
    LGP_CUDA(cudaGetLastError());

    const char *graph_env = std::getenv("LGP_CG_GRAPH");
    if (graph_env && graph_env[0] == '0') {
        // Host-driven loop: the same kernels launched one by one, the done flag read back after
        // every chunk (a profiler then sees each launch on its own).
        int launched = 0;
        while (true) {
            for (int k = 0; k < kChunk; ++k) {
                if ((s = matvec_prepared(ctx, pp, b.p, t, b.Kp, t, t, prec, &b.state->done, st, dist_form)) != LGP_OK)
                    return s;
                launch_cg_after_matvec(pp.N, pp.Np, t, b, st);
            }
            launch_cg_chunk_tally(b.state, st);
            ++launched;
            LGP_CUDA(cudaMemcpyAsync(ctx->h_state, b.state, sizeof(CgState), cudaMemcpyDeviceToHost, st));
            LGP_CUDA(cudaStreamSynchronize(st));
            if (ctx->h_state->done || ctx->h_state->loop_chunks >= ctx->h_state->max_chunks) break;
        }
        *bout = b;
        if (chunks_run) *chunks_run = launched;
        return LGP_OK;
    }

    // Graph key: everything baked into the captured launches.
    std::vector<unsigned char> key;
    auto put = [&key](const void *p, size_t n) {
        const unsigned char *c = (const unsigned char *)p;
        key.insert(key.end(), c, c + n);
    };
    put(&pp.kp, sizeof pp.kp);
    put(&pp.N, sizeof pp.N);
    put(&pp.xs, sizeof pp.xs);
    put(&t, sizeof t);
    put(&prec, sizeof prec);
    put(&dist_form, sizeof dist_form);
    // the buffers field by field (the structs have padding bytes)
    const void *ptrs[] = {b.x, b.r, b.p, b.Kp, b.z, b.partial, b.state, b.hist_alpha, b.hist_beta,
                          b.pc.L64, b.pc.L32, b.pc.Cinv, b.pc.part, b.pc.U};
    put(ptrs, sizeof ptrs);
    put(&b.G, sizeof b.G);
    put(&b.pc.k, sizeof b.pc.k);
    put(&b.pc.G, sizeof b.pc.G);
    put(&b.pc.Np, sizeof b.pc.Np);
    put(&b.pc.noise, sizeof b.pc.noise);
    put(&ctx->mv_partial.p, sizeof(void *));
    put(&ctx->vsplit.p, sizeof(void *));
    put(&ctx->wait_budget, sizeof ctx->wait_budget);
    if (!ctx->cg_exec || ctx->cg_key != key) {
        if (ctx->cg_exec) {
            cudaGraphExecDestroy(ctx->cg_exec);
            ctx->cg_exec = nullptr;
        }
        // One graph for the whole solve: a conditional WHILE node whose body is a chunk of
        // kChunk iterations followed by a kernel that sets the condition to "not done and under
        // the chunk cap", so the iteration loop runs on the device with no host round trip.
        cudaGraph_t g = nullptr;
        LGP_CUDA(cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle h;
        cudaError_t ce = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
        // the parameter struct holds a union with no default constructor: zero raw storage instead
        alignas(cudaGraphNodeParams) unsigned char np_storage[sizeof(cudaGraphNodeParams)] = {};
        cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(np_storage);
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if (ce == cudaSuccess) ce = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
        if (ce != cudaSuccess) {
            cudaGraphDestroy(g);
            return fail(ctx, LGP_ERR_CUDA, "conditional graph node: %s", cudaGetErrorString(ce));
        }
        cudaGraph_t body = np.conditional.phGraph_out[0];
        ce = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) {
            cudaGraphDestroy(g);
            return fail(ctx, LGP_ERR_CUDA, "capture to graph: %s", cudaGetErrorString(ce));
        }
        lgp_status cs = LGP_OK;
        for (int k = 0; k < kChunk && cs == LGP_OK; ++k) {
            cs = matvec_prepared(ctx, pp, b.p, t, b.Kp, t, t, prec, &b.state->done, st, dist_form);
            if (cs == LGP_OK) launch_cg_after_matvec(pp.N, pp.Np, t, b, st);
        }
        if (cs == LGP_OK) launch_cg_loop_condition(h, b.state, st);
        cudaGraph_t captured = nullptr;
        ce = cudaStreamEndCapture(st, &captured);
        if (cs != LGP_OK) {
            cudaGraphDestroy(g);
            return cs;
        }
        if (ce != cudaSuccess) {
            cudaGraphDestroy(g);
            return fail(ctx, LGP_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
        }
        ce = cudaGraphInstantiate(&ctx->cg_exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            ctx->cg_exec = nullptr;
            return fail(ctx, LGP_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ce));
        }
        ctx->cg_key = key;
    }
    LGP_CUDA(cudaGraphLaunch(ctx->cg_exec, st));
    const int launched = 1;
    LGP_CUDA(cudaMemcpyAsync(ctx->h_state, b.state, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    *bout = b;
    if (chunks_run) *chunks_run = launched;
    return LGP_OK;
}

// The single-column path of lgp_lml_and_grad (LGP_OPT_SINGLE_RHS): each of the t columns of B is
// solved by its own CG run with the float32 one-column product, as the paper's plain CG loop does
// (Sec. 5), and the runs are assembled into t-column results (solutions, CG state, Lanczos history) for
// the same quadrature and adjoint kernels as the batched path.
lgp_status run_cg_columns(lgp_ctx *ctx, const Prepared &pp, const float *B, int t, const lgp_options *opt,
                          int hist_len, CgBuffers *bout, int *chunks_run) {
    NvtxRange nvtx_range("lgp.cg_columns");
    cudaStream_t st = ctx->work;
    const int Gt = cg_num_blocks(pp.N, t, ctx->num_sms);
    lgp_status s;
    // every t-column buffer exists before the first solve, so nothing moves between the column runs
    if ((s = ensure(ctx, ctx->cg_partial, (size_t)Gt * 3 * t * sizeof(double))) != LGP_OK ||
        (s = ensure(ctx, ctx->sr_x, (size_t)pp.Np * t * sizeof(float))) != LGP_OK ||
        (s = ensure(ctx, ctx->sr_state, sizeof(CgState))) != LGP_OK ||
        (s = ensure(ctx, ctx->sr_hist, (size_t)2 * std::max(hist_len, 1) * t * sizeof(double))) != LGP_OK)
        return s;
    CgState *dst = (CgState *)ctx->sr_state.p;
    double *dst_alpha = (double *)ctx->sr_hist.p;
    double *dst_beta = dst_alpha + (size_t)std::max(hist_len, 1) * t;
    float *xs = (float *)ctx->sr_x.p;
    LGP_CUDA(cudaMemsetAsync(dst, 0, sizeof(CgState), st));
    int chunks = 0;
    for (int c = 0; c < t; ++c) {
        CgBuffers b1;
        int ran = 0;
        if ((s = run_cg(ctx, pp, B + c, t, 1, opt, hist_len, LGP_PREC_FP32, &b1, &ran)) != LGP_OK) return s;
        launch_copy_cols(b1.x, 1, xs, t, pp.N, 1, c, st);
        launch_cg_gather_column(b1, hist_len, dst, dst_alpha, dst_beta, t, c, st);
        LGP_CUDA(cudaGetLastError());
        chunks += ran;
    }
    CgBuffers b;
    b.x = xs;
    b.r = b.p = b.Kp = b.z = nullptr;
    b.partial = (double *)ctx->cg_partial.p;
    b.G = Gt;
    b.state = dst;
    b.hist_alpha = dst_alpha;
    b.hist_beta = dst_beta;
    b.pc = Precond();
    LGP_CUDA(cudaMemcpyAsync(ctx->h_state, dst, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    *bout = b;
    if (chunks_run) *chunks_run = chunks;
    return LGP_OK;
}

// Make the internal stream wait for the caller's stream.
lgp_status enter(lgp_ctx *ctx, cudaStream_t user) {
    LGP_CUDA(cudaSetDevice(ctx->device));
    LGP_CUDA(cudaEventRecord(ctx->ev_in, user));
    LGP_CUDA(cudaStreamWaitEvent(ctx->work, ctx->ev_in, 0));
    return LGP_OK;
}

// Make the caller's stream wait for the internal stream, then synchronise it.
lgp_status leave_sync(lgp_ctx *ctx, cudaStream_t user) {
    LGP_CUDA(cudaEventRecord(ctx->ev_out, ctx->work));
    LGP_CUDA(cudaStreamWaitEvent(user, ctx->ev_out, 0));
    LGP_CUDA(cudaStreamSynchronize(ctx->work));
    return LGP_OK;
}

lgp_status cg_status_of(lgp_ctx *ctx, const CgState &h, int t, int *iters, double *rel, int x_nonfinite) {
    if (x_nonfinite) return fail(ctx, LGP_ERR_NONFINITE, "X contains NaN or Inf");
    bool unconverged = false;
    for (int c = 0; c < t; ++c) {
        if (iters) iters[c] = h.iters[c];
        const double rr = h.bnorm2[c] > 0.0 ? std::sqrt(h.rr[c] / h.bnorm2[c]) : 0.0;
        if (rel) rel[c] = rr;
        if (h.active[c]) unconverged = true;
    }
    if (h.status == LGP_ERR_NONFINITE) return fail(ctx, LGP_ERR_NONFINITE, "non-finite value in B or a CG scalar");
    if (h.status == LGP_ERR_BREAKDOWN)
        return fail(ctx, LGP_ERR_BREAKDOWN, "CG breakdown: p^T K_y p <= 0 (K_y not positive definite in float32)");
    if (unconverged) {
        fail(ctx, LGP_WARN_NOT_CONVERGED, "CG reached max_iter before tol on some column");
        return LGP_WARN_NOT_CONVERGED;
    }
    return LGP_OK;
}

// Smallest problem the batched solver times for the tensor-core route (smaller ones stay in the batch).
constexpr int64_t kBatchTcMinN = 2048;

// Route of one problem of a batched solve with t <= 16 columns, chosen by what each route costs per
// CG iteration, timed on the caller's own X and right-hand sides:
// - persistent batch launch (float32 products): the problem's marginal cost there, i.e. one float32
//   product with its t columns minus the same product on its first 256 rows (the launch floor, which
//   the batch launch pays once for all its problems);
// - tensor-core route: an iteration of a standalone CG solve with the split-F16 product, its columns
//   zero-padded to 16 (the product, the CG updates and the graph launches, all paid per problem):
//   the difference of two short solves (1 and 3 chunks of iterations, at tol 0) over 2 chunks.
// The tensor-core route is kept only if at least 10% cheaper. The short solves run only when the bare
// tensor-core product already passes that test. Cached per shape in the context and, with
// LGP_AUTOTUNE_CACHE, in the same file as the product choices (key suffix |route).
lgp_status batch_route(lgp_ctx *ctx, const lgp_hyper *h, const float *X, int64_t N, const float *B, int t,
                       int *route) {
    NvtxRange nvtx_range("lgp.batch_route");
    const std::vector<int64_t> key = {pad_rows(N), (int64_t)h->D, (int64_t)h->kind, (int64_t)t};
    auto it = ctx->batch_routes.find(key);
    if (it != ctx->batch_routes.end()) {
        *route = it->second;
        return LGP_OK;
    }
    *route = 0;
    const char *env = std::getenv("LGP_AUTOTUNE");
    if (N < kBatchTcMinN || t > 16 || !tc_supported(16) || (env && env[0] == '0')) {
        ctx->batch_routes[key] = 0;
        return LGP_OK;
    }
    const char *cache_path = std::getenv("LGP_AUTOTUNE_CACHE");
    const std::string cache_key = cache_path ? tune_cache_key(ctx, key) + "|route" : std::string();
    int cached = 0;
    if (cache_path && tune_cache_lookup(cache_path, cache_key, &cached) && (cached == 0 || cached == 1)) {
        ctx->batch_routes[key] = cached;
        *route = cached;
        return LGP_OK;
    }
    cudaStream_t st = ctx->work;
    constexpr int tp = 16;
    constexpr int64_t kFloorRows = 256;
    lgp_status s;
    if ((s = ensure(ctx, ctx->rhs, (size_t)pad_rows(N) * tp * sizeof(float))) != LGP_OK ||
        (s = ensure(ctx, ctx->sr_x, (size_t)pad_rows(N) * tp * sizeof(float))) != LGP_OK)
        return s;
    float *vpad = (float *)ctx->rhs.p, *out = (float *)ctx->sr_x.p;
    cudaEvent_t e0, e1;
    LGP_CUDA(cudaEventCreate(&e0));
    LGP_CUDA(cudaEventCreate(&e1));
    // mean time of fn() over `reps` calls on the stream, after one untimed call
    auto timed = [&](auto fn, int reps, float *mean_ms) -> lgp_status {
        *mean_ms = 0.0f;
        for (int rep = 0; rep <= reps; ++rep) {
            cudaEventRecord(e0, st);
            lgp_status r = fn();
            cudaEventRecord(e1, st);
            if (r != LGP_OK) return r;
            float m = 0.0f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&m, e0, e1) != cudaSuccess)
                return fail(ctx, LGP_ERR_CUDA, "batch route timing failed");
            if (rep > 0) *mean_ms += m / reps;
        }
        return LGP_OK;
    };
    float ms_floor = 0.0f, ms_fp32 = 0.0f, ms_tc = 0.0f;
    Prepared pp;
    // the launch floor: the float32 product of the first rows only (B is row-major, so its first rows
    // are that problem's right-hand sides)
    if ((s = prepare_x(ctx, h, X, kFloorRows, st, &pp)) == LGP_OK)
        s = timed([&] { return matvec_prepared(ctx, pp, B, t, out, t, t, LGP_PREC_FP32, nullptr, st); }, 2, &ms_floor);
    if (s == LGP_OK) s = prepare_x(ctx, h, X, N, st, &pp);
    if (s == LGP_OK) {
        LGP_CUDA(cudaMemsetAsync(vpad, 0, (size_t)pp.Np * tp * sizeof(float), st));
        launch_copy_cols(B, t, vpad, tp, N, t, 0, st);
        LGP_CUDA(cudaGetLastError());
        s = autotune_tc(ctx, pp, vpad, tp, out, tp, tp, LGP_PREC_SPLIT_F16, st);
    }
    if (s == LGP_OK)
        s = timed([&] { return matvec_prepared(ctx, pp, B, t, out, t, t, LGP_PREC_FP32, nullptr, st); }, 2, &ms_fp32);
    if (s == LGP_OK)
        s = timed([&] { return matvec_prepared(ctx, pp, vpad, tp, out, tp, tp, LGP_PREC_SPLIT_F16, nullptr, st); }, 2,
                  &ms_tc);
    const float marginal = ms_fp32 - ms_floor;
    if (s == LGP_OK && ms_tc < 0.9f * marginal) {
        lgp_options o = {};
        o.tol = 0.0;  // never met: each short solve runs its whole chunk budget
        o.prec = LGP_PREC_SPLIT_F16;
        float ms_short[2] = {0.0f, 0.0f};
        for (int k = 0; k < 2 && s == LGP_OK; ++k) {
            o.max_iter = (1 + 2 * k) * kChunk;
            s = timed(
                [&] {
                    CgBuffers b;
                    return run_cg(ctx, pp, vpad, tp, tp, &o, 0, LGP_PREC_SPLIT_F16, &b);
                },
                2, &ms_short[k]);
        }
        if (s == LGP_OK) *route = (ms_short[1] - ms_short[0]) / (2 * kChunk) < 0.9f * marginal ? 1 : 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != LGP_OK) return s;
    ctx->batch_routes[key] = *route;
    if (cache_path) tune_cache_store(cache_path, cache_key, *route);
    return LGP_OK;
}

// One problem of a batched solve on the tensor-core route: its t columns zero-padded to 16 (a zero
// column takes no iteration), one CG solve with the split-F16 product, the first t columns copied to
// Xsol. Fills iters and rel_resid for its t columns; synchronises the internal stream.
lgp_status batch_tc_solve(lgp_ctx *ctx, const lgp_hyper *h, const float *X, const float *B, float *Xsol, int64_t N,
                          int t, const lgp_options *opt, int *iters, double *rel, bool *unconverged) {
    NvtxRange nvtx_range("lgp.batch_tc_solve");
    cudaStream_t st = ctx->work;
    Prepared pp;
    lgp_status s;
    if ((s = prepare_x(ctx, h, X, N, st, &pp)) != LGP_OK) return s;
    constexpr int tp = 16;
    if ((s = ensure(ctx, ctx->rhs, (size_t)pp.Np * tp * sizeof(float))) != LGP_OK) return s;
    float *bpad = (float *)ctx->rhs.p;
    LGP_CUDA(cudaMemsetAsync(bpad, 0, (size_t)pp.Np * tp * sizeof(float), st));
    launch_copy_cols(B, t, bpad, tp, N, t, 0, st);
    LGP_CUDA(cudaGetLastError());
    lgp_options o = *opt;
    o.prec = LGP_PREC_SPLIT_F16;
    o.precond_rank = 0;
    o.flags = 0;
    CgBuffers b;
    if ((s = run_cg(ctx, pp, bpad, tp, tp, &o, 0, LGP_PREC_SPLIT_F16, &b)) != LGP_OK) return s;
    launch_copy_cols(b.x, tp, Xsol, t, N, t, 0, st);
    LGP_CUDA(cudaGetLastError());
    LGP_CUDA(cudaMemcpyAsync(ctx->h_flags, ctx->flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    LGP_CUDA(cudaStreamSynchronize(st));
    if (ctx->h_flags[1]) return fail(ctx, LGP_ERR_TIMEOUT, "a bounded device wait ran out (code %d)", ctx->h_flags[1]);
    if (ctx->h_flags[0]) return fail(ctx, LGP_ERR_NONFINITE, "some X[g] contains NaN or Inf");
    int it_all[kMaxT];
    double rel_all[kMaxT];
    const lgp_status cs = cg_status_of(ctx, *ctx->h_state, tp, it_all, rel_all, 0);
    if (cs < 0) return cs;
    for (int c = 0; c < t; ++c) {
        iters[c] = it_all[c];
        rel[c] = rel_all[c];
        *unconverged |= ctx->h_state->active[c] != 0;
    }
    return LGP_OK;
}

// The work list of a persistent batched solve: per problem its layout in the shared buffers, its vector
// blocks, and its (row block, column split) items.
struct BatchPlan {
    std::vector<BatchGp> gps;
    std::vector<KernelParams> kps;
    std::vector<const float *> X;
    std::vector<BatchItem> items;
    std::vector<BatchVecBlock> vblocks;
    int64_t xs_total = 0, rows_total = 0, part_total = 0;
};

// Appends one problem (rows N, parameters kp, caller's X, B, Xsol) with its row blocks split S ways over
// whole 64-column tiles.
void plan_add_problem(BatchPlan &P, int64_t N, const KernelParams &kp, const float *X, const float *B, float *Xsol,
                      int t, int64_t S) {
    const int q = (int)P.gps.size();
    const int rows_per_vblock = std::max(1, 4096 / t);
    const int bm = batch_item_rows();
    BatchGp G;
    G.N = N;
    G.Np = pad_rows(N);
    G.xs_off = P.xs_total;
    G.vec_off = P.rows_total;
    G.kind = kp.kind;
    G.dpad = kp.dpad;
    G.D = kp.D;
    G.log2s2 = kp.log2_s2;
    G.noise = kp.noise;
    G.B = B;
    G.Xsol = Xsol;
    G.blk0 = (int)P.vblocks.size();
    for (int64_t r0 = 0; r0 < G.N; r0 += rows_per_vblock)
        P.vblocks.push_back({q, r0, std::min<int64_t>(G.N, r0 + rows_per_vblock)});
    G.blk1 = (int)P.vblocks.size();
    const int64_t rb_n = (G.N + bm - 1) / bm;
    const int64_t col_tiles = (G.N + 63) / 64;
    S = std::max<int64_t>(1, std::min<int64_t>(S, col_tiles));
    G.cols_per_split = (col_tiles + S - 1) / S * 64;
    G.splits = (int)((G.N + G.cols_per_split - 1) / G.cols_per_split);
    G.part_off = P.part_total;
    if (G.splits > 1) P.part_total += (int64_t)G.splits * G.Np * t;
    for (int64_t rb = 0; rb < rb_n; ++rb)
        for (int sp = 0; sp < G.splits; ++sp) P.items.push_back({q, (int)rb, sp});
    P.xs_total += G.Np * G.dpad;
    P.rows_total += G.Np;
    P.gps.push_back(G);
    P.kps.push_back(kp);
    P.X.push_back(X);
}

// Column splits of a problem alone in the persistent product by the fixed rule: about two items per CTA
// slot (its last iterations may run with no other problem left), at least four column tiles per split.
int64_t batch_split_rule(const lgp_ctx *ctx, int64_t N) {
    const int bm = batch_item_rows();
    const int64_t rb_n = (N + bm - 1) / bm;
    const int64_t col_tiles = (N + 63) / 64;
    const int64_t S = std::max<int64_t>(1, (2 * ctx->num_sms + rb_n - 1) / rb_n);
    return std::min<int64_t>(S, std::max<int64_t>(1, col_tiles / 4));
}

// Sorts the plan's items (longest first: an item of problem g costs ~min(N_g, cols_per_split_g)), places
// the plan in the context's buffers, uploads it, prescales every problem's X and fills the device
// arguments A. Stream-ordered on st.
lgp_status upload_batch_plan(lgp_ctx *ctx, BatchPlan &P, int t, cudaStream_t st, BatchArgs *Aout) {
    lgp_status s;
    const int n_b = (int)P.gps.size();
    std::stable_sort(P.items.begin(), P.items.end(), [&](const BatchItem &a, const BatchItem &b) {
        return std::min(P.gps[a.gp].N, P.gps[a.gp].cols_per_split) > std::min(P.gps[b.gp].N, P.gps[b.gp].cols_per_split);
    });
    const int ng_t = n_b * t;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    const size_t o_gps = off; off = al(off + P.gps.size() * sizeof(BatchGp));
    const size_t o_items = off; off = al(off + P.items.size() * sizeof(BatchItem));
    const size_t o_vb = off; off = al(off + P.vblocks.size() * sizeof(BatchVecBlock));
    const size_t o_rr = off; off = al(off + 4 * (size_t)ng_t * sizeof(double));
    const size_t o_act = off; off = al(off + 2 * (size_t)ng_t * sizeof(int));
    const size_t o_gpd = off; off = al(off + (size_t)n_b * sizeof(int));
    const size_t o_misc = off; off = al(off + 256);
    if ((s = ensure(ctx, ctx->batch_meta, off)) != LGP_OK) return s;
    if ((s = ensure(ctx, ctx->xs, (size_t)P.xs_total * sizeof(float))) != LGP_OK) return s;
    if ((s = ensure(ctx, ctx->cg_vec, (size_t)4 * P.rows_total * t * sizeof(float))) != LGP_OK) return s;
    if ((s = ensure(ctx, ctx->cg_partial, P.vblocks.size() * (size_t)t * sizeof(double))) != LGP_OK) return s;
    if ((s = ensure(ctx, ctx->batch_part, (size_t)std::max<int64_t>(P.part_total, 1) * sizeof(float))) != LGP_OK)
        return s;
    if ((s = ensure(ctx, ctx->flags, 64)) != LGP_OK) return s;
    unsigned char *meta = (unsigned char *)ctx->batch_meta.p;
    BatchArgs A;
    A.gps = (const BatchGp *)(meta + o_gps);
    A.items = (const BatchItem *)(meta + o_items);
    A.vblocks = (const BatchVecBlock *)(meta + o_vb);
    A.n_gp = n_b;
    A.n_items = (int)P.items.size();
    A.n_vblocks = (int)P.vblocks.size();
    A.t = t;
    A.tt = 1;
    while (A.tt < t) A.tt *= 2;
    A.Xs = (const float *)ctx->xs.p;
    float *v = (float *)ctx->cg_vec.p;
    A.x = v;
    A.r = v + P.rows_total * t;
    A.p = v + 2 * P.rows_total * t;
    A.kp = v + 3 * P.rows_total * t;
    A.part = (float *)ctx->batch_part.p;
    A.partial = (double *)ctx->cg_partial.p;
    double *dd = (double *)(meta + o_rr);
    A.rr = dd;
    A.bnorm2 = dd + ng_t;
    A.alpha = dd + 2 * ng_t;
    A.beta = dd + 3 * ng_t;
    int *ii = (int *)(meta + o_act);
    A.active = ii;
    A.iters = ii + ng_t;
    A.gp_done = (int *)(meta + o_gpd);
    A.done = (int *)(meta + o_misc);
    A.item_counter = (int *)(meta + o_misc + 4);
    A.st = (BatchState *)(meta + o_misc + 64);
    LGP_CUDA(cudaMemcpyAsync(meta + o_gps, P.gps.data(), P.gps.size() * sizeof(BatchGp), cudaMemcpyHostToDevice, st));
    LGP_CUDA(cudaMemcpyAsync(meta + o_items, P.items.data(), P.items.size() * sizeof(BatchItem),
                             cudaMemcpyHostToDevice, st));
    LGP_CUDA(cudaMemcpyAsync(meta + o_vb, P.vblocks.data(), P.vblocks.size() * sizeof(BatchVecBlock),
                             cudaMemcpyHostToDevice, st));
    for (int q = 0; q < n_b; ++q)
        launch_prep_x(P.X[q], P.gps[q].N, P.kps[q].D, P.kps[q].dpad, P.kps[q].scale,
                      (float *)ctx->xs.p + P.gps[q].xs_off, P.gps[q].Np, (int *)ctx->flags.p, st);
    LGP_CUDA(cudaGetLastError());
    *Aout = A;
    return LGP_OK;
}

// Column splits of one problem of the persistent batch, timed per shape (padded N, D, kind, t) on the
// caller's own X and right-hand sides: the problem alone in the work list (the case its split count
// decides: its last iterations, with no other problem left) with the fixed rule's count and with a
// quarter, half, double and four times that many (at least one, at most one 64-column tile per split).
// Each candidate: one untimed and three timed products (the persistent launch and its split
// reduction, CUDA events). Cached in the context and, with LGP_AUTOTUNE_CACHE, in the product-choice
// file (key suffix |split); LGP_AUTOTUNE=0 keeps the rule.
lgp_status batch_split_choice(lgp_ctx *ctx, const KernelParams &kp, const lgp_hyper *h, const float *X,
                              const float *B, int64_t N, int t, int64_t *S_out) {
    const std::vector<int64_t> key = {pad_rows(N), (int64_t)h->D, (int64_t)h->kind, (int64_t)t};
    const int64_t rule = batch_split_rule(ctx, N);
    *S_out = rule;
    auto it = ctx->batch_splits.find(key);
    if (it != ctx->batch_splits.end()) {
        *S_out = it->second;
        return LGP_OK;
    }
    const char *env = std::getenv("LGP_AUTOTUNE");
    const int64_t col_tiles = (N + 63) / 64;
    if ((env && env[0] == '0') || col_tiles < 2) {
        ctx->batch_splits[key] = (int)rule;
        return LGP_OK;
    }
    const char *cache_path = std::getenv("LGP_AUTOTUNE_CACHE");
    const std::string cache_key = cache_path ? tune_cache_key(ctx, key) + "|split" : std::string();
    int cached = 0;
    if (cache_path && tune_cache_lookup(cache_path, cache_key, &cached) && cached >= 1) {
        ctx->batch_splits[key] = cached;
        *S_out = cached;
        return LGP_OK;
    }
    std::vector<int64_t> cands;
    for (int64_t c : {rule / 4, rule / 2, rule, 2 * rule, 4 * rule}) {
        c = std::max<int64_t>(1, std::min<int64_t>(c, col_tiles));
        if (std::find(cands.begin(), cands.end(), c) == cands.end()) cands.push_back(c);
    }
    cudaStream_t st = ctx->work;
    cudaEvent_t e0, e1;
    LGP_CUDA(cudaEventCreate(&e0));
    LGP_CUDA(cudaEventCreate(&e1));
    lgp_status s = LGP_OK;
    float best_ms = 0.0f;
    int64_t best = rule;
    for (size_t k = 0; k < cands.size() && s == LGP_OK; ++k) {
        BatchPlan P;
        plan_add_problem(P, N, kp, X, B, nullptr, t, cands[k]);
        BatchArgs A;
        if ((s = upload_batch_plan(ctx, P, t, st, &A)) != LGP_OK) break;
        if (launch_batch_init(A, 0.0, 1, st) != cudaSuccess) {
            s = fail(ctx, LGP_ERR_CUDA, "batch split tuning: init failed");
            break;
        }
        float ms = 0.0f;
        for (int rep = 0; rep < 4 && s == LGP_OK; ++rep) {
            cudaEventRecord(e0, st);
            const cudaError_t ce = launch_batch_product(A, ctx->num_sms, st);
            cudaEventRecord(e1, st);
            float m = 0.0f;
            if (ce != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&m, e0, e1) != cudaSuccess)
                s = fail(ctx, LGP_ERR_CUDA, "batch split tuning: timing failed");
            else if (rep > 0)
                ms += m;
        }
        if (s == LGP_OK && (k == 0 || ms < best_ms)) {
            best_ms = ms;
            best = cands[k];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != LGP_OK) return s;
    ctx->batch_splits[key] = (int)best;
    *S_out = best;
    if (cache_path) tune_cache_store(cache_path, cache_key, (int)best);
    return LGP_OK;
}

}  // namespace

// ============================================================================ C ABI

extern "C" {

int32_t lgp_version(void) { return kVersion; }

const char *lgp_status_string(int32_t s) {
    switch (s) {
        case LGP_OK: return "LGP_OK";
        case LGP_WARN_NOT_CONVERGED: return "LGP_WARN_NOT_CONVERGED";
        case LGP_ERR_INVALID_ARG: return "LGP_ERR_INVALID_ARG";
        case LGP_ERR_UNSUPPORTED: return "LGP_ERR_UNSUPPORTED";
        case LGP_ERR_CUDA: return "LGP_ERR_CUDA";
        case LGP_ERR_NONFINITE: return "LGP_ERR_NONFINITE";
        case LGP_ERR_BREAKDOWN: return "LGP_ERR_BREAKDOWN";
        case LGP_ERR_TIMEOUT: return "LGP_ERR_TIMEOUT";
        case LGP_ERR_WORKSPACE: return "LGP_ERR_WORKSPACE";
    }
    return "LGP_UNKNOWN_STATUS";
}

lgp_status lgp_create(lgp_ctx **out, int32_t device) {
    if (!out) return LGP_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        (void)cudaGetLastError();
        return LGP_ERR_INVALID_ARG;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return LGP_ERR_CUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return LGP_ERR_UNSUPPORTED;
    lgp_ctx *ctx = new lgp_ctx();
    ctx->device = device;
    ctx->num_sms = prop.multiProcessorCount;
    bool ok = cudaSetDevice(device) == cudaSuccess &&
              cudaStreamCreateWithFlags(&ctx->work, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&ctx->ev_chunk[0], cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&ctx->ev_chunk[1], cudaEventDisableTiming) == cudaSuccess &&
              cudaMallocHost(&ctx->h_state, sizeof(CgState)) == cudaSuccess &&
              cudaMallocHost(&ctx->h_done, 2 * sizeof(int)) == cudaSuccess &&
              cudaMallocHost(&ctx->h_scal, kMaxT * 4 * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&ctx->h_flags, 4 * sizeof(int)) == cudaSuccess;
    if (ok) {
        ok = ensure(ctx, ctx->flags, 64) == LGP_OK && cudaMemset(ctx->flags.p, 0, 64) == cudaSuccess;
    }
    if (!ok) {
        lgp_destroy(ctx);
        return LGP_ERR_CUDA;
    }
    *out = ctx;
    return LGP_OK;
}

void lgp_destroy(lgp_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->work) cudaStreamSynchronize(ctx->work);
    if (ctx->cg_exec) cudaGraphExecDestroy(ctx->cg_exec);
    for (cudaEvent_t e : ctx->kev)
        if (e) cudaEventDestroy(e);
    DevBuf *bufs[] = {&ctx->pc_l64,     &ctx->pc_l32,   &ctx->pc_d,      &ctx->pc_info,    &ctx->pc_part,
                      &ctx->pc_u,       &ctx->pc_cinv,  &ctx->pc_gram,   &ctx->pc_e,       &ctx->pc_rhs,
                      &ctx->batch_part, &ctx->pred_xs,  &ctx->pred_z,    &ctx->pred_q,     &ctx->xs,
                      &ctx->mv_partial, &ctx->cg_vec,   &ctx->cg_partial, &ctx->cg_state,  &ctx->cg_hist,
                      &ctx->scal,       &ctx->rhs,      &ctx->adj_b,     &ctx->adj_partial, &ctx->vsplit,
                      &ctx->flags,      &ctx->batch_meta, &ctx->sr_x,      &ctx->sr_state,   &ctx->sr_hist,
                      &ctx->sr_tmp};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (ctx->h_state) cudaFreeHost(ctx->h_state);
    if (ctx->h_done) cudaFreeHost(ctx->h_done);
    if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
    if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    if (ctx->ev_chunk[0]) cudaEventDestroy(ctx->ev_chunk[0]);
    if (ctx->ev_chunk[1]) cudaEventDestroy(ctx->ev_chunk[1]);
    if (ctx->work) cudaStreamDestroy(ctx->work);
    delete ctx;
}

const char *lgp_last_error_message(const lgp_ctx *ctx) {
    if (!ctx) return "no context";
    return ctx->err.c_str();
}

int64_t lgp_workspace_bytes(const lgp_ctx *ctx) { return ctx ? ctx->ws_bytes : 0; }

int32_t lgp_matvec_precision(const lgp_ctx *ctx, int32_t t, int32_t prec) {
    (void)ctx;
    if (t < 1 || t > kMaxT) return LGP_ERR_UNSUPPORTED;
    int tp = t;
    return resolve_prec_padded(t, prec, &tp);
}

int32_t lgp_tc_kernel_choice(const lgp_ctx *ctx, int64_t N, int32_t D, int32_t kind, int32_t t, int32_t prec) {
    if (!ctx || N < 1 || D < 1 || D > kMaxD || !kind_supported(kind)) return LGP_ERR_INVALID_ARG;
    if (t < 1 || t > kMaxT) return LGP_ERR_UNSUPPORTED;
    const int p = resolve_prec(t, prec);
    if (p < 0) return p;
    if (!is_tc(p)) return LGP_ERR_UNSUPPORTED;
    const std::vector<int64_t> key = {pad_rows(N), (int64_t)t, (int64_t)tc_fmt(p), (int64_t)D, (int64_t)kind};
    auto it = ctx->tc_splits.find(key);
    if (it == ctx->tc_splits.end()) return LGP_TC_UNTUNED;
    return it->second == kTcSymmetric ? LGP_TC_SYMMETRIC : LGP_TC_ROW;
}

int32_t lgp_batch_route_choice(const lgp_ctx *ctx, int64_t N, int32_t D, int32_t kind, int32_t t) {
    if (!ctx || N < 1 || D < 1 || D > kMaxD || !kind_supported(kind) || t < 1 || t > 16) return LGP_ERR_INVALID_ARG;
    const std::vector<int64_t> key = {pad_rows(N), (int64_t)D, (int64_t)kind, (int64_t)t};
    auto it = ctx->batch_routes.find(key);
    if (it == ctx->batch_routes.end()) return LGP_BATCH_UNTUNED;
    return it->second ? LGP_BATCH_TENSOR : LGP_BATCH_PERSISTENT;
}

lgp_status lgp_set_kernel_timing(lgp_ctx *ctx, int32_t on) {
    if (!ctx) return LGP_ERR_INVALID_ARG;
    LGP_CUDA(cudaSetDevice(ctx->device));
    if (on) {
        for (cudaEvent_t &e : ctx->kev)
            if (!e) LGP_CUDA(cudaEventCreate(&e));
    }
    ctx->kernel_timing = on != 0;
    ctx->kev_set = false;
    return LGP_OK;
}

lgp_status lgp_last_kernel_ms(lgp_ctx *ctx, float *ms) {
    if (!ctx || !ms) return LGP_ERR_INVALID_ARG;
    if (!ctx->kev_set) return fail(ctx, LGP_ERR_INVALID_ARG, "no product has been timed since timing was switched on");
    LGP_CUDA(cudaSetDevice(ctx->device));
    LGP_CUDA(cudaEventSynchronize(ctx->kev[1]));
    LGP_CUDA(cudaEventElapsedTime(ms, ctx->kev[0], ctx->kev[1]));
    return LGP_OK;
}

int32_t lgp_batch_split_choice(const lgp_ctx *ctx, int64_t N, int32_t D, int32_t kind, int32_t t) {
    if (!ctx || N < 1 || D < 1 || D > kMaxD || !kind_supported(kind) || t < 1 || t > 16) return LGP_ERR_INVALID_ARG;
    const std::vector<int64_t> key = {pad_rows(N), (int64_t)D, (int64_t)kind, (int64_t)t};
    auto it = ctx->batch_splits.find(key);
    return it == ctx->batch_splits.end() ? 0 : it->second;
}

int32_t lgp_batch_split_rule(const lgp_ctx *ctx, int64_t N) {
    if (!ctx || N < 1) return LGP_ERR_INVALID_ARG;
    return (int32_t)batch_split_rule(ctx, N);
}

lgp_status lgp_tc_distance_form(lgp_ctx *ctx, lgp_stream stream, int32_t *form, float *norm_max) {
    if (!ctx || !form) return LGP_ERR_INVALID_ARG;
    if (norm_max) *norm_max = -1.0f;
    if (ctx->sym_kind < 0) {
        *form = LGP_DIST_NONE;
        return LGP_OK;
    }
    if (!dot_form_allowed(ctx->sym_kind, ctx->sym_D)) {
        *form = LGP_DIST_DIFF;
        return LGP_OK;
    }
    LGP_CUDA(cudaSetDevice(ctx->device));
    LGP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    LGP_CUDA(cudaStreamSynchronize(ctx->work));
    unsigned int bits = 0;
    LGP_CUDA(cudaMemcpy(&bits, (const char *)ctx->vsplit.p + tc_dot_gate_offset(ctx->sym_Np, ctx->sym_t), sizeof bits,
                        cudaMemcpyDeviceToHost));
    float a;
    std::memcpy(&a, &bits, sizeof a);
    if (norm_max) *norm_max = a;
    *form = a <= dot_gate_limit(ctx->sym_kind) ? LGP_DIST_DOT : LGP_DIST_DIFF;
    return LGP_OK;
}

void lgp_set_wait_budget(lgp_ctx *ctx, int64_t cycles) {
    if (ctx) ctx->wait_budget = cycles > 0 ? cycles : kDefaultWaitBudget;
}

lgp_status lgp_check_device_status(lgp_ctx *ctx, lgp_stream stream) {
    if (!ctx) return LGP_ERR_INVALID_ARG;
    cudaStream_t user = (cudaStream_t)stream;
    LGP_CUDA(cudaSetDevice(ctx->device));
    LGP_CUDA(cudaStreamSynchronize(user));
    LGP_CUDA(cudaStreamSynchronize(ctx->work));
    LGP_CUDA(cudaMemcpy(ctx->h_flags, ctx->flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost));
    LGP_CUDA(cudaMemset(ctx->flags.p, 0, 4 * sizeof(int)));
    if (ctx->h_flags[1]) return fail(ctx, LGP_ERR_TIMEOUT, "a bounded device wait ran out (code %d)", ctx->h_flags[1]);
    return LGP_OK;
}

lgp_status lgp_kernel_matvec(lgp_ctx *ctx, const lgp_hyper *hyp, const float *X, const float *V, float *out,
                             int64_t N, int32_t t, int32_t prec, lgp_stream stream) {
    NvtxRange nvtx_range("lgp_kernel_matvec");
    if (!ctx) return LGP_ERR_INVALID_ARG;
    if (N < 1) return fail(ctx, LGP_ERR_INVALID_ARG, "N=%lld must be >= 1", (long long)N);
    if (t < 1 || t > kMaxT) return fail(ctx, LGP_ERR_UNSUPPORTED, "t=%d outside 1..%d", t, kMaxT);
    lgp_status s;
    LGP_CUDA(cudaSetDevice(ctx->device));
    if ((s = check_dev_ptr(ctx, X, "X")) || (s = check_dev_ptr(ctx, V, "V")) || (s = check_dev_ptr(ctx, out, "out")))
        return s;
    if (out == V || (const float *)out == X) return fail(ctx, LGP_ERR_INVALID_ARG, "out aliases an input");
    int tp = t;
    const int p = resolve_prec_padded(t, prec, &tp);
    if (p < 0) return fail(ctx, (lgp_status)p, "precision %d unsupported for t=%d", prec, t);
    cudaStream_t st = (cudaStream_t)stream;
    Prepared pp;
    if ((s = prepare_x(ctx, hyp, X, N, st, &pp)) != LGP_OK) return s;
    // an explicit split precision at other t: the product runs on tp zero-padded columns
    const float *Vu = V;
    float *Ou = out;
    if (tp != t) {
        if ((s = ensure(ctx, ctx->rhs, (size_t)pp.Np * tp * sizeof(float))) != LGP_OK ||
            (s = ensure(ctx, ctx->sr_x, (size_t)pp.Np * tp * sizeof(float))) != LGP_OK)
            return s;
        float *vpad = (float *)ctx->rhs.p;
        LGP_CUDA(cudaMemsetAsync(vpad, 0, (size_t)pp.Np * tp * sizeof(float), st));
        launch_copy_cols(V, t, vpad, tp, N, t, 0, st);
        LGP_CUDA(cudaGetLastError());
        Vu = vpad;
        Ou = (float *)ctx->sr_x.p;
    }
    if (is_tc(p)) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        LGP_CUDA(cudaStreamIsCapturing(st, &cap));
        if (cap == cudaStreamCaptureStatusNone && (s = autotune_tc(ctx, pp, Vu, tp, Ou, tp, tp, p, st)) != LGP_OK)
            return s;
    }
    if ((s = matvec_prepared(ctx, pp, Vu, tp, Ou, tp, tp, p, nullptr, st)) != LGP_OK) return s;
    if (tp != t) {
        launch_copy_cols(Ou, tp, out, t, N, t, 0, st);
        LGP_CUDA(cudaGetLastError());
    }
    return LGP_OK;
}

lgp_status lgp_kernel_matvec_grad(lgp_ctx *ctx, const lgp_hyper *hyp, const float *X, const float *W, float *dK_W,
                                  int64_t N, int32_t t, lgp_stream stream) {
    NvtxRange nvtx_range("lgp_kernel_matvec_grad");
    if (!ctx) return LGP_ERR_INVALID_ARG;
    if (N < 1) return fail(ctx, LGP_ERR_INVALID_ARG, "N=%lld must be >= 1", (long long)N);
    if (t < 1 || t > kMaxT) return fail(ctx, LGP_ERR_UNSUPPORTED, "t=%d outside 1..%d", t, kMaxT);
    lgp_status s;
    LGP_CUDA(cudaSetDevice(ctx->device));
    if ((s = check_dev_ptr(ctx, X, "X")) || (s = check_dev_ptr(ctx, W, "W")) || (s = check_dev_ptr(ctx, dK_W, "dK_W")))
        return s;
    if ((const float *)dK_W == W) return fail(ctx, LGP_ERR_INVALID_ARG, "dK_W aliases W");
    cudaStream_t st = (cudaStream_t)stream;
    Prepared pp;
    if ((s = prepare_x(ctx, hyp, X, N, st, &pp)) != LGP_OK) return s;
    const int64_t pf = mv_grad_partial_floats(N, pp.Np, t, pp.kp.D, ctx->num_sms);
    if ((s = ensure(ctx, ctx->mv_partial, (size_t)std::max<int64_t>(pf, 1) * sizeof(float))) != LGP_OK) return s;
    LGP_CUDA(launch_mv_grad(pp.kp, pp.xs, N, pp.Np, W, t, dK_W, (float *)ctx->mv_partial.p,
                            (int64_t)(ctx->mv_partial.bytes / sizeof(float)), ctx->num_sms, st));
    return LGP_OK;
}

lgp_status lgp_rademacher_probes(lgp_ctx *ctx, uint64_t seed, int64_t N, int32_t m, float *Z, int64_t ldz,
                                 lgp_stream stream) {
    if (!ctx) return LGP_ERR_INVALID_ARG;
    if (N < 1 || m < 1 || ldz < m) return fail(ctx, LGP_ERR_INVALID_ARG, "need N >= 1, m >= 1, ldz >= m");
    lgp_status s;
    LGP_CUDA(cudaSetDevice(ctx->device));
    if ((s = check_dev_ptr(ctx, Z, "Z"))) return s;
    launch_rademacher(seed, N, m, Z, ldz, 0, (cudaStream_t)stream);
    LGP_CUDA(cudaGetLastError());
    return LGP_OK;
}

lgp_status lgp_cg_solve(lgp_ctx *ctx, const lgp_hyper *hyp, const float *X, const float *B, float *Xsol, int64_t N,
                        int32_t t, const lgp_options *opt, int32_t *iters, double *rel_resid, lgp_stream stream) {
    NvtxRange nvtx_range("lgp_cg_solve");
    if (!ctx) return LGP_ERR_INVALID_ARG;
    if (N < 1) return fail(ctx, LGP_ERR_INVALID_ARG, "N=%lld must be >= 1", (long long)N);
    if (t < 1 || t > kMaxT) return fail(ctx, LGP_ERR_UNSUPPORTED, "t=%d outside 1..%d", t, kMaxT);
    lgp_status s;
    if ((s = check_opts(ctx, opt, false)) != LGP_OK) return s;
    LGP_CUDA(cudaSetDevice(ctx->device));
    if ((s = check_dev_ptr(ctx, X, "X")) || (s = check_dev_ptr(ctx, B, "B")) || (s = check_dev_ptr(ctx, Xsol, "Xsol")))
        return s;
    if ((const float *)Xsol == B) return fail(ctx, LGP_ERR_INVALID_ARG, "Xsol aliases B");
    int tp = t;
    const int prec = resolve_prec_padded(t, opt->prec, &tp);
    if (prec < 0) return fail(ctx, (lgp_status)prec, "precision %d unsupported for t=%d", opt->prec, t);
    cudaStream_t user = (cudaStream_t)stream;
    if ((s = enter(ctx, user)) != LGP_OK) return s;
    cudaStream_t st = ctx->work;
    LGP_CUDA(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), st));
    Prepared pp;
    if ((s = prepare_x(ctx, hyp, X, N, st, &pp)) != LGP_OK) return s;
    // an explicit split precision at other t: the solve runs on tp columns, the extra ones zero (a zero
    // column takes no iteration), and the warm start, if any, is padded the same way
    const float *Bu = B;
    const float *x0 = (opt->flags & LGP_OPT_WARM_START) ? Xsol : nullptr;
    if (tp != t) {
        if ((s = ensure(ctx, ctx->rhs, (size_t)pp.Np * tp * sizeof(float))) != LGP_OK ||
            (s = ensure(ctx, ctx->sr_x, (size_t)pp.Np * tp * sizeof(float))) != LGP_OK)
            return s;
        float *bpad = (float *)ctx->rhs.p;
        LGP_CUDA(cudaMemsetAsync(bpad, 0, (size_t)pp.Np * tp * sizeof(float), st));
        launch_copy_cols(B, t, bpad, tp, N, t, 0, st);
        if (x0) {
            float *x0pad = (float *)ctx->sr_x.p;
            LGP_CUDA(cudaMemsetAsync(x0pad, 0, (size_t)pp.Np * tp * sizeof(float), st));
            launch_copy_cols(Xsol, t, x0pad, tp, N, t, 0, st);
            x0 = x0pad;
        }
        LGP_CUDA(cudaGetLastError());
        Bu = bpad;
    }
    Precond pc;
    if (opt->precond_rank > 0 && (s = build_precond(ctx, hyp, X, pp, opt->precond_rank, tp, &pc)) != LGP_OK) return s;
    CgBuffers b;
    if ((s = run_cg(ctx, pp, Bu, tp, tp, opt, 0, prec, &b, nullptr, opt->precond_rank > 0 ? &pc : nullptr, x0)) !=
        LGP_OK)
        return s;
    if (tp != t)
        launch_copy_cols(b.x, tp, Xsol, t, N, t, 0, st);
    else
        launch_cg_copy_out(b, N, t, Xsol, t, st);
    LGP_CUDA(cudaGetLastError());
    LGP_CUDA(cudaMemcpyAsync(ctx->h_flags, ctx->flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->work));
    if ((s = leave_sync(ctx, user)) != LGP_OK) return s;
    if (ctx->h_flags[1]) return fail(ctx, LGP_ERR_TIMEOUT, "a bounded device wait ran out (code %d)", ctx->h_flags[1]);
    return cg_status_of(ctx, *ctx->h_state, t, iters, rel_resid, ctx->h_flags[0]);
}

lgp_status lgp_lml_and_grad(lgp_ctx *ctx, const lgp_hyper *hyp, const float *X, const float *y, int64_t N,
                            const lgp_options *opt, double *lml, double *grad, lgp_lml_info *info,
                            lgp_stream stream) {
    NvtxRange nvtx_range("lgp_lml_and_grad");
    if (!ctx) return LGP_ERR_INVALID_ARG;
    if (N < 1) return fail(ctx, LGP_ERR_INVALID_ARG, "N=%lld must be >= 1", (long long)N);
    lgp_status s;
    if ((s = check_opts(ctx, opt, true)) != LGP_OK) return s;
    LGP_CUDA(cudaSetDevice(ctx->device));
    if ((s = check_dev_ptr(ctx, X, "X")) || (s = check_dev_ptr(ctx, y, "y"))) return s;
    const int t = opt->n_probes + 1;
    const int L = opt->lanczos_steps;
    const bool single = (opt->flags & LGP_OPT_SINGLE_RHS) != 0;
    if (single && opt->precond_rank > 0)
        return fail(ctx, LGP_ERR_UNSUPPORTED, "the single-column path runs without a preconditioner");
    const int prec = single ? (int)LGP_PREC_FP32 : resolve_prec(t, opt->prec);
    if (prec < 0) return fail(ctx, (lgp_status)prec, "precision %d unsupported for t=%d", opt->prec, t);
    cudaStream_t user = (cudaStream_t)stream;
    if ((s = enter(ctx, user)) != LGP_OK) return s;
    cudaStream_t st = ctx->work;
    LGP_CUDA(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), st));
    Prepared pp;
    if ((s = prepare_x(ctx, hyp, X, N, st, &pp)) != LGP_OK) return s;
    // right-hand-side block [y, z_1..z_m]: Rademacher probes, or probes with covariance P
    // (z = L e1 + sigma e2 from a Rademacher block of N + k rows) when preconditioned
    const int k = opt->precond_rank;
    Precond pc;
    if (k > 0 && (s = build_precond(ctx, hyp, X, pp, k, t, &pc)) != LGP_OK) return s;
    if ((s = ensure(ctx, ctx->rhs, (size_t)pp.Np * t * sizeof(float))) != LGP_OK) return s;
    float *rhs = (float *)ctx->rhs.p;
    launch_copy_cols(y, 1, rhs, t, N, 1, 0, st);
    if (k > 0) {
        if ((s = ensure(ctx, ctx->pc_e, (size_t)(N + k) * (t - 1) * sizeof(float))) != LGP_OK) return s;
        launch_rademacher(opt->seed, N + k, t - 1, (float *)ctx->pc_e.p, t - 1, 0, st);
        launch_precond_probes(pc.L64, pc.Np, k, (const float *)ctx->pc_e.p, N, t - 1, std::sqrt(pc.noise), rhs, t, 1,
                              st);
    } else {
        launch_rademacher(opt->seed, N, t - 1, rhs, t, 1, st);
    }
    LGP_CUDA(cudaGetLastError());
    CgBuffers b;
    int chunks = 0;
    if (single) {
        if ((s = run_cg_columns(ctx, pp, rhs, t, opt, L, &b, &chunks)) != LGP_OK) return s;
    } else if ((s = run_cg(ctx, pp, rhs, t, t, opt, L, prec, &b, &chunks, k > 0 ? &pc : nullptr)) != LGP_OK) {
        return s;
    }
    // the probe side of the trace terms: P^{-1} z_c (z_c itself without a preconditioner); column 0 stays y
    const float *rhs_t = rhs;
    if (k > 0) {
        if ((s = ensure(ctx, ctx->pc_rhs, (size_t)pp.Np * t * sizeof(float))) != LGP_OK) return s;
        float *prhs = (float *)ctx->pc_rhs.p;
        launch_precond_apply(b.pc, rhs, t, prhs, t, nullptr, N, t, nullptr, b.G, nullptr, st);
        launch_copy_cols(y, 1, prhs, t, N, 1, 0, st);
        LGP_CUDA(cudaGetLastError());
        rhs_t = prhs;
    }
    // scalars: dots[0..2t), slq[4], grad[D+2]
    const int G = b.G;
    if ((s = ensure(ctx, ctx->scal, (size_t)(2 * kMaxT + 4 + kMaxD + 2) * sizeof(double))) != LGP_OK) return s;
    double *dots = (double *)ctx->scal.p;
    double *slq = dots + 2 * kMaxT;
    double *gdev = slq + 4;
    launch_col_dots(b.x, rhs_t, N, t, b.partial, G, dots, st);
    launch_slq_lml(b, t, L, dots, N, slq, st);
    LGP_CUDA(cudaGetLastError());
    if (grad && !single) {
        if ((s = ensure(ctx, ctx->adj_b, (size_t)pp.Np * t * sizeof(float))) != LGP_OK) return s;
        const int64_t pd = adjoint_partial_doubles(N, t, pp.kp.D, ctx->num_sms);
        if ((s = ensure(ctx, ctx->adj_partial, (size_t)pd * sizeof(double))) != LGP_OK) return s;
        launch_adjoint_rhs(b.x, rhs_t, N, t, (float *)ctx->adj_b.p, st);
        int nblk = 0;
        LGP_CUDA(launch_adjoint_bilinear(pp.kp, pp.xs, N, pp.Np, b.x, (const float *)ctx->adj_b.p, t,
                                         (double *)ctx->adj_partial.p, pd, &nblk, ctx->num_sms, st));
        launch_grad_finalize((const double *)ctx->adj_partial.p, nblk, pp.kp.D, dots, t, pp.kp.noise, gdev, st);
        LGP_CUDA(cudaGetLastError());
    } else if (grad) {
        // single-column path: one adjoint pass per column (its solution against its right-hand side), the
        // block partials of column c in region c; the finalisation sums all regions
        if ((s = ensure(ctx, ctx->adj_b, (size_t)pp.Np * t * sizeof(float))) != LGP_OK) return s;
        const int64_t pd = adjoint_partial_doubles(N, 1, pp.kp.D, ctx->num_sms);
        if ((s = ensure(ctx, ctx->adj_partial, (size_t)pd * t * sizeof(double))) != LGP_OK) return s;
        if ((s = ensure(ctx, ctx->sr_tmp, (size_t)2 * pp.Np * sizeof(float))) != LGP_OK) return s;
        float *adj_b = (float *)ctx->adj_b.p, *ta = (float *)ctx->sr_tmp.p, *tb = ta + pp.Np;
        launch_adjoint_rhs(b.x, rhs_t, N, t, adj_b, st);
        int nblk = 0;
        for (int c = 0; c < t; ++c) {
            launch_copy_cols(b.x + c, t, ta, 1, N, 1, 0, st);
            launch_copy_cols(adj_b + c, t, tb, 1, N, 1, 0, st);
            LGP_CUDA(launch_adjoint_bilinear(pp.kp, pp.xs, N, pp.Np, ta, tb, 1, (double *)ctx->adj_partial.p + c * pd,
                                             pd, &nblk, ctx->num_sms, st));
        }
        if ((int64_t)nblk * (pp.kp.D + 1) != pd)
            return fail(ctx, LGP_ERR_CUDA, "adjoint partial layout mismatch (%d blocks)", nblk);
        launch_grad_finalize((const double *)ctx->adj_partial.p, nblk * t, pp.kp.D, dots, t, pp.kp.noise, gdev, st);
        LGP_CUDA(cudaGetLastError());
    }
    LGP_CUDA(cudaMemcpyAsync(ctx->h_scal, dots, (size_t)(2 * kMaxT + 4 + kMaxD + 2) * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
    LGP_CUDA(cudaMemcpyAsync(ctx->h_flags, ctx->flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    if ((s = leave_sync(ctx, user)) != LGP_OK) return s;
    if (ctx->h_flags[1]) return fail(ctx, LGP_ERR_TIMEOUT, "a bounded device wait ran out (code %d)", ctx->h_flags[1]);
    std::vector<int> it(t);
    std::vector<double> rel(t);
    lgp_status cs = cg_status_of(ctx, *ctx->h_state, t, it.data(), rel.data(), ctx->h_flags[0]);
    if (cs < 0) return cs;
    const double *hs = ctx->h_scal + 2 * kMaxT;
    if (hs[3] != 0.0) return fail(ctx, LGP_ERR_NONFINITE, "non-positive Ritz value in a Lanczos tridiagonal");
    if (lml) *lml = hs[0];
    if (grad)
        for (int p = 0; p < pp.kp.D + 2; ++p) grad[p] = hs[4 + p];
    if (info) {
        info->lml = hs[0];
        info->quad = hs[1];
        info->logdet = hs[2];
        info->t = t;
        info->prec_used = prec;
        info->iters_max = *std::max_element(it.begin(), it.end());
        info->iters_min = *std::min_element(it.begin(), it.end());
        info->max_rel_resid = *std::max_element(rel.begin(), rel.end());
        // chunks the device loop ran (each: kChunk iterations + the condition kernel)
        const int ran = ctx->h_state->loop_chunks;
        info->cg_chunks = ran;
        info->logdet_precond = k > 0 ? pc.logdet : 0.0;
        (void)chunks;
        // prep_x, y copy, probes, CG init (2), the loop's chunks, column dots (2), SLQ (2), adjoint (3)
        // preconditioned: 3 more launches per iteration and in the CG init; the build (init, 2 per rank step, Gram,
        // float32 copy), the P-distributed probes, and P^{-1} of the probe block with the y copy
        const int pc_iter = k > 0 ? 3 : 0;
        const int pc_once = k > 0 ? (2 * k + 3) + 3 + 1 + 4 : 0;
        // the products' X-only operands, built once before the loop (transpose; box and operands of the dot form)
        const int opnd_once = is_tc(prec) && tc_operands_valid(ctx, pp, t, prec) ? (ctx->opnd_dot ? 3 : 1) : 0;
        if (!single) {
            info->launches = 3 + 2 +
                             ran * (kChunk * (cg_iteration_launches(ctx, pp, t, prec, ctx->cg_dist_form) + pc_iter) + 1) +
                             2 + 2 + (grad ? 3 : 0) + pc_once + opnd_once;
        } else {
            // per column: CG init (2), copy and gather (2); the chunks of all columns; per column in the
            // gradient: two column copies and one adjoint pass
            info->launches = 3 + 4 * t + ran * (kChunk * (mv_simt_launches(pp.N, pp.Np, 1, ctx->num_sms) + 5) + 1) +
                             2 + 2 + (grad ? 2 + 3 * t : 0);
        }
    }
    return cs;
}

// Column count of a prediction solve block: padded with zero columns (inactive from the start) up to
// 16 or 32 when the tensor-core product can then take the block, else t itself.
static int predict_width(int t, int req_prec) {
    if (req_prec == LGP_PREC_FP32 || t <= 8 || !tc_supported(16)) return t;
    return t <= 16 ? 16 : 32;
}

lgp_status lgp_predict(lgp_ctx *ctx, const lgp_hyper *hyp, const float *X, const float *y, int64_t N,
                       const float *Xs, int64_t M, const lgp_options *opt, float *mean, float *var,
                       lgp_predict_info *info, lgp_stream stream) {
    NvtxRange nvtx_range("lgp_predict");
    constexpr int kChunkCols = 32;
    if (!ctx) return LGP_ERR_INVALID_ARG;
    if (N < 1) return fail(ctx, LGP_ERR_INVALID_ARG, "N=%lld must be >= 1", (long long)N);
    if (M < 1) return fail(ctx, LGP_ERR_INVALID_ARG, "M=%lld must be >= 1", (long long)M);
    lgp_status s;
    if ((s = check_opts(ctx, opt, false)) != LGP_OK) return s;
    const int m = var ? opt->n_probes : 0;
    if (m < 0 || m > kChunkCols - 1)
        return fail(ctx, LGP_ERR_UNSUPPORTED, "n_probes=%d outside 0..%d", opt->n_probes, kChunkCols - 1);
    LGP_CUDA(cudaSetDevice(ctx->device));
    if ((s = check_dev_ptr(ctx, X, "X")) || (s = check_dev_ptr(ctx, y, "y")) || (s = check_dev_ptr(ctx, Xs, "Xs")) ||
        (s = check_dev_ptr(ctx, mean, "mean")))
        return s;
    if (var && (s = check_dev_ptr(ctx, var, "var")) != LGP_OK) return s;
    if (var == mean) return fail(ctx, LGP_ERR_INVALID_ARG, "var aliases mean");
    cudaStream_t user = (cudaStream_t)stream;
    if ((s = enter(ctx, user)) != LGP_OK) return s;
    cudaStream_t st = ctx->work;
    LGP_CUDA(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), st));
    Prepared pp;
    if ((s = prepare_x(ctx, hyp, X, N, st, &pp)) != LGP_OK) return s;
    // test points, prescaled like X (their non-finite check shares the flag of X)
    const int64_t Mp = pad_rows(M);
    if ((s = ensure(ctx, ctx->pred_xs, (size_t)Mp * pp.kp.dpad * sizeof(float))) != LGP_OK) return s;
    float *xs_star = (float *)ctx->pred_xs.p;
    launch_prep_x(Xs, M, pp.kp.D, pp.kp.dpad, pp.kp.scale, xs_star, Mp, (int *)ctx->flags.p, st);
    LGP_CUDA(cudaGetLastError());

    Precond pc;
    if (opt->precond_rank > 0 &&
        (s = build_precond(ctx, hyp, X, pp, opt->precond_rank, m > 0 ? m + 1 : kChunkCols, &pc)) != LGP_OK)
        return s;
    const Precond *pcp = opt->precond_rank > 0 ? &pc : nullptr;
    int solves = 0, iters_max = 0, prec_first = LGP_PREC_FP32;
    double rel_max = 0.0;
    bool unconverged = false;
    // one batched CG solve of the block rhs [Np, t]; its state is checked on the host
    auto solve = [&](const float *rhs, int t, CgBuffers *b) -> lgp_status {
        int prec = opt->prec;
        if (prec != LGP_PREC_FP32 && !(tc_supported(t) && (t == 16 || t == 32))) prec = LGP_PREC_FP32;
        prec = resolve_prec(t, prec);
        if (prec < 0) return fail(ctx, (lgp_status)prec, "precision %d unsupported for t=%d", opt->prec, t);
        if (solves == 0) prec_first = prec;
        lgp_status r = run_cg(ctx, pp, rhs, t, t, opt, 0, prec, b, nullptr, pcp);
        if (r != LGP_OK) return r;
        LGP_CUDA(cudaMemcpyAsync(ctx->h_flags, ctx->flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
        LGP_CUDA(cudaStreamSynchronize(st));
        if (ctx->h_flags[1]) return fail(ctx, LGP_ERR_TIMEOUT, "a bounded device wait ran out (code %d)", ctx->h_flags[1]);
        std::vector<int> it(t);
        std::vector<double> rel(t);
        const lgp_status cs = cg_status_of(ctx, *ctx->h_state, t, it.data(), rel.data(), ctx->h_flags[0]);
        if (cs < 0) return cs;
        unconverged |= cs == LGP_WARN_NOT_CONVERGED;
        ++solves;
        iters_max = std::max(iters_max, *std::max_element(it.begin(), it.end()));
        rel_max = std::max(rel_max, *std::max_element(rel.begin(), rel.end()));
        return LGP_OK;
    };
    // out [Nr, ldo] = K(rows, cols) V on the FP32 cross product
    auto cross = [&](const float *xr, int64_t nr, int64_t npr, const float *xc, int64_t nc, int64_t npc, const float *V,
                     int64_t ldv, int t, float *out, int64_t ldo) -> lgp_status {
        const int64_t pf = mv_simt_cross_partial_floats(nr, npr, nc, t, ctx->num_sms);
        lgp_status r = ensure(ctx, ctx->mv_partial, (size_t)std::max<int64_t>(pf, 1) * sizeof(float));
        if (r != LGP_OK) return r;
        MvLaunch mm;
        mm.kp = &pp.kp;
        mm.Xs = xc;
        mm.N = nc;
        mm.Np = npc;
        mm.V = V;
        mm.ldv = ldv;
        mm.out = out;
        mm.ldo = ldo;
        mm.t = t;
        mm.partial = (float *)ctx->mv_partial.p;
        mm.partial_cap = (int64_t)(ctx->mv_partial.bytes / sizeof(float));
        mm.skip = nullptr;
        mm.num_sms = ctx->num_sms;
        mm.Xr = xr;
        mm.Nr = nr;
        mm.Npr = npr;
        LGP_CUDA(launch_mv_simt(mm, st));
        return LGP_OK;
    };

    if (m > 0) {
        // probe route: one solve of [y, K_f* Z], then Q = K_*f K_y^{-1} K_f* Z
        const int t = m + 1;
        if ((s = ensure(ctx, ctx->rhs, (size_t)pp.Np * t * sizeof(float))) != LGP_OK) return s;
        if ((s = ensure(ctx, ctx->pred_z, (size_t)Mp * m * sizeof(float))) != LGP_OK) return s;
        if ((s = ensure(ctx, ctx->pred_q, (size_t)Mp * m * sizeof(float))) != LGP_OK) return s;
        float *rhs = (float *)ctx->rhs.p, *Z = (float *)ctx->pred_z.p, *Q = (float *)ctx->pred_q.p;
        launch_rademacher(opt->seed, M, m, Z, m, 0, st);
        launch_copy_cols(y, 1, rhs, t, N, 1, 0, st);
        LGP_CUDA(cudaGetLastError());
        if ((s = cross(pp.xs, N, pp.Np, xs_star, M, Mp, Z, m, m, rhs + 1, t)) != LGP_OK) return s;
        CgBuffers b;
        if ((s = solve(rhs, t, &b)) != LGP_OK) return s;
        if ((s = cross(xs_star, M, Mp, pp.xs, N, pp.Np, b.x, t, 1, mean, 1)) != LGP_OK) return s;
        if ((s = cross(xs_star, M, Mp, pp.xs, N, pp.Np, b.x + 1, t, m, Q, m)) != LGP_OK) return s;
        launch_var_from_probes(Z, m, Q, m, M, m, pp.kp.s2, var, st);
        LGP_CUDA(cudaGetLastError());
    } else {
        // exact route: blocks [y, k(X, x*_0..)] then [k(X, x*_j0..)], up to 32 columns each
        if ((s = ensure(ctx, ctx->scal, (size_t)(2 * kMaxT + 4 + kMaxD + 2) * sizeof(double))) != LGP_OK) return s;
        int64_t j0 = 0;
        for (bool first = true; first || (var && j0 < M); first = false) {
            const int lead = first ? 1 : 0;
            const int tc = var ? (int)std::min<int64_t>(kChunkCols - lead, M - j0) : 0;
            const int t = predict_width(lead + tc, opt->prec);
            if ((s = ensure(ctx, ctx->rhs, (size_t)pp.Np * t * sizeof(float))) != LGP_OK) return s;
            float *rhs = (float *)ctx->rhs.p;
            if (t > lead + tc) LGP_CUDA(cudaMemsetAsync(rhs, 0, (size_t)pp.Np * t * sizeof(float), st));
            if (first) launch_copy_cols(y, 1, rhs, t, N, 1, 0, st);
            if (tc) launch_kernel_cols(pp.kp, pp.xs, N, pp.Np, xs_star, j0, tc, rhs, t, lead, st);
            LGP_CUDA(cudaGetLastError());
            CgBuffers b;
            if ((s = solve(rhs, t, &b)) != LGP_OK) return s;
            if (first && (s = cross(xs_star, M, Mp, pp.xs, N, pp.Np, b.x, t, 1, mean, 1)) != LGP_OK) return s;
            if (tc) {
                double *dots = (double *)ctx->scal.p;
                launch_col_dots(b.x, rhs, N, t, b.partial, b.G, dots, st);
                launch_var_from_dots(dots, lead, lead + tc, pp.kp.s2, var, j0, st);
                LGP_CUDA(cudaGetLastError());
            }
            j0 += tc;
        }
    }
    LGP_CUDA(cudaMemcpyAsync(ctx->h_flags, ctx->flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    if ((s = leave_sync(ctx, user)) != LGP_OK) return s;
    if (ctx->h_flags[1]) return fail(ctx, LGP_ERR_TIMEOUT, "a bounded device wait ran out (code %d)", ctx->h_flags[1]);
    if (ctx->h_flags[0]) return fail(ctx, LGP_ERR_NONFINITE, "X or Xs contains NaN or Inf");
    if (info) {
        info->solves = solves;
        info->iters_max = iters_max;
        info->max_rel_resid = rel_max;
        info->var_probes = m;
        info->prec_used = prec_first;
    }
    if (unconverged) {
        fail(ctx, LGP_WARN_NOT_CONVERGED, "CG reached max_iter before tol on some column");
        return LGP_WARN_NOT_CONVERGED;
    }
    return LGP_OK;
}

lgp_status lgp_batch_cg_solve(lgp_ctx *ctx, int32_t n_gp, const lgp_hyper *hyp, const float *const *X,
                              const float *const *B, float *const *Xsol, const int64_t *N, int32_t t,
                              const lgp_options *opt, int32_t *iters, double *rel_resid, lgp_stream stream) {
    NvtxRange nvtx_range("lgp_batch_cg_solve");
    if (!ctx) return LGP_ERR_INVALID_ARG;
    if (n_gp < 1 || n_gp > 4096) return fail(ctx, LGP_ERR_UNSUPPORTED, "n_gp=%d outside 1..4096", n_gp);
    if (t < 1 || t > 16) return fail(ctx, LGP_ERR_UNSUPPORTED, "batched solve supports 1 <= t <= 16 (got %d)", t);
    if (!hyp || !X || !B || !Xsol || !N) return fail(ctx, LGP_ERR_INVALID_ARG, "NULL problem array");
    lgp_status s;
    if ((s = check_opts(ctx, opt, false)) != LGP_OK) return s;
    LGP_CUDA(cudaSetDevice(ctx->device));
    std::vector<KernelParams> kps_all(n_gp);
    for (int g = 0; g < n_gp; ++g) {
        if (N[g] < 1) return fail(ctx, LGP_ERR_INVALID_ARG, "N[%d]=%lld must be >= 1", g, (long long)N[g]);
        if ((s = make_params(ctx, &hyp[g], &kps_all[g])) != LGP_OK) return s;
        char nm[32];
        snprintf(nm, sizeof nm, "X[%d]", g);
        if ((s = check_dev_ptr(ctx, X[g], nm))) return s;
        snprintf(nm, sizeof nm, "B[%d]", g);
        if ((s = check_dev_ptr(ctx, B[g], nm))) return s;
        snprintf(nm, sizeof nm, "Xsol[%d]", g);
        if ((s = check_dev_ptr(ctx, Xsol[g], nm))) return s;
        if ((const float *)Xsol[g] == B[g]) return fail(ctx, LGP_ERR_INVALID_ARG, "Xsol[%d] aliases B[%d]", g, g);
    }
    cudaStream_t user = (cudaStream_t)stream;
    if ((s = enter(ctx, user)) != LGP_OK) return s;
    cudaStream_t st = ctx->work;
    LGP_CUDA(cudaMemsetAsync(ctx->flags.p, 0, 4 * sizeof(int), st));
    // Route of each problem (timed once per shape): large problems whose tensor-core product measures
    // faster solve on their own with it; the rest share the persistent batch launch.
    std::vector<int> bids;  // problems of the persistent batch launch
    std::vector<int> tc_ids;
    for (int g = 0; g < n_gp; ++g) {
        int route = 0;
        if (opt->prec != LGP_PREC_FP32 && (s = batch_route(ctx, &hyp[g], X[g], N[g], B[g], t, &route)) != LGP_OK)
            return s;
        (route ? tc_ids : bids).push_back(g);
    }
    ctx->last_batch_tc = (int)tc_ids.size();
    bool unconverged = false;
    for (int g : tc_ids) {
        if ((s = batch_tc_solve(ctx, &hyp[g], X[g], B[g], Xsol[g], N[g], t, opt, iters ? iters + (int64_t)g * t : nullptr,
                                rel_resid ? rel_resid + (int64_t)g * t : nullptr, &unconverged)) != LGP_OK)
            return s;
    }
    if (bids.empty()) {
        if ((s = leave_sync(ctx, user)) != LGP_OK) return s;
        if (unconverged) {
            fail(ctx, LGP_WARN_NOT_CONVERGED, "some batched column reached max_iter before tol");
            return LGP_WARN_NOT_CONVERGED;
        }
        return LGP_OK;
    }
    const int n_b = (int)bids.size();
    // the work list of the persistent launch: each problem's column splits timed per shape (the problem
    // alone), then every persistent-route problem with its own splits
    BatchPlan P;
    for (int q = 0; q < n_b; ++q) {
        const int g = bids[q];
        int64_t S = 1;
        if ((s = batch_split_choice(ctx, kps_all[g], &hyp[g], X[g], B[g], N[g], t, &S)) != LGP_OK) return s;
        plan_add_problem(P, N[g], kps_all[g], X[g], B[g], Xsol[g], t, S);
    }
    const int ng_t = n_b * t;
    BatchArgs A;
    if ((s = upload_batch_plan(ctx, P, t, st, &A)) != LGP_OK) return s;
    LGP_CUDA(launch_batch_init(A, opt->tol, opt->max_iter, st));

    // one graph: a conditional WHILE node whose body is a chunk of iterations plus the condition kernel,
    // so every iteration of every problem runs without a host round trip
    cudaGraph_t graph = nullptr;
    LGP_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    cudaError_t ce = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    alignas(cudaGraphNodeParams) unsigned char np_storage[sizeof(cudaGraphNodeParams)] = {};
    cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(np_storage);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (ce == cudaSuccess) ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    if (ce == cudaSuccess)
        ce = cudaStreamBeginCaptureToGraph(st, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(ctx, LGP_ERR_CUDA, "batch conditional graph: %s", cudaGetErrorString(ce));
    }
    for (int k = 0; k < kChunk && ce == cudaSuccess; ++k) ce = launch_batch_iteration(A, ctx->num_sms, st);
    if (ce == cudaSuccess) ce = launch_batch_loop_condition(h, A, st);
    cudaGraph_t captured = nullptr;
    cudaError_t ce2 = cudaStreamEndCapture(st, &captured);
    if (ce != cudaSuccess || ce2 != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(ctx, LGP_ERR_CUDA, "batch graph capture failed: %s",
                    cudaGetErrorString(ce != cudaSuccess ? ce : ce2));
    }
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(ctx, LGP_ERR_CUDA, "batch graph instantiate failed: %s", cudaGetErrorString(ce));
    ce = cudaGraphLaunch(exec, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    cudaGraphExecDestroy(exec);
    if (ce != cudaSuccess) return fail(ctx, LGP_ERR_CUDA, "batch loop failed: %s", cudaGetErrorString(ce));
    LGP_CUDA(launch_batch_copy_out(A, st));
    std::vector<int> h_it(ng_t), h_act(ng_t);
    std::vector<double> h_rr(ng_t), h_b2(ng_t);
    BatchState h_st;
    LGP_CUDA(cudaMemcpyAsync(h_it.data(), A.iters, ng_t * sizeof(int), cudaMemcpyDeviceToHost, st));
    LGP_CUDA(cudaMemcpyAsync(h_act.data(), A.active, ng_t * sizeof(int), cudaMemcpyDeviceToHost, st));
    LGP_CUDA(cudaMemcpyAsync(h_rr.data(), A.rr, ng_t * sizeof(double), cudaMemcpyDeviceToHost, st));
    LGP_CUDA(cudaMemcpyAsync(h_b2.data(), A.bnorm2, ng_t * sizeof(double), cudaMemcpyDeviceToHost, st));
    LGP_CUDA(cudaMemcpyAsync(&h_st, A.st, sizeof(BatchState), cudaMemcpyDeviceToHost, st));
    LGP_CUDA(cudaMemcpyAsync(ctx->h_flags, ctx->flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    if ((s = leave_sync(ctx, user)) != LGP_OK) return s;
    if (ctx->h_flags[0]) return fail(ctx, LGP_ERR_NONFINITE, "some X[g] contains NaN or Inf");
    for (int k = 0; k < ng_t; ++k) {
        const int64_t dst = (int64_t)bids[k / t] * t + k % t;
        if (iters) iters[dst] = h_it[k];
        if (rel_resid) rel_resid[dst] = h_b2[k] > 0.0 ? std::sqrt(h_rr[k] / h_b2[k]) : 0.0;
        if (h_act[k]) unconverged = true;
    }
    if (h_st.status & 1) return fail(ctx, LGP_ERR_NONFINITE, "non-finite value in some B[g] or a CG scalar");
    if (h_st.status & 2) return fail(ctx, LGP_ERR_BREAKDOWN, "CG breakdown in a batched problem");
    if (unconverged) {
        fail(ctx, LGP_WARN_NOT_CONVERGED, "some batched column reached max_iter before tol");
        return LGP_WARN_NOT_CONVERGED;
    }
    return LGP_OK;
}

}  // extern "C"
