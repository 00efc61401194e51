// C ABI of the SPARKLING GB300 library (declared in include/sparkling.h).
//
// Host-side orchestration only: argument validation, the device workspace,
// the even work split of the pair kernels, the autotuner, the batched step's
// work list and CUDA graph, the multi-resolution driver's loop and
// checkpoints, launch bookkeeping (counts and optional CUDA-event timing) and
// status reporting.  All arithmetic of the hot path runs in the kernels of
// the other csrc/ files.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/sparkling.h"
#include "kernels.h"

using namespace sparkling;

// SPARKLING_STEP_AUTO: steps of this many samples or more take the
// persistent engine (measured faster on the 1e7-sample workload).
constexpr int64_t kStepEngineMin = (int64_t)1 << 22;

struct sparkling_ctx {
    int device = 0;
    bool inited = false;
    int sms = 0;
    int *d_status = nullptr;    // device control block (DevCtl): status word, wait budget
    long long wait_cycles = kWaitCycles;   // budget of the kernels' bounded waits
    size_t mem_limit = 0;       // cap on the context's device allocations (0: none)
    int proj_mode = SPARKLING_PROJECTION_FP64;
    int step_path = SPARKLING_STEP_AUTO;
    double *d_small = nullptr;  // [0..1] energy, [2..5] violation bits, [6] notconv (int)
    void *ws = nullptr;
    size_t ws_bytes = 0;
    // host-buffer entry points keep their device copies here
    void *h_K = nullptr;
    size_t h_K_bytes = 0;
    float *h_rho = nullptr;
    size_t h_rho_bytes = 0;
    std::string err;
    bool timing = false;
    struct Pending { int kind; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    double ms[SPARKLING_KERNEL_COUNT] = {};
    int64_t nlaunch[SPARKLING_KERNEL_COUNT] = {};
    int64_t launches = 0;
    // occupancy cache [acc][energy][variant] (the directed repulsion has no
    // plain FP64-accumulate form: it runs with the FP64 fold, rep_acc())
    int occ_attr[3][2][kAttrVariants] = {};
    int occ_rep[2][2][kRepVariants] = {};
    bool occ_done = false;
    // autotuner: tile shape per (acc, padded row length) for the attraction
    // and per acc for the repulsion; -1 = not tuned yet
    bool autotune = true;
    std::vector<std::pair<int64_t, int>> attr_choice;   // key acc * 2^20 + gxp
    int rep_choice[2] = {-1, -1};
    bool rep_symmetric = true;     // repulsion: symmetric kernel (else the directed shapes)
    int occ_sym[2][kSymVariants] = {};
    int sym_choice = -1;           // shape of the symmetric kernel (tuned or pinned; -1: none)
    int pin_attr = -1;             // attraction shape pinned by sparkling_set_shape
    std::string tune_log;
    // batched step: cached work list, workspace layout and CUDA graph
    struct Batch {
        bool valid = false;
        int B = 0, Ns = 0, acc = -1, dtype = -1, ctas = 0, items_per_cta = 0;
        int64_t n_pair_items = 0;
        int64_t n_lead_items = 0;         // pair items ahead of the first projection item
        std::vector<double> item_pairs;   // pair count of every item (0: projection)
        std::vector<int64_t> off;
        std::vector<int32_t> dims;
        std::vector<EngineTraj> traj;
        std::vector<EngineItem> items;
        std::vector<size_t> o_rho, o_coords;
        size_t o_pos = 0, o_traj = 0, o_items = 0, o_cnt = 0, o_part = 0, o_gstate = 0, end = 0;
        bool sym = false;                 // repulsion by the batched symmetric kernel
        bool one_launch = false;          // symmetric repulsion items in the engine's work list
        bool roles = false;               // role dispatch over the list's three parts
        int32_t n_attr = 0, n_sym = 0;    // sizes of its attraction and symmetric parts
        int32_t wait_scale = 4;           // projection waits: this many wait budgets
        size_t o_racc = 0, o_symtraj = 0;
        int64_t sym_units = 0;
        std::vector<SymTraj> symtraj;
        bool proj_in_smem = false;
        int64_t kernels_per_step = 0;
        // graph of the device work of one step (counters, packs, engine)
        cudaGraphExec_t exec = nullptr;
        std::vector<const void *> graph_key;
        int graph_variant = -1;
        float graph_eps2 = -1.f;          // eps^2 baked into the captured launch
        int graph_proj = -1;              // projection mode baked into the captured launch
        int eager_calls = 0;
    } batch;
    cudaStream_t cap_stream = nullptr;  // private stream the batched step is captured on
    EngineTraj *h_traj = nullptr;   // pinned staging of the trajectory descriptors
    size_t h_traj_cap = 0;
    int items_per_cta = 16;         // work-list granularity
    int engine_choice[2][2] = {{-1, -1}, {-1, -1}};   // [acc][K dtype] engine tile shape
    // fast attraction: the node field of one density (field.cu)
    int attr_mode = SPARKLING_ATTRACTION_DIRECT;
    float4 *field = nullptr;
    size_t field_cap = 0;
    bool field_valid = false;
    const void *field_rho = nullptr;
    int field_n[3] = {0, 0, 0};
    double field_lo = 0.0, field_hi = 0.0, field_eps = 0.0;
    // kernel H(r) = sqrt(r^2 + eps^2); eps = 0 is the plain norm
    double eps = 0.0;
    // fast repulsion (mesh.cu)
    int rep_mode = SPARKLING_REPULSION_DIRECT;
    sparkling_mesh mesh_params = {};
    MeshState *mesh = nullptr;
};

namespace {

thread_local std::string g_err = "no error";

// Accumulation of the directed repulsion for a requested mode: the plain
// FP64-accumulate form applies to the attraction; the repulsion then folds
// its FP32 block sums in FP64.
int rep_acc(int acc) { return acc > SPARKLING_ACC_FP64 ? SPARKLING_ACC_FP64 : acc; }

// eps^2 as the pair kernels add it to r^2 (never below the zero-distance guard)
float eps2_of(const sparkling_ctx *ctx)
{
    const float e2 = (float)(ctx->eps * ctx->eps);
    return e2 > kEps2 ? e2 : kEps2;
}

int fail(sparkling_ctx *ctx, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    else g_err = buf;
    return code;
}

int cuda_fail(sparkling_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, SPARKLING_E_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);                                   \
    } while (0)

int lazy_init(sparkling_ctx *ctx)
{
    if (ctx->inited) {
        CK(cudaSetDevice(ctx->device));
        return SPARKLING_OK;
    }
    int n = 0;
    CK(cudaGetDeviceCount(&n));
    if (ctx->device >= n)
        return fail(ctx, SPARKLING_E_CUDA, "device %d not present (%d devices)", ctx->device, n);
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device));
    CK(cudaMalloc(&ctx->d_status, sizeof(DevCtl)));
    DevCtl ctl{};
    ctl.wait_cycles = ctx->wait_cycles;
    CK(cudaMemcpy(ctx->d_status, &ctl, sizeof(DevCtl), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_small, 8 * sizeof(double)));
    CK(cudaMemset(ctx->d_small, 0, 8 * sizeof(double)));
    ctx->inited = true;
    return SPARKLING_OK;
}

// Device memory of the current device (the context's: lazy_init makes it
// current), or managed memory.
bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Sub-allocation of one contiguous workspace.
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    }
};

// Device bytes the context holds besides the buffer being replaced.
size_t held_bytes(const sparkling_ctx *ctx) { return ctx->ws_bytes + ctx->h_K_bytes + ctx->h_rho_bytes + ctx->field_cap; }

// The context's allocation cap (sparkling_set_memory_limit): a request that
// would take the context's device memory past it fails before any launch.
int check_limit(sparkling_ctx *ctx, size_t other, size_t bytes, const char *what)
{
    if (ctx->mem_limit && other + bytes > ctx->mem_limit)
        return fail(ctx, SPARKLING_E_NOMEM,
                    "%s of %zu bytes would take the context to %zu bytes, over its limit of %zu",
                    what, bytes, other + bytes, ctx->mem_limit);
    return SPARKLING_OK;
}

// Every call carves the workspace from its start, so a call overwrites what
// the batched step keeps there across calls (its uploaded work list and
// descriptors): the batch is planned and uploaded again at its next call.
int ensure_ws(sparkling_ctx *ctx, size_t bytes)
{
    ctx->batch.valid = false;
    if (bytes <= ctx->ws_bytes) return SPARKLING_OK;
    const size_t other = held_bytes(ctx) - ctx->ws_bytes;
    int s;
    if ((s = check_limit(ctx, other, bytes, "workspace"))) return s;
    // Growth is rare (first call of a larger problem): synchronise so that no
    // queued kernel still uses the old buffer, then reallocate with headroom.
    CK(cudaDeviceSynchronize());
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    size_t want = align_up(bytes + bytes / 8, 1 << 20);
    if (ctx->mem_limit && other + want > ctx->mem_limit) want = bytes;
    cudaError_t e = cudaMalloc(&ctx->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, SPARKLING_E_NOMEM, "workspace allocation of %zu bytes failed: %s", want,
                    cudaGetErrorString(e));
    }
    ctx->ws_bytes = want;
    return SPARKLING_OK;
}

cudaEvent_t get_event(sparkling_ctx *ctx)
{
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bookkeeping around one launch: count it and, when timing is on, bracket it
// with events on the launch stream.
struct LaunchScope {
    sparkling_ctx *ctx;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    LaunchScope(sparkling_ctx *c, int k, cudaStream_t s) : ctx(c), kind(k), st(s)
    {
        if (ctx->timing) {
            a = get_event(ctx);
            b = get_event(ctx);
            if (a) cudaEventRecord(a, st);
        }
    }
    // nkernels: kernels launched inside the scope (all counted in
    // sparkling_launch_count); the timing table counts the scope once.
    void done(int nkernels = 1)
    {
        ctx->launches += nkernels;
        ctx->nlaunch[kind] += 1;
        if (a && b) {
            cudaEventRecord(b, st);
            ctx->pending.push_back({kind, a, b});
        }
    }
};

// The device work of one whole step (sparkling_step), timed as one scope of
// kind SPARKLING_KERNEL_STEP when timing is on.  Launches inside it are
// counted by their own scopes.
struct StepScope {
    sparkling_ctx *ctx;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    StepScope(sparkling_ctx *c, cudaStream_t s) : ctx(c), st(s)
    {
        if (ctx->timing) {
            a = get_event(ctx);
            b = get_event(ctx);
            if (a) cudaEventRecord(a, st);
        }
    }
    void done()
    {
        ctx->nlaunch[SPARKLING_KERNEL_STEP] += 1;
        if (a && b) {
            cudaEventRecord(b, st);
            ctx->pending.push_back({SPARKLING_KERNEL_STEP, a, b});
            a = b = nullptr;
        }
    }
    ~StepScope()
    {   // an early return: the events go back to the pool unrecorded
        if (a) ctx->pool.push_back(a);
        if (b) ctx->pool.push_back(b);
    }
};

int validate_grid(sparkling_ctx *ctx, const sparkling_grid *g, bool need_ptr)
{
    if (!g) return fail(ctx, SPARKLING_E_INVAL, "grid is NULL");
    for (int a = 0; a < 3; ++a)
        if (g->n[a] < 1)
            return fail(ctx, SPARKLING_E_INVAL, "grid n[%d] = %d must be >= 1", a, g->n[a]);
    if (g->n[0] > kMaxNx)
        return fail(ctx, SPARKLING_E_INVAL, "grid nx = %d exceeds %d", g->n[0], kMaxNx);
    if ((int64_t)g->n[1] * g->n[2] > (int64_t)1 << 30)
        return fail(ctx, SPARKLING_E_INVAL, "grid ny*nz too large");
    if (!(std::isfinite(g->lo) && std::isfinite(g->hi) && g->hi > g->lo))
        return fail(ctx, SPARKLING_E_INVAL, "grid needs finite lo < hi (got %g, %g)", g->lo, g->hi);
    if (need_ptr && !g->rho) return fail(ctx, SPARKLING_E_INVAL, "grid->rho is NULL");
    return SPARKLING_OK;
}

int validate_dtype(sparkling_ctx *ctx, int dt, const char *what)
{
    if (dt != SPARKLING_F32 && dt != SPARKLING_F64)
        return fail(ctx, SPARKLING_E_INVAL, "%s dtype %d is not SPARKLING_F32/F64", what, dt);
    return SPARKLING_OK;
}

int validate_proj(sparkling_ctx *ctx, const sparkling_proj *p, int64_t Ns)
{
    if (!p) return fail(ctx, SPARKLING_E_INVAL, "proj is NULL");
    if (!(p->alpha > 0) || !(p->beta > 0) || std::isnan(p->alpha) || std::isnan(p->beta))
        return fail(ctx, SPARKLING_E_INVAL, "alpha, beta must be > 0 (inf allowed)");
    if (!(p->box > 0) || std::isnan(p->box))
        return fail(ctx, SPARKLING_E_INVAL, "box must be > 0");
    if (p->n_iter < 0) return fail(ctx, SPARKLING_E_INVAL, "n_iter must be >= 0");
    if (p->pin_index >= Ns)
        return fail(ctx, SPARKLING_E_INVAL, "pin_index %d >= Ns %lld", p->pin_index, (long long)Ns);
    if (p->pin_index >= 0)
        for (int c = 0; c < 3; ++c)
            if (!std::isfinite(p->pin[c])) return fail(ctx, SPARKLING_E_INVAL, "pin must be finite");
    if (std::isnan(p->tol)) return fail(ctx, SPARKLING_E_INVAL, "tol is NaN");
    if (p->tol > 0) {
        if (!(p->margin >= 0 && p->margin < 1))
            return fail(ctx, SPARKLING_E_INVAL, "margin must be in [0, 1)");
        if (p->check_every < 1)
            return fail(ctx, SPARKLING_E_INVAL, "check_every must be >= 1 in converged mode");
    }
    return SPARKLING_OK;
}

// Plan of one gradient/energy evaluation.
struct PairPlan {
    int64_t N;
    int nx, ny, nz, gxp;
    int64_t tiles;
    int va, vr;            // tile shapes (autotuner variants) of the two pair kernels
    Split spa, spr;
    size_t o_pos, o_rho, o_coords, o_parta, o_partr, o_racc, o_eblocks, o_g64, o_adir, o_rdir, end;
};

int ensure_occupancy(sparkling_ctx *ctx)
{
    if (ctx->occ_done) return SPARKLING_OK;
    for (int acc = 0; acc < 3; ++acc)
        for (int e = 0; e < 2; ++e) {
            for (int v = 0; v < kAttrVariants; ++v)
                ctx->occ_attr[acc][e][v] = attraction_ctas_per_sm(acc, e != 0, v);
            if (acc < 2)
                for (int v = 0; v < kRepVariants; ++v)
                    ctx->occ_rep[acc][e][v] = repulsion_ctas_per_sm(acc, e != 0, v);
        }
    for (int e = 0; e < 2; ++e)
        for (int v = 0; v < kSymVariants; ++v)
            ctx->occ_sym[e][v] = repulsion_sym_ctas_per_sm(e != 0, v);
    cudaGetLastError();
    for (int e = 0; e < 2; ++e)
        for (int v = 0; v < kSymVariants; ++v)
            if (ctx->occ_sym[e][v] < 1) ctx->rep_symmetric = false;
    for (int acc = 0; acc < 3; ++acc)
        for (int e = 0; e < 2; ++e)
            if (ctx->occ_attr[acc][e][kAttrDefault] < 1 || ctx->occ_rep[rep_acc(acc)][e][kRepDefault] < 1)
                return fail(ctx, SPARKLING_E_CUDA, "pair kernels cannot be resident (occupancy 0)");
    ctx->occ_done = true;
    return SPARKLING_OK;
}

int attr_choice_of(const sparkling_ctx *ctx, int acc, int gxp)
{
    if (ctx->pin_attr >= 0) return ctx->pin_attr;
    const int64_t key = (int64_t)acc * (1 << 20) + gxp;
    for (const auto &kv : ctx->attr_choice)
        if (kv.first == key) return kv.second;
    return -1;
}

// Splits of the two pair kernels for the chosen tile shapes.
void set_splits(sparkling_ctx *ctx, PairPlan &P, int acc, bool energy, int va, int vr)
{
    const int e = energy ? 1 : 0;
    const int64_t rows = (int64_t)P.ny * P.nz;
    const int64_t nblocks = (P.N + kSrcBlock - 1) / kSrcBlock;
    if (ctx->occ_attr[acc][e][va] < 1) va = kAttrDefault;   // a pinned shape that cannot be resident
    P.va = va;
    P.vr = vr;
    P.spa = make_split(P.tiles, rows, (int64_t)ctx->sms * ctx->occ_attr[acc][e][va]);
    P.spr = make_split(P.tiles, nblocks, (int64_t)ctx->sms * ctx->occ_rep[rep_acc(acc)][e][vr]);
}

int plan_pairs(sparkling_ctx *ctx, int64_t N, const sparkling_grid *g, int acc, bool energy,
               bool need_g64, PairPlan &P, Carve &cv)
{
    int s;
    if ((s = ensure_occupancy(ctx))) return s;
    P.N = N;
    P.nx = g->n[0]; P.ny = g->n[1]; P.nz = g->n[2];
    P.gxp = (P.nx + 3) / 4 * 4;
    P.tiles = (N + kTile - 1) / kTile;
    const int va = attr_choice_of(ctx, acc, P.gxp), vr = ctx->rep_choice[rep_acc(acc)];
    set_splits(ctx, P, acc, energy, va < 0 ? kAttrDefault : va, vr < 0 ? kRepDefault : vr);
    // Partial buffers big enough for every tile shape and for the tuning
    // trials (which run on a prefix of the tiles with one wave of CTAs).
    int64_t max_ctas = 0;
    for (int e = 0; e < 2; ++e) {
        for (int v = 0; v < kAttrVariants; ++v)
            max_ctas = std::max<int64_t>(max_ctas, (int64_t)ctx->sms * ctx->occ_attr[acc][e][v]);
        for (int v = 0; v < kRepVariants; ++v)
            max_ctas = std::max<int64_t>(max_ctas, (int64_t)ctx->sms * ctx->occ_rep[rep_acc(acc)][e][v]);
    }
    const int64_t part_units = std::max<int64_t>(P.tiles * ((max_ctas + P.tiles - 1) / P.tiles + 1),
                                                 max_ctas + 2 * P.tiles);
    const int64_t rows = (int64_t)P.ny * P.nz;
    P.o_pos = cv.take((size_t)N * sizeof(float4));
    P.o_rho = cv.take((size_t)rows * P.gxp * sizeof(float));
    P.o_coords = cv.take(((size_t)P.gxp + P.ny + P.nz) * sizeof(float));
    P.o_parta = cv.take((size_t)part_units * kTile * sizeof(dacc4));
    P.o_partr = cv.take((size_t)part_units * kTile * sizeof(dacc4));
    P.o_racc = cv.take((size_t)N * 3 * sizeof(unsigned long long));
    P.o_eblocks = cv.take((size_t)energy_blocks(N) * sizeof(double2));
    P.o_g64 = need_g64 ? cv.take((size_t)N * 3 * sizeof(double)) : 0;
    P.o_adir = ctx->attr_mode == SPARKLING_ATTRACTION_FIELD ? cv.take((size_t)N * sizeof(dacc4)) : 0;
    P.o_rdir = ctx->rep_mode == SPARKLING_REPULSION_MESH ? cv.take((size_t)N * sizeof(dacc4)) : 0;
    P.end = cv.off;
    return SPARKLING_OK;
}

template <typename T> T *at(sparkling_ctx *ctx, size_t off)
{
    return reinterpret_cast<T *>(static_cast<char *>(ctx->ws) + off);
}

// Autotuner: time every tile shape of a pair kernel on a prefix of the
// caller's own (already packed) problem -- about 1e11 pairs, one wave of
// CTAs, one warm-up and one timed launch each -- and keep the fastest.  The
// trials write into the partial buffers, which the real launch overwrites.
// Runs once per key (acc and padded row length for the attraction, acc for
// the repulsion) and synchronises the stream.
int tune_pairs(sparkling_ctx *ctx, PairPlan &P, int acc, AttrArgs aa, RepArgs ra, bool do_attr,
               bool do_rep, bool do_sym, unsigned long long *racc, cudaStream_t st)
{
    cudaEvent_t e0 = get_event(ctx), e1 = get_event(ctx);
    const int64_t rows = (int64_t)P.ny * P.nz;
    const int64_t nblocks = (P.N + kSrcBlock - 1) / kSrcBlock;
    const double budget = 1e11;
    char line[160];
    auto timed = [&](auto launch) -> double {
        cudaError_t err = launch();
        if (err != cudaSuccess) return -1.0;
        cudaEventRecord(e0, st);
        err = launch();
        cudaEventRecord(e1, st);
        if (err != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    if (do_attr) {
        const int64_t P3 = rows * P.nx;
        int64_t tt = (int64_t)(budget / ((double)kTile * (double)P3) + 0.5);
        tt = std::max<int64_t>(1, std::min<int64_t>(tt, P.tiles));
        int best = kAttrDefault;
        double best_rate = 0.0;
        for (int v = 0; v < kAttrVariants; ++v) {
            const int occ = ctx->occ_attr[acc][0][v];
            if (occ < 1) continue;
            aa.sp = make_split(tt, rows, (int64_t)ctx->sms * occ);
            const double ms = timed([&] { return launch_attraction(aa, acc, false, v, st); });
            const double pairs = (double)std::min<int64_t>(tt * kTile, P.N) * (double)P3;
            const double rate = ms > 0 ? pairs / (ms * 1e-3) : 0.0;
            snprintf(line, sizeof line, "attraction gxp=%d threads=%d: %.4g pairs/s\n", P.gxp,
                     attr_variant_threads(v), rate);
            ctx->tune_log += line;
            if (rate > best_rate) { best_rate = rate; best = v; }
        }
        ctx->attr_choice.push_back({(int64_t)acc * (1 << 20) + P.gxp, best});
    }
    if (do_rep) {
        int64_t tt = (int64_t)(budget / ((double)kTile * (double)P.N) + 0.5);
        tt = std::max<int64_t>(1, std::min<int64_t>(tt, P.tiles));
        int best = kRepDefault;
        double best_rate = 0.0;
        for (int v = 0; v < kRepVariants; ++v) {
            const int occ = ctx->occ_rep[rep_acc(acc)][0][v];
            if (occ < 1) continue;
            ra.sp = make_split(tt, nblocks, (int64_t)ctx->sms * occ);
            const double ms = timed([&] { return launch_repulsion(ra, rep_acc(acc), false, v, st); });
            const double pairs = (double)std::min<int64_t>(tt * kTile, P.N) * (double)P.N;
            const double rate = ms > 0 ? pairs / (ms * 1e-3) : 0.0;
            snprintf(line, sizeof line, "repulsion threads=%d unroll=%d: %.4g pairs/s\n",
                     rep_variant_threads(v), rep_variant_unroll(v), rate);
            ctx->tune_log += line;
            if (rate > best_rate) { best_rate = rate; best = v; }
        }
        ctx->rep_choice[rep_acc(acc)] = best;
    }
    if (do_sym) {
        // a sub-triangle of about 1e11 directed pairs (the first tt tiles)
        int64_t tt = (int64_t)(std::sqrt(budget) / kTile + 0.5);
        tt = std::max<int64_t>(1, std::min<int64_t>(tt, P.tiles));
        SymArgs sa{};
        sa.pos = ra.pos; sa.N = std::min<int64_t>(P.N, tt * kTile); sa.tiles = tt;
        sa.acc = racc; sa.status = ctx->d_status; sa.eps2 = ra.eps2;
        int best = kSymDefault;
        double best_rate = 0.0;
        for (int v = 0; v < kSymVariants; ++v) {
            sa.ctas = (int64_t)ctx->sms * ctx->occ_sym[0][v];
            const double ms = timed([&] { return launch_repulsion_sym(sa, false, v, st); });
            const double pairs = (double)sa.N * (double)(sa.N - 1);
            const double rate = ms > 0 ? pairs / (ms * 1e-3) : 0.0;
            snprintf(line, sizeof line,
                     "repulsion symmetric threads=%d sources/lane=%d %s-paired: %.4g pairs/s\n",
                     sym_variant_threads(v), sym_variant_sources(v),
                     sym_variant_source_paired(v) ? "source" : "target", rate);
            ctx->tune_log += line;
            if (rate > best_rate) { best_rate = rate; best = v; }
        }
        ctx->sym_choice = best;
    }
    ctx->pool.push_back(e0);
    ctx->pool.push_back(e1);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(ctx, err, "autotuner trial");
    return SPARKLING_OK;
}

bool field_matches(const sparkling_ctx *ctx, const sparkling_grid *g)
{
    return ctx->field_valid && ctx->field_rho == g->rho && ctx->field_n[0] == g->n[0] &&
           ctx->field_n[1] == g->n[1] && ctx->field_n[2] == g->n[2] && ctx->field_lo == g->lo &&
           ctx->field_hi == g->hi && ctx->field_eps == ctx->eps;
}

// (Re)build the node field of g's density into the context (blocking).
int build_field(sparkling_ctx *ctx, const sparkling_grid *g, cudaStream_t st)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(ctx, SPARKLING_E_INVAL,
                    "the attraction field must be built outside stream capture "
                    "(call sparkling_attraction_field first)");
    const size_t bytes = field_bytes(g->n[0], g->n[1], g->n[2]);
    ctx->field_valid = false;
    if (bytes > ctx->field_cap) {
        int s;
        if ((s = check_limit(ctx, held_bytes(ctx) - ctx->field_cap, bytes, "attraction field")))
            return s;
        CK(cudaStreamSynchronize(st));
        cudaFree(ctx->field);
        ctx->field = nullptr;
        ctx->field_cap = 0;
        cudaError_t e = cudaMalloc(&ctx->field, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, SPARKLING_E_NOMEM, "field allocation of %zu bytes failed", bytes);
        }
        ctx->field_cap = bytes;
    }
    const char *what = "";
    cudaError_t e = field_build(g->rho, g->n[0], g->n[1], g->n[2], g->lo, g->hi, ctx->eps,
                                ctx->field, ctx->sms, st, &what);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ctx, SPARKLING_E_NOMEM, "attraction field: %s allocation failed", what);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    ctx->launches += 13;
    ctx->field_valid = true;
    ctx->field_rho = g->rho;
    for (int a = 0; a < 3; ++a) ctx->field_n[a] = g->n[a];
    ctx->field_lo = g->lo;
    ctx->field_hi = g->hi;
    ctx->field_eps = ctx->eps;
    return SPARKLING_OK;
}

MeshConfig mesh_config(const sparkling_ctx *ctx)
{
    const sparkling_mesh &m = ctx->mesh_params;
    MeshConfig c;
    c.n_cells = m.n_cells;
    c.lo = m.lo;
    c.hi = m.hi;
    c.sigma = m.sigma_cells * (m.hi - m.lo) / m.n_cells;
    c.rc = m.rc_sigmas * c.sigma;
    c.eps = ctx->eps;
    return c;
}

// Kernel spectra of the context's mesh (built when the mesh or eps changed).
int ensure_mesh(sparkling_ctx *ctx, cudaStream_t st)
{
    const MeshConfig c = mesh_config(ctx);
    if (!ctx->mesh) ctx->mesh = mesh_state_create();
    if (mesh_matches(ctx->mesh, c)) return SPARKLING_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(ctx, SPARKLING_E_INVAL, "the fast-repulsion mesh must be built outside stream capture");
    const char *what = "";
    cudaError_t e = mesh_build(ctx->mesh, c, ctx->sms, st, &what);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ctx, SPARKLING_E_NOMEM, "fast repulsion: %s allocation failed", what);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    ctx->launches += 12;
    return SPARKLING_OK;
}

// pack -> (autotune) -> attraction -> repulsion -> combine (gradient) or
// energy reduction.  In field mode the attraction is the interpolated node
// field.
int run_pairs(sparkling_ctx *ctx, const void *K, int K_dtype, const sparkling_grid *g, int acc,
              bool energy, PairPlan &P, void *G, int G_dtype, void *A, void *R, bool g64,
              cudaStream_t st, double scale = 1.0, const double *scale_dev = nullptr)
{
    float4 *pos = at<float4>(ctx, P.o_pos);
    float *rho = at<float>(ctx, P.o_rho);
    float *coords = at<float>(ctx, P.o_coords);
    const bool field_mode = ctx->attr_mode == SPARKLING_ATTRACTION_FIELD;
    if (field_mode && !field_matches(ctx, g)) {
        int s = build_field(ctx, g, st);
        if (s) return s;
    }
    {
        LaunchScope ls(ctx, SPARKLING_KERNEL_PACK, st);
        CK(launch_pack_positions(K, K_dtype, P.N, pos, ctx->d_status, ctx->sms, st));
        CK(launch_pack_grid(g->rho, P.nx, P.ny, P.nz, P.gxp, g->lo, g->hi, rho, coords,
                            ctx->d_status, ctx->sms, st));
        ls.done(2);
    }
    AttrArgs aa{};
    aa.tgt = pos; aa.N = P.N; aa.rho = rho; aa.coords = coords;
    aa.gxp = P.gxp; aa.ny = P.ny; aa.nz = P.nz;
    aa.rows_per_stage = kStageFloats / P.gxp;
    aa.hx = (float)((g->hi - g->lo) / P.nx);
    aa.x0 = g->lo + 0.5 * ((g->hi - g->lo) / P.nx);
    aa.part = at<dacc4>(ctx, P.o_parta); aa.status = ctx->d_status;
    aa.eps2 = eps2_of(ctx);
    RepArgs ra{};
    ra.pos = pos; ra.N = P.N; ra.part = at<dacc4>(ctx, P.o_partr);
    ra.status = ctx->d_status;
    ra.eps2 = aa.eps2;
    const bool mesh_mode = ctx->rep_mode == SPARKLING_REPULSION_MESH;
    const bool need_a = !field_mode && attr_choice_of(ctx, acc, P.gxp) < 0,
               need_r = !mesh_mode && !ctx->rep_symmetric && ctx->rep_choice[rep_acc(acc)] < 0,
               need_s = !mesh_mode && ctx->rep_symmetric && ctx->sym_choice < 0;
    if (ctx->autotune && (need_a || need_r || need_s)) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(st, &cap));
        if (cap == cudaStreamCaptureStatusNone) {
            int s = tune_pairs(ctx, P, acc, aa, ra, need_a, need_r, need_s,
                               at<unsigned long long>(ctx, P.o_racc), st);
            if (s) return s;
            const int va = attr_choice_of(ctx, acc, P.gxp), vr = ctx->rep_choice[rep_acc(acc)];
            set_splits(ctx, P, acc, energy, va < 0 ? kAttrDefault : va, vr < 0 ? kRepDefault : vr);
        }
    }
    aa.sp = P.spa;
    ra.sp = P.spr;
    dacc4 *a_direct = field_mode ? at<dacc4>(ctx, P.o_adir) : nullptr;
    {
        LaunchScope ls(ctx, SPARKLING_KERNEL_ATTRACTION, st);
        if (field_mode)
            CK(launch_interp(pos, P.N, ctx->field, P.nx, P.ny, P.nz, g->lo, g->hi, a_direct,
                             ctx->sms, st));
        else
            CK(launch_attraction(aa, acc, energy, P.va, st));
        ls.done();
    }
    unsigned long long *racc = nullptr;
    dacc4 *r_direct = nullptr;
    if (mesh_mode) {
        int s;
        if ((s = ensure_mesh(ctx, st))) return s;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(st, &cap));
        r_direct = at<dacc4>(ctx, P.o_rdir);
        const char *what = "";
        int nk = 0;
        LaunchScope ls(ctx, SPARKLING_KERNEL_REPULSION, st);
        cudaError_t e = mesh_eval(ctx->mesh, pos, P.N, energy, r_direct, ctx->d_status, ctx->sms, st,
                                  &what, &nk, cap != cudaStreamCaptureStatusNone);
        if (e == cudaErrorStreamCaptureUnsupported)
            return fail(ctx, SPARKLING_E_INVAL,
                        "the fast repulsion's buffers for N = %lld are allocated by a first call "
                        "of that size outside stream capture", (long long)P.N);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return fail(ctx, SPARKLING_E_NOMEM, "fast repulsion: %s allocation failed", what);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, what);
        ls.done(nk);
    } else if (ctx->rep_symmetric) {
        // every unordered pair once, exact fixed-point totals
        racc = at<unsigned long long>(ctx, P.o_racc);
        SymArgs sa{};
        sa.pos = pos; sa.N = P.N; sa.tiles = P.tiles;
        const int sv = ctx->sym_choice < 0 ? kSymDefault : ctx->sym_choice;
        sa.ctas = (int64_t)ctx->sms * ctx->occ_sym[energy ? 1 : 0][sv];
        sa.acc = racc; sa.status = ctx->d_status; sa.eps2 = ra.eps2;
        LaunchScope ls(ctx, SPARKLING_KERNEL_REPULSION, st);
        CK(cudaMemsetAsync(racc, 0, (size_t)P.N * (energy ? 1 : 3) * sizeof(unsigned long long), st));
        CK(launch_repulsion_sym(sa, energy, sv, st));
        ls.done();
    } else {
        LaunchScope ls(ctx, SPARKLING_KERNEL_REPULSION, st);
        CK(launch_repulsion(ra, rep_acc(acc), energy, P.vr, st));
        ls.done();
    }
    CombineArgs cb{};
    cb.N = P.N; cb.part_a = aa.part; cb.part_r = ra.part; cb.spa = P.spa; cb.spr = P.spr;
    cb.G = G; cb.A = A; cb.R = R;
    cb.G64 = g64 ? at<double>(ctx, P.o_g64) : nullptr;
    cb.racc = racc;
    cb.a_direct = a_direct;
    cb.r_direct = r_direct;
    cb.scale = scale;
    cb.scale_dev = scale_dev;
    cb.eps = ctx->eps;
    cb.energy_blocks = at<double2>(ctx, P.o_eblocks);
    {
        LaunchScope ls(ctx, SPARKLING_KERNEL_COMBINE, st);
        if (energy) {
            CK(launch_combine_energy(cb, ctx->d_small, st));
            ls.done(2);
        } else {
            CK(launch_combine(cb, G_dtype, ctx->sms, st));
            ls.done();
        }
    }
    return SPARKLING_OK;
}

int read_status(sparkling_ctx *ctx, cudaStream_t st)
{
    int h = 0;
    CK(cudaMemcpyAsync(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h) CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
    if (h & kDevTimeout)
        return fail(ctx, SPARKLING_E_TIMEOUT, "a bounded device wait ran out; results are incomplete");
    if (h & kDevNonFinite)
        return fail(ctx, SPARKLING_E_NONFINITE, "non-finite sample or density value, or negative density");
    if (h & kDevRange)
        return fail(ctx, SPARKLING_E_RANGE, "a sample lies outside the fast-repulsion mesh");
    return SPARKLING_OK;
}

int common_checks(sparkling_ctx *ctx, const void *K, int K_dtype, int64_t N, const sparkling_grid *g,
                  int acc)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    if (!K) return fail(ctx, SPARKLING_E_INVAL, "K is NULL");
    int s;
    if ((s = validate_dtype(ctx, K_dtype, "K"))) return s;
    if (N < 2) return fail(ctx, SPARKLING_E_INVAL, "N = %lld must be >= 2", (long long)N);
    if (N > ((int64_t)1 << 31) - kTile)
        return fail(ctx, SPARKLING_E_INVAL, "N = %lld is too large", (long long)N);
    if (acc != SPARKLING_ACC_KAHAN32 && acc != SPARKLING_ACC_FP64 && acc != SPARKLING_ACC_FP64_PAIR)
        return fail(ctx, SPARKLING_E_INVAL, "acc %d is not KAHAN32/FP64/FP64_PAIR", acc);
    if ((s = validate_grid(ctx, g, true))) return s;
    return SPARKLING_OK;
}

// Launch shape of the projection: one CTA per shot up to one wave; the
// per-CTA state goes to the workspace when it does not fit in shared memory.
struct ProjPlan {
    int grid = 0;
    bool global_state = false;
    size_t o_state = 0;
};

int plan_project(sparkling_ctx *ctx, int K_dtype, int64_t Nc, int64_t Ns, Carve &cv, ProjPlan &L)
{
    const int ns = (int)Ns;
    const int occ = project_ctas_per_sm(K_dtype, ns);
    if (occ < 1) {
        cudaGetLastError();
        return fail(ctx, SPARKLING_E_CUDA, "projection kernel cannot be resident for Ns = %d", ns);
    }
    int64_t grid = (int64_t)ctx->sms * occ;
    if (grid > Nc) grid = Nc;
    L.grid = (int)grid;
    L.global_state = !project_state_in_smem(ns);
    if (L.global_state) L.o_state = cv.take((size_t)grid * project_state_bytes(ns));
    return SPARKLING_OK;
}

// Projection of Nc shots (with an optional gradient step k = K - eta G64).
// The workspace must already hold the plan's state region.
int run_project(sparkling_ctx *ctx, void *K, int K_dtype, int64_t Nc, int64_t Ns,
                const sparkling_proj *pr, const double *G64, double eta, const ProjPlan &L,
                bool want_viol, cudaStream_t st)
{
    ProjArgs p{};
    p.K = K; p.G = G64; p.eta = eta; p.Nc = Nc; p.Ns = (int)Ns;
    p.alpha = pr->alpha; p.beta = pr->beta; p.box = pr->box; p.tol = pr->tol;
    p.margin = pr->margin;
    for (int c = 0; c < 3; ++c) p.pin[c] = pr->pin[c];
    p.pin_index = pr->pin_index < 0 ? -1 : pr->pin_index;
    p.n_iter = pr->n_iter;
    p.check_every = pr->check_every;
    p.status = ctx->d_status;
    p.viol = want_viol ? reinterpret_cast<unsigned long long *>(ctx->d_small + 2) : nullptr;
    p.notconv = pr->tol > 0 ? reinterpret_cast<int *>(ctx->d_small + 6) : nullptr;
    p.gstate = L.global_state ? at<double>(ctx, L.o_state) : nullptr;
    p.mixed = ctx->proj_mode == SPARKLING_PROJECTION_MIXED ? 1 : 0;
    if (want_viol || p.notconv)
        CK(cudaMemsetAsync(ctx->d_small + 2, 0, 5 * sizeof(double), st));
    LaunchScope ls(ctx, SPARKLING_KERNEL_PROJECT, st);
    CK(launch_project(p, K_dtype, L.grid, st));
    ls.done();
    return SPARKLING_OK;
}

int finish_project(sparkling_ctx *ctx, const sparkling_proj *pr, double *viol_host, cudaStream_t st)
{
    double h[5] = {0, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(h, ctx->d_small + 2, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
    int s = read_status(ctx, st);
    if (s) return s;
    if (viol_host)
        for (int e = 0; e < 4; ++e) viol_host[e] = h[e];
    int notconv = 0;
    std::memcpy(&notconv, &h[4], sizeof(int));
    if (pr->tol > 0 && notconv > 0)
        return fail(ctx, SPARKLING_E_NOTCONV, "%d shot(s) did not certify within %d iterations",
                    notconv, pr->n_iter);
    return SPARKLING_OK;
}

int check_shots(sparkling_ctx *ctx, int64_t Nc, int64_t Ns)
{
    if (Nc < 1) return fail(ctx, SPARKLING_E_INVAL, "Nc = %lld must be >= 1", (long long)Nc);
    if (Ns < 1 || Ns > 65536)
        return fail(ctx, SPARKLING_E_INVAL, "Ns = %lld must be in [1, 65536]", (long long)Ns);
    if (Nc > ((int64_t)1 << 40) / Ns) return fail(ctx, SPARKLING_E_INVAL, "Nc * Ns too large");
    return SPARKLING_OK;
}

} // namespace

// ---------------------------------------------------------------------------
// Batched step on the persistent engine.

namespace {

int64_t pair_cost(int64_t N, int64_t P) { return N * P + N * N; }

// Work list of one batched step: per trajectory and target tile, attraction
// items (runs of grid rows) and repulsion items -- runs of source blocks
// (directed), or, in the one-launch shape, runs of source tiles J >= the
// target tile (symmetric) -- each of about total / (ctas * items_per_cta)
// pairs, and one projection item per shot.  With `sym` the repulsion runs in
// a separate kernel and the list holds no repulsion items.  Attraction and
// repulsion items alternate so that neighbouring CTAs (and hence the CTAs
// resident on one SM) mix SFU-bound and FP32-bound work.
// The projection items of trajectory t are placed once at least 2 * ctas
// pair items have followed t's last pair item (the rest close the list): by
// the time a CTA takes one, t's pair items -- dispensed two waves of CTAs
// earlier -- are done, so it rarely waits, and the projections' FP64 work
// overlaps later trajectories' pair items.  Every pair item of t still comes
// before every projection item of t in the list, the order that makes every
// wait of a projection item end.
void build_work_list(sparkling_ctx::Batch &b, const std::vector<int64_t> &off,
                     const sparkling_grid *grids, int ctas, int items_per_cta, bool sym,
                     bool one_launch)
{
    const int B = (int)off.size() - 1;
    int64_t total = 0;
    for (int t = 0; t < B; ++t) {
        const int64_t P = (int64_t)grids[t].n[0] * grids[t].n[1] * grids[t].n[2];
        const int64_t N = off[t + 1] - off[t];
        total += sym ? N * P : pair_cost(N, P);
    }
    const double target = (double)total / ((double)ctas * items_per_cta);
    b.traj.assign(B, EngineTraj());
    b.items.clear();
    b.item_pairs.clear();
    b.n_pair_items = 0;
    b.n_lead_items = -1;
    auto project_items = [&](int t) {
        if (b.n_lead_items < 0) b.n_lead_items = (int64_t)b.items.size();
        for (int c = 0; c < b.traj[t].Nc; ++c) {
            EngineItem it;
            it.kind = kItemProject; it.traj = t; it.tile = c; it.slot = 0; it.u0 = 0; it.u1 = 0;
            b.items.push_back(it);
            b.item_pairs.push_back(0.0);
        }
    };
    std::vector<int64_t> ends;       // pair items placed up to the end of trajectory t
    int released = 0;                // trajectories whose projection items are placed
    int64_t part = 0;
    for (int t = 0; t < B; ++t) {
        EngineTraj &tr = b.traj[t];
        const int64_t N = off[t + 1] - off[t];
        const int nx = grids[t].n[0], ny = grids[t].n[1], nz = grids[t].n[2];
        const int gxp = (nx + 3) / 4 * 4;
        const int64_t rows = (int64_t)ny * nz;
        const int64_t blocks = (N + kSrcBlock - 1) / kSrcBlock;
        int64_t rc = (int64_t)(target / ((double)kTile * gxp) + 0.5);
        rc = rc < 1 ? 1 : (rc > rows ? rows : rc);
        int64_t sc = (int64_t)(target / ((double)kTile * kSrcBlock) + 0.5);
        sc = sc < 1 ? 1 : (sc > blocks ? blocks : sc);
        const int ach = (int)((rows + rc - 1) / rc);
        const int rch = sym || one_launch ? 0 : (int)((blocks + sc - 1) / sc);
        // symmetric items: runs of up to L source tiles (a tile pair is
        // about 2 * kTile^2 directed pairs)
        int64_t L = (int64_t)(target / (2.0 * kTile * kTile) + 0.5);
        L = L < 1 ? 1 : (L > 64 ? 64 : L);
        tr.off = off[t];
        tr.N = N;
        tr.Ns = b.Ns;
        tr.Nc = (int32_t)(N / b.Ns);
        tr.gxp = gxp; tr.ny = ny; tr.nz = nz;
        tr.rows_per_stage = kStageFloats / gxp;
        tr.tiles = (int32_t)((N + kTile - 1) / kTile);
        tr.a_chunks = ach;
        tr.slots = ach + rch;
        tr.part_off = part * kTile;
        part += (int64_t)tr.tiles * tr.slots;
        tr.n_pair_items = tr.tiles * tr.slots;
        auto count_of = [&](int64_t J) { return (double)std::min<int64_t>(kTile, N - J * kTile); };
        for (int64_t tile = 0; tile < tr.tiles; ++tile) {
            int ia = 0, ir = 0;
            const int64_t nsr = one_launch ? (tr.tiles - tile + L - 1) / L : 0;
            int64_t is = 0;
            while (ia < ach || ir < rch || is < nsr) {
                const double tgt = count_of(tile);
                if (ia < ach) {
                    EngineItem it;
                    it.kind = kItemAttraction; it.traj = t; it.tile = (int32_t)tile; it.slot = ia;
                    it.u0 = ia * rc;
                    it.u1 = (ia + 1) * rc < rows ? (ia + 1) * rc : rows;
                    b.items.push_back(it);
                    b.item_pairs.push_back(tgt * (double)(it.u1 - it.u0) * nx);
                    ++ia;
                }
                if (ir < rch) {
                    EngineItem it;
                    it.kind = kItemRepulsion; it.traj = t; it.tile = (int32_t)tile;
                    it.slot = ach + ir;
                    it.u0 = ir * sc;
                    it.u1 = (ir + 1) * sc < blocks ? (ir + 1) * sc : blocks;
                    b.items.push_back(it);
                    b.item_pairs.push_back(tgt * (double)(std::min<int64_t>(it.u1 * kSrcBlock, N) -
                                                          it.u0 * kSrcBlock));
                    ++ir;
                }
                if (is < nsr) {
                    EngineItem it;
                    it.kind = kItemSym; it.traj = t; it.tile = (int32_t)tile; it.slot = 0;
                    it.u0 = tile + is * L;
                    it.u1 = std::min<int64_t>(it.u0 + L, tr.tiles);
                    double pairs = 0.0;   // directed: the diagonal pair once, the others twice
                    for (int64_t J = it.u0; J < it.u1; ++J)
                        pairs += (J == tile ? 1.0 : 2.0) * tgt * count_of(J);
                    b.items.push_back(it);
                    b.item_pairs.push_back(pairs);
                    ++tr.n_pair_items;
                    ++is;
                }
            }
        }
        b.n_pair_items += tr.n_pair_items;
        ends.push_back(b.n_pair_items);
        while (released < t && b.n_pair_items - ends[released] >= 2 * (int64_t)ctas)
            project_items(released++);
    }
    while (released < B) project_items(released++);
    // A projection item may wait for a pair item that another CTA has only
    // just started: allow twice the longest item's time at a conservative 4
    // pairs per CTA per clock (measured: ~4.8 for attraction, ~5.3 directed
    // repulsion pairs), and never less than four wait budgets.
    double most = 0.0;
    for (double v : b.item_pairs) most = std::max(most, v);
    const double scale = std::ceil(2.0 * most / 4.0 / (double)kWaitCycles);
    b.wait_scale = (int32_t)std::min(1024.0, std::max(4.0, scale));
}

// Role dispatch: the list reordered into its attraction items, its
// symmetric items and its projection items, each part in list order.
void split_work_list(sparkling_ctx::Batch &b)
{
    std::vector<EngineItem> items;
    std::vector<double> pairs;
    items.reserve(b.items.size());
    pairs.reserve(b.items.size());
    int32_t part[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
        const int kind = k == 0 ? kItemAttraction : k == 1 ? kItemSym : kItemProject;
        for (size_t i = 0; i < b.items.size(); ++i)
            if (b.items[i].kind == kind) {
                items.push_back(b.items[i]);
                pairs.push_back(b.item_pairs[i]);
                ++part[k];
            }
    }
    b.items.swap(items);
    b.item_pairs.swap(pairs);
    b.n_attr = part[0];
    b.n_sym = part[1];
    b.n_lead_items = part[0] + part[1];
}

int validate_batch(sparkling_ctx *ctx, int32_t B, const int64_t *off, const void *K, int K_dtype,
                   int32_t Ns, const sparkling_grid *grids, const double *eta,
                   const sparkling_proj *proj, int acc)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    int s;
    if (B < 1) return fail(ctx, SPARKLING_E_INVAL, "B = %d must be >= 1", B);
    if (!off || !K || !grids || !eta || !proj)
        return fail(ctx, SPARKLING_E_INVAL, "traj_off, K, grids, eta and proj are required");
    if ((s = validate_dtype(ctx, K_dtype, "K"))) return s;
    if (acc != SPARKLING_ACC_KAHAN32 && acc != SPARKLING_ACC_FP64)
        return fail(ctx, SPARKLING_E_INVAL, "acc %d is not KAHAN32/FP64", acc);
    if (Ns < 1 || Ns > 65536) return fail(ctx, SPARKLING_E_INVAL, "Ns = %d out of range", Ns);
    if (off[0] != 0) return fail(ctx, SPARKLING_E_INVAL, "traj_off[0] must be 0");
    for (int t = 0; t < B; ++t) {
        const int64_t N = off[t + 1] - off[t];
        if (N < 2 || N % Ns != 0 || N > ((int64_t)1 << 31) - kTile)
            return fail(ctx, SPARKLING_E_INVAL,
                        "trajectory %d has %lld samples: need >= 2, a multiple of Ns = %d", t,
                        (long long)N, Ns);
        if ((s = validate_grid(ctx, &grids[t], true))) return s;
        if ((s = validate_proj(ctx, &proj[t], Ns))) return s;
        if (proj[t].tol > 0)
            return fail(ctx, SPARKLING_E_INVAL, "converged mode is not available in the batched step");
        if (!std::isfinite(eta[t])) return fail(ctx, SPARKLING_E_INVAL, "eta[%d] not finite", t);
    }
    return SPARKLING_OK;
}

// Pack the samples of all trajectories and every density grid.
int batch_pack(sparkling_ctx *ctx, const void *K, int K_dtype, const sparkling_grid *grids,
               cudaStream_t st)
{
    sparkling_ctx::Batch &b = ctx->batch;
    const int B = b.B;
    CK(launch_pack_positions(K, K_dtype, b.off[B], at<float4>(ctx, b.o_pos), ctx->d_status,
                             ctx->sms, st));
    for (int t = 0; t < B; ++t)
        CK(launch_pack_grid(grids[t].rho, grids[t].n[0], grids[t].n[1], grids[t].n[2],
                            b.traj[t].gxp, grids[t].lo, grids[t].hi, at<float>(ctx, b.o_rho[t]),
                            at<float>(ctx, b.o_coords[t]), ctx->d_status, ctx->sms, st));
    return SPARKLING_OK;
}

// Reset the counters and run the first n_items items of the work list with
// engine tile shape `variant`.
int batch_engine(sparkling_ctx *ctx, void *K, int K_dtype, int acc, int variant, int64_t n_items,
                 cudaStream_t st)
{
    sparkling_ctx::Batch &b = ctx->batch;
    CK(cudaMemsetAsync(at<unsigned int>(ctx, b.o_cnt), 0,
                       (size_t)(3 + b.B + kSmSlots) * sizeof(unsigned int), st));
    EngineArgs e{};
    e.traj = at<EngineTraj>(ctx, b.o_traj);
    e.items = at<EngineItem>(ctx, b.o_items);
    e.n_items = (int32_t)n_items;
    e.proj_in_smem = b.proj_in_smem ? 1 : 0;
    e.proj_mixed = ctx->proj_mode == SPARKLING_PROJECTION_MIXED ? 1 : 0;
    e.pos = at<float4>(ctx, b.o_pos);
    e.K = K;
    e.part = at<dacc4>(ctx, b.o_part);
    e.queue = at<unsigned int>(ctx, b.o_cnt);
    e.done = e.queue + 3;
    e.sm_slots = e.done + b.B;
    e.roles = b.roles ? 1 : 0;
    e.wait_scale = b.wait_scale;
    e.n_attr = b.n_attr;
    e.n_sym = b.n_sym;
    e.gstate = b.proj_in_smem ? nullptr : at<double>(ctx, b.o_gstate);
    e.status = ctx->d_status;
    e.eps2 = eps2_of(ctx);
    e.racc = b.sym || b.one_launch ? at<unsigned long long>(ctx, b.o_racc) : nullptr;
    const int ctas = ctx->sms * engine_ctas_per_sm(acc, K_dtype, variant);
    CK(launch_engine(e, acc, K_dtype, variant, std::min(ctas, b.ctas), st));
    return SPARKLING_OK;
}

// Device work of one batched step on `st`: pack, then the whole work list.
int batch_device_work(sparkling_ctx *ctx, void *K, int K_dtype, const sparkling_grid *grids,
                      int acc, int variant, cudaStream_t st)
{
    int s;
    if ((s = batch_pack(ctx, K, K_dtype, grids, st))) return s;
    sparkling_ctx::Batch &b = ctx->batch;
    if (b.sym) {
        // every unordered pair of every trajectory once, fixed-point totals
        unsigned long long *racc = at<unsigned long long>(ctx, b.o_racc);
        CK(cudaMemsetAsync(racc, 0, (size_t)b.off[b.B] * 3 * sizeof(unsigned long long), st));
        SymArgs sa{};
        sa.pos = at<float4>(ctx, b.o_pos);
        sa.N = b.off[b.B];
        sa.tiles = 0;
        sa.acc = racc;
        sa.status = ctx->d_status;
        sa.eps2 = eps2_of(ctx);
        sa.traj = at<SymTraj>(ctx, b.o_symtraj);
        sa.B = b.B;
        sa.units = b.sym_units;
        const int sv = ctx->sym_choice < 0 ? kSymDefault : ctx->sym_choice;
        sa.ctas = std::min<int64_t>((int64_t)ctx->sms * ctx->occ_sym[0][sv], b.sym_units);
        CK(launch_repulsion_sym(sa, false, sv, st));
    } else if (b.one_launch) {
        // the engine's symmetric items add into these totals
        CK(cudaMemsetAsync(at<unsigned long long>(ctx, b.o_racc), 0,
                           (size_t)b.off[b.B] * 3 * sizeof(unsigned long long), st));
    }
    return batch_engine(ctx, K, K_dtype, acc, variant, (int64_t)b.items.size(), st);
}

// Engine autotuner: time each tile shape on a prefix of the pair items (about
// 1.5e11 pairs; pair items only write partial slots, which the real step
// overwrites, so K is untouched) after one warm-up, and keep the fastest.
int tune_engine(sparkling_ctx *ctx, void *K, int K_dtype, const sparkling_grid *grids, int acc,
                cudaStream_t st)
{
    sparkling_ctx::Batch &b = ctx->batch;
    int s;
    if ((s = batch_pack(ctx, K, K_dtype, grids, st))) return s;
    int64_t n = 0;
    double pairs = 0.0;
    // a prefix of pair items only (they write partial slots and counters,
    // which the real step resets and overwrites; K is untouched)
    while (n < b.n_lead_items && pairs < 1.5e11) pairs += b.item_pairs[n++];
    cudaEvent_t e0 = get_event(ctx), e1 = get_event(ctx);
    int best = 0;
    double best_rate = 0.0;
    for (int v = 0; v < kEngineVariants; ++v) {
        if (engine_ctas_per_sm(acc, K_dtype, v) < 1) { cudaGetLastError(); continue; }
        if ((s = batch_engine(ctx, K, K_dtype, acc, v, n, st))) return s;
        CK(cudaEventRecord(e0, st));
        if ((s = batch_engine(ctx, K, K_dtype, acc, v, n, st))) return s;
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double rate = ms > 0 ? pairs / (ms * 1e-3) : 0.0;
        char line[160];
        snprintf(line, sizeof line, "engine threads=%d: %.4g pairs/s (%lld pair items)\n",
                 engine_variant_threads(v), rate, (long long)n);
        ctx->tune_log += line;
        if (rate > best_rate) { best_rate = rate; best = v; }
    }
    ctx->pool.push_back(e0);
    ctx->pool.push_back(e1);
    ctx->engine_choice[acc][K_dtype] = best;
    return SPARKLING_OK;
}

} // namespace

// Lets other translation units of the library (noalloc.cu) report a failure
// through sparkling_last_error(NULL).
void sparkling_set_thread_error(const char *msg) { g_err = msg; }

extern "C" {

SPARKLING_API int sparkling_create(sparkling_ctx **out, int device)
{
    if (!out) return fail(nullptr, SPARKLING_E_INVAL, "out is NULL");
    *out = nullptr;
    if (device < 0) return fail(nullptr, SPARKLING_E_INVAL, "device %d < 0", device);
    sparkling_ctx *c = new (std::nothrow) sparkling_ctx();
    if (!c) return fail(nullptr, SPARKLING_E_NOMEM, "host allocation failed");
    c->device = device;
    c->err = "no error";
    *out = c;
    return SPARKLING_OK;
}

SPARKLING_API void sparkling_destroy(sparkling_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->inited) {
        cudaSetDevice(ctx->device);
        cudaDeviceSynchronize();
        if (ctx->batch.exec) cudaGraphExecDestroy(ctx->batch.exec);
        if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
        if (ctx->h_traj) cudaFreeHost(ctx->h_traj);
        cudaFree(ctx->ws);
        cudaFree(ctx->field);
        mesh_state_destroy(ctx->mesh);
        cudaFree(ctx->h_K);
        cudaFree(ctx->h_rho);
        cudaFree(ctx->d_status);
        cudaFree(ctx->d_small);
        for (auto &p : ctx->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        for (auto e : ctx->pool) cudaEventDestroy(e);
    }
    delete ctx;
}

SPARKLING_API const char *sparkling_last_error(const sparkling_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_err.c_str();
}

SPARKLING_API const char *sparkling_version(void) { return "sparkling-gb300 0.1 sm_103a"; }

SPARKLING_API int sparkling_grad(sparkling_ctx *ctx, const void *K, int K_dtype, int64_t N,
                                 const sparkling_grid *grid, int acc, void *G, int G_dtype, void *A,
                                 void *R, void *stream)
{
    int s;
    if ((s = common_checks(ctx, K, K_dtype, N, grid, acc))) return s;
    if (!G) return fail(ctx, SPARKLING_E_INVAL, "G is NULL");
    if ((s = validate_dtype(ctx, G_dtype, "G"))) return s;
    if ((s = lazy_init(ctx))) return s;
    if (!is_device_ptr(K) || !is_device_ptr(G) || !is_device_ptr(grid->rho) ||
        (A && !is_device_ptr(A)) || (R && !is_device_ptr(R)))
        return fail(ctx, SPARKLING_E_INVAL, "K, G, A, R and grid->rho must be device memory");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PairPlan P;
    Carve cv;
    if ((s = plan_pairs(ctx, N, grid, acc, false, false, P, cv))) return s;
    if ((s = ensure_ws(ctx, P.end))) return s;
    return run_pairs(ctx, K, K_dtype, grid, acc, false, P, G, G_dtype, A, R, false, st);
}

SPARKLING_API int sparkling_energy_backward(sparkling_ctx *ctx, const void *K, int K_dtype,
                                            int64_t N, const sparkling_grid *grid, int acc,
                                            const double *g_dev, double scale, void *dK,
                                            int dK_dtype, void *stream)
{
    int s;
    if ((s = common_checks(ctx, K, K_dtype, N, grid, acc))) return s;
    if (!dK) return fail(ctx, SPARKLING_E_INVAL, "dK is NULL");
    if ((s = validate_dtype(ctx, dK_dtype, "dK"))) return s;
    if (!std::isfinite(scale)) return fail(ctx, SPARKLING_E_INVAL, "scale must be finite");
    if ((s = lazy_init(ctx))) return s;
    if (!is_device_ptr(K) || !is_device_ptr(dK) || !is_device_ptr(grid->rho) ||
        (g_dev && !is_device_ptr(g_dev)))
        return fail(ctx, SPARKLING_E_INVAL, "K, dK, g_dev and grid->rho must be device memory");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PairPlan P;
    Carve cv;
    if ((s = plan_pairs(ctx, N, grid, acc, false, false, P, cv))) return s;
    if ((s = ensure_ws(ctx, P.end))) return s;
    return run_pairs(ctx, K, K_dtype, grid, acc, false, P, dK, dK_dtype, nullptr, nullptr, false, st,
                     scale / (double)N, g_dev);
}

SPARKLING_API int sparkling_energy(sparkling_ctx *ctx, const void *K, int K_dtype, int64_t N,
                                   const sparkling_grid *grid, int acc, double *F_host,
                                   double *Fa_host, double *Fr_host, void *stream)
{
    int s;
    if ((s = common_checks(ctx, K, K_dtype, N, grid, acc))) return s;
    if ((s = lazy_init(ctx))) return s;
    if (!is_device_ptr(K) || !is_device_ptr(grid->rho))
        return fail(ctx, SPARKLING_E_INVAL, "K and grid->rho must be device memory");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PairPlan P;
    Carve cv;
    if ((s = plan_pairs(ctx, N, grid, acc, true, false, P, cv))) return s;
    if ((s = ensure_ws(ctx, P.end))) return s;
    if ((s = run_pairs(ctx, K, K_dtype, grid, acc, true, P, nullptr, 0, nullptr, nullptr, false, st)))
        return s;
    double h[2];
    CK(cudaMemcpyAsync(h, ctx->d_small, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if ((s = read_status(ctx, st))) return s;
    if (Fa_host) *Fa_host = h[0];
    if (Fr_host) *Fr_host = h[1];
    if (F_host) *F_host = h[0] - h[1];
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_project(sparkling_ctx *ctx, void *K, int K_dtype, int64_t Nc, int64_t Ns,
                                    const sparkling_proj *proj, double *viol_host, void *stream)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    int s;
    if (!K) return fail(ctx, SPARKLING_E_INVAL, "K is NULL");
    if ((s = validate_dtype(ctx, K_dtype, "K"))) return s;
    if ((s = check_shots(ctx, Nc, Ns))) return s;
    if ((s = validate_proj(ctx, proj, Ns))) return s;
    if ((s = lazy_init(ctx))) return s;
    if (!is_device_ptr(K)) return fail(ctx, SPARKLING_E_INVAL, "K must be device memory");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Carve cv;
    ProjPlan L;
    if ((s = plan_project(ctx, K_dtype, Nc, Ns, cv, L))) return s;
    if ((s = ensure_ws(ctx, cv.off))) return s;
    if ((s = run_project(ctx, K, K_dtype, Nc, Ns, proj, nullptr, 0.0, L, viol_host != nullptr, st)))
        return s;
    if (viol_host || proj->tol > 0) return finish_project(ctx, proj, viol_host, st);
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_step(sparkling_ctx *ctx, void *K, int K_dtype, int64_t Nc, int64_t Ns,
                                 const sparkling_grid *grid, int acc, double eta,
                                 const sparkling_proj *proj, void *stream)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    int s;
    if ((s = check_shots(ctx, Nc, Ns))) return s;
    if ((s = common_checks(ctx, K, K_dtype, Nc * Ns, grid, acc))) return s;
    if ((s = validate_proj(ctx, proj, Ns))) return s;
    if (!std::isfinite(eta)) return fail(ctx, SPARKLING_E_INVAL, "eta must be finite");
    if ((s = lazy_init(ctx))) return s;
    if (!is_device_ptr(K) || !is_device_ptr(grid->rho))
        return fail(ctx, SPARKLING_E_INVAL, "K and grid->rho must be device memory");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t N = Nc * Ns;
    // The persistent engine takes the whole step in one launch (B = 1) where
    // it applies: direct sums, a per-target fold it has, fixed iterations.
    const bool engine_applies = ctx->attr_mode == SPARKLING_ATTRACTION_DIRECT &&
                                ctx->rep_mode == SPARKLING_REPULSION_DIRECT &&
                                (acc == SPARKLING_ACC_KAHAN32 || acc == SPARKLING_ACC_FP64) &&
                                !(proj->tol > 0) && N >= 2 && N <= ((int64_t)1 << 31) - kTile;
    if (engine_applies && (ctx->step_path == SPARKLING_STEP_ENGINE ||
                           (ctx->step_path == SPARKLING_STEP_AUTO && N >= kStepEngineMin))) {
        StepScope whole(ctx, st);
        const int64_t off[2] = {0, N};
        if ((s = sparkling_step_batched(ctx, 1, off, K, K_dtype, (int32_t)Ns, grid, &eta, proj, acc,
                                        SPARKLING_BATCH_GRAPH, stream)))
            return s;
        whole.done();
        return SPARKLING_OK;
    }
    PairPlan P;
    Carve cv;
    if ((s = plan_pairs(ctx, N, grid, acc, false, true, P, cv))) return s;
    ProjPlan L;
    if ((s = plan_project(ctx, K_dtype, Nc, Ns, cv, L))) return s;
    if ((s = ensure_ws(ctx, cv.off))) return s;
    // the whole device work of the step, timed as one scope when timing is on
    StepScope whole(ctx, st);
    if ((s = run_pairs(ctx, K, K_dtype, grid, acc, false, P, nullptr, K_dtype, nullptr, nullptr, true,
                       st)))
        return s;
    if ((s = run_project(ctx, K, K_dtype, Nc, Ns, proj, at<double>(ctx, P.o_g64), eta, L, false, st)))
        return s;
    whole.done();
    if (proj->tol > 0) return finish_project(ctx, proj, nullptr, st);
    return SPARKLING_OK;
}

// ---------------------------------------------------------------------------
// Multi-resolution driver (Algorithm 1).

namespace {

int validate_schedule(sparkling_ctx *ctx, const sparkling_schedule *sc)
{
    if (!sc) return fail(ctx, SPARKLING_E_INVAL, "sched is NULL");
    if (!(sc->eta > 0) || !std::isfinite(sc->eta))
        return fail(ctx, SPARKLING_E_INVAL, "sched->eta must be finite and > 0");
    if (!(sc->eta_min > 0) || !(sc->eta_max >= sc->eta_min) || std::isnan(sc->eta_max))
        return fail(ctx, SPARKLING_E_INVAL, "sched needs 0 < eta_min <= eta_max");
    if (!(sc->alpha_factor > 0) || !(sc->beta_factor > 0) || !std::isfinite(sc->alpha_factor) ||
        !std::isfinite(sc->beta_factor))
        return fail(ctx, SPARKLING_E_INVAL, "sched alpha_factor, beta_factor must be finite and > 0");
    if (sc->n_git < 0 || sc->n_fixed < 0)
        return fail(ctx, SPARKLING_E_INVAL, "sched n_git, n_fixed must be >= 0");
    return SPARKLING_OK;
}

int optimize_checks(sparkling_ctx *ctx, void *K, int K_dtype, int64_t Nc, int64_t Ns,
                    const sparkling_grid *grid, const sparkling_proj *proj, int acc,
                    const sparkling_schedule *sc)
{
    int s;
    if ((s = check_shots(ctx, Nc, Ns))) return s;
    if ((s = common_checks(ctx, K, K_dtype, Nc * Ns, grid, acc))) return s;
    if ((s = validate_proj(ctx, proj, Ns))) return s;
    return validate_schedule(ctx, sc);
}

// The iterations of sparkling_optimize (arguments already validated).
int run_optimize(sparkling_ctx *ctx, void *K, int K_dtype, int64_t Nc, int64_t Ns,
                 const sparkling_grid *grid, const sparkling_proj *proj, int acc,
                 const sparkling_schedule *sc, double *trace, cudaStream_t st)
{
    const int64_t N = Nc * Ns, n3 = 3 * N;
    PairPlan P;
    Carve cv;
    int s;
    if ((s = plan_pairs(ctx, N, grid, acc, false, true, P, cv))) return s;
    ProjPlan L;
    if ((s = plan_project(ctx, K_dtype, Nc, Ns, cv, L))) return s;
    const size_t o_kp = cv.take((size_t)n3 * sizeof(double));
    const size_t o_gp = cv.take((size_t)n3 * sizeof(double));
    const size_t o_part = cv.take((size_t)bb_blocks(n3, ctx->sms) * sizeof(double2));
    if ((s = ensure_ws(ctx, cv.off))) return s;
    const double *G64 = at<double>(ctx, P.o_g64);
    double step = sc->eta;
    for (int t = 0; t < sc->n_git; ++t) {
        if ((s = run_pairs(ctx, K, K_dtype, grid, acc, false, P, nullptr, K_dtype, nullptr, nullptr,
                           true, st)))
            return s;
        const bool bb = t >= sc->n_fixed && t > 0;
        {
            LaunchScope ls(ctx, SPARKLING_KERNEL_DRIVER, st);
            CK(launch_bb(K, K_dtype, at<double>(ctx, o_kp), G64, at<double>(ctx, o_gp), n3, bb,
                         at<double2>(ctx, o_part), ctx->d_small + 2, ctx->sms, st));
            ls.done(bb ? 2 : 1);
        }
        if (t < sc->n_fixed) {
            step = sc->eta;
        } else if (bb) {
            double h[2];
            CK(cudaMemcpyAsync(h, ctx->d_small + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
            if ((s = read_status(ctx, st))) return s;
            if (h[1] > 0.0 && std::isfinite(h[0] / h[1]))
                step = std::min(std::max(h[0] / h[1], sc->eta_min), sc->eta_max);
        }
        if (trace) trace[t] = step;
        if ((s = run_project(ctx, K, K_dtype, Nc, Ns, proj, G64, step, L, false, st))) return s;
        if (proj->tol > 0 && (s = finish_project(ctx, proj, nullptr, st))) return s;
    }
    return read_status(ctx, st);
}

int write_checkpoint(sparkling_ctx *ctx, const char *prefix, int level, const void *K, int K_dtype,
                     int64_t Nc, int64_t Ns, cudaStream_t st)
{
    const size_t bytes = (size_t)Nc * Ns * 3 * (K_dtype == SPARKLING_F32 ? 4 : 8);
    std::vector<char> host(bytes);
    CK(cudaMemcpyAsync(host.data(), K, bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    char path[4096];
    if (snprintf(path, sizeof path, "%s_level%d.bin", prefix, level) >= (int)sizeof path)
        return fail(ctx, SPARKLING_E_IO, "checkpoint path too long");
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(ctx, SPARKLING_E_IO, "cannot open %s for writing", path);
    char head[64] = {0};
    std::memcpy(head, "SPKLCKPT", 8);
    const int64_t fields[5] = {1, Nc, Ns, level, K_dtype};
    std::memcpy(head + 8, fields, sizeof fields);
    bool ok = std::fwrite(head, 1, sizeof head, f) == sizeof head &&
              std::fwrite(host.data(), 1, bytes, f) == bytes;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(ctx, SPARKLING_E_IO, "writing %s failed", path);
    return SPARKLING_OK;
}

} // namespace

SPARKLING_API int sparkling_upsample(sparkling_ctx *ctx, const void *Kc, void *Kf, int dtype,
                                     int64_t Nc, int64_t d, void *stream)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    int s;
    if (!Kc || !Kf) return fail(ctx, SPARKLING_E_INVAL, "Kc and Kf are required");
    if ((s = validate_dtype(ctx, dtype, "K"))) return s;
    if (Nc < 1 || d < 1 || Nc > ((int64_t)1 << 40) / d)
        return fail(ctx, SPARKLING_E_INVAL, "Nc = %lld, d = %lld out of range", (long long)Nc,
                    (long long)d);
    const size_t es = dtype == SPARKLING_F32 ? 4 : 8;
    const char *a = static_cast<const char *>(Kc), *b = static_cast<const char *>(Kf);
    if (a < b + (size_t)Nc * 2 * d * 3 * es && b < a + (size_t)Nc * d * 3 * es)
        return fail(ctx, SPARKLING_E_INVAL, "Kc and Kf overlap");
    if ((s = lazy_init(ctx))) return s;
    if (!is_device_ptr(Kc) || !is_device_ptr(Kf))
        return fail(ctx, SPARKLING_E_INVAL, "Kc and Kf must be device memory");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LaunchScope ls(ctx, SPARKLING_KERNEL_DRIVER, st);
    CK(launch_upsample(Kc, Kf, dtype, Nc, d, ctx->sms, st));
    ls.done();
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_optimize(sparkling_ctx *ctx, void *K, int K_dtype, int64_t Nc,
                                     int64_t Ns, const sparkling_grid *grid,
                                     const sparkling_proj *proj, int acc,
                                     const sparkling_schedule *sched, double *trace, void *stream)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    int s;
    if ((s = optimize_checks(ctx, K, K_dtype, Nc, Ns, grid, proj, acc, sched))) return s;
    if ((s = lazy_init(ctx))) return s;
    if (!is_device_ptr(K) || !is_device_ptr(grid->rho))
        return fail(ctx, SPARKLING_E_INVAL, "K and grid->rho must be device memory");
    return run_optimize(ctx, K, K_dtype, Nc, Ns, grid, proj, acc, sched, trace,
                        static_cast<cudaStream_t>(stream));
}

SPARKLING_API int sparkling_multires(sparkling_ctx *ctx, void *K, int K_dtype, int64_t Nc,
                                     int64_t Ns, const sparkling_grid *grid,
                                     const sparkling_proj *proj, int acc,
                                     const sparkling_schedule *sched, int32_t start_level,
                                     const char *checkpoint_prefix, double *trace, void *stream)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    int s;
    if (start_level < 0 || start_level > 20 || Ns % ((int64_t)1 << start_level) != 0)
        return fail(ctx, SPARKLING_E_INVAL, "Ns = %lld must be a multiple of 2^start_level (%d)",
                    (long long)Ns, start_level);
    if ((s = optimize_checks(ctx, K, K_dtype, Nc, Ns, grid, proj, acc, sched))) return s;
    if ((s = check_shots(ctx, Nc, Ns >> start_level))) return s;
    if (Nc * (Ns >> start_level) < 2)
        return fail(ctx, SPARKLING_E_INVAL, "the first level needs at least 2 samples");
    if ((s = lazy_init(ctx))) return s;
    if (!is_device_ptr(K) || !is_device_ptr(grid->rho))
        return fail(ctx, SPARKLING_E_INVAL, "K and grid->rho must be device memory");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t es = K_dtype == SPARKLING_F32 ? 4 : 8;
    for (int l = start_level; l >= 0; --l) {
        const int64_t Nsl = Ns >> l;
        sparkling_proj pl = *proj;
        pl.alpha = proj->alpha * std::pow(sched->alpha_factor, (double)l);
        pl.beta = proj->beta * std::pow(sched->beta_factor, (double)l);
        pl.pin_index = proj->pin_index >= 0 ? proj->pin_index >> l : -1;
        if ((s = run_optimize(ctx, K, K_dtype, Nc, Nsl, grid, &pl, acc, sched, trace, st))) return s;
        if (trace) trace += sched->n_git;
        if (checkpoint_prefix &&
            (s = write_checkpoint(ctx, checkpoint_prefix, l, K, K_dtype, Nc, Nsl, st)))
            return s;
        if (l > 0) {
            Carve cv;
            const size_t o_up = cv.take((size_t)Nc * 2 * Nsl * 3 * es);
            if ((s = ensure_ws(ctx, cv.off))) return s;
            void *tmp = at<char>(ctx, o_up);
            {
                LaunchScope ls(ctx, SPARKLING_KERNEL_DRIVER, st);
                CK(launch_upsample(K, tmp, K_dtype, Nc, Nsl, ctx->sms, st));
                ls.done();
            }
            CK(cudaMemcpyAsync(K, tmp, (size_t)Nc * 2 * Nsl * 3 * es, cudaMemcpyDeviceToDevice, st));
        }
    }
    return read_status(ctx, st);
}

SPARKLING_API int sparkling_step_batched(sparkling_ctx *ctx, int32_t B, const int64_t *traj_off,
                                         void *K, int K_dtype, int32_t Ns,
                                         const sparkling_grid *grids, const double *eta,
                                         const sparkling_proj *proj, int acc, int flags,
                                         void *stream)
{
    int s;
    if ((s = validate_batch(ctx, B, traj_off, K, K_dtype, Ns, grids, eta, proj, acc))) return s;
    if ((s = lazy_init(ctx))) return s;
    if ((s = ensure_occupancy(ctx))) return s;
    if (!is_device_ptr(K)) return fail(ctx, SPARKLING_E_INVAL, "K must be device memory");
    for (int t = 0; t < B; ++t)
        if (!is_device_ptr(grids[t].rho))
            return fail(ctx, SPARKLING_E_INVAL, "grids[%d].rho must be device memory", t);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    sparkling_ctx::Batch &b = ctx->batch;
    std::vector<int64_t> off(traj_off, traj_off + B + 1);
    std::vector<int32_t> dims;
    for (int t = 0; t < B; ++t)
        for (int a = 0; a < 3; ++a) dims.push_back(grids[t].n[a]);
    // one launch (the default): the symmetric repulsion as items of the
    // engine's work list; it needs the symmetric arithmetic and the one-launch
    // shape to be resident, else the repulsion runs ahead in its own kernel
    const bool one_launch = !(flags & SPARKLING_BATCH_TWO_LAUNCHES) && ctx->rep_symmetric &&
                            engine_ctas_per_sm(acc, K_dtype, kEngineOneLaunch) >= 1;
    cudaGetLastError();
    int occ = 0;
    if (one_launch)
        occ = engine_ctas_per_sm(acc, K_dtype, kEngineOneLaunch);
    else
        for (int v = 0; v < kEngineVariants; ++v)
            occ = std::max(occ, engine_ctas_per_sm(acc, K_dtype, v));
    cudaGetLastError();
    if (occ < 1) return fail(ctx, SPARKLING_E_CUDA, "engine kernel cannot be resident");
    const int ctas = ctx->sms * occ;   // the largest wave of any engine shape
    const bool same = b.valid && b.B == B && b.Ns == Ns && b.acc == acc && b.dtype == K_dtype &&
                      b.ctas == ctas && b.items_per_cta == ctx->items_per_cta && b.off == off &&
                      b.dims == dims && b.one_launch == one_launch;
    if (!same) {
        if (b.exec) { cudaGraphExecDestroy(b.exec); b.exec = nullptr; }
        b = sparkling_ctx::Batch();
        b.B = B; b.Ns = Ns; b.acc = acc; b.dtype = K_dtype; b.ctas = ctas;
        b.items_per_cta = ctx->items_per_cta;
        b.off = off; b.dims = dims;
        b.one_launch = one_launch;
        b.sym = ctx->rep_symmetric && !one_launch;
        build_work_list(b, off, grids, ctas, ctx->items_per_cta, b.sym, b.one_launch);
        b.roles = one_launch;
        if (b.roles) split_work_list(b);
        Carve cv;
        b.o_pos = cv.take((size_t)off[B] * sizeof(float4));
        for (int t = 0; t < B; ++t) {
            b.o_rho.push_back(cv.take((size_t)b.traj[t].ny * b.traj[t].nz * b.traj[t].gxp * sizeof(float)));
            b.o_coords.push_back(cv.take(((size_t)b.traj[t].gxp + b.traj[t].ny + b.traj[t].nz) * sizeof(float)));
        }
        b.o_traj = cv.take((size_t)B * sizeof(EngineTraj));
        b.o_items = cv.take(b.items.size() * sizeof(EngineItem));
        b.o_cnt = cv.take((size_t)(3 + B + kSmSlots) * sizeof(unsigned int));
        int64_t parts = 0;
        for (int t = 0; t < B; ++t) parts += (int64_t)b.traj[t].tiles * b.traj[t].slots;
        b.o_part = cv.take((size_t)parts * kTile * sizeof(dacc4));
        b.proj_in_smem = project_state_bytes(Ns) <= engine_proj_smem_limit();
        if (!b.proj_in_smem) b.o_gstate = cv.take((size_t)ctas * project_state_bytes(Ns));
        if (b.sym || b.one_launch)
            b.o_racc = cv.take((size_t)off[B] * 3 * sizeof(unsigned long long));
        if (b.sym) {
            b.o_symtraj = cv.take((size_t)B * sizeof(SymTraj));
            int64_t u = 0;
            for (int t = 0; t < B; ++t) {
                SymTraj q;
                q.off = off[t];
                q.N = off[t + 1] - off[t];
                q.tiles = (q.N + kTile - 1) / kTile;
                q.unit0 = u;
                u += tri_count(q.tiles);
                b.symtraj.push_back(q);
            }
            b.sym_units = u;
        }
        b.end = cv.off;
        b.kernels_per_step = 2 + B + (b.sym ? 1 : 0);   // packs, (symmetric repulsion), engine
        if ((s = ensure_ws(ctx, b.end))) { b.valid = false; return s; }
        CK(cudaMemcpyAsync(at<EngineItem>(ctx, b.o_items), b.items.data(),
                           b.items.size() * sizeof(EngineItem), cudaMemcpyHostToDevice, st));
        if (b.sym)
            CK(cudaMemcpyAsync(at<SymTraj>(ctx, b.o_symtraj), b.symtraj.data(),
                               (size_t)B * sizeof(SymTraj), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        b.valid = true;
    }
    // Per-call trajectory descriptors (step sizes, constraints, grid origin).
    if (ctx->h_traj_cap < (size_t)B) {
        CK(cudaStreamSynchronize(st));
        if (ctx->h_traj) cudaFreeHost(ctx->h_traj);
        ctx->h_traj = nullptr;
        ctx->h_traj_cap = 0;
        CK(cudaMallocHost((void **)&ctx->h_traj, (size_t)B * sizeof(EngineTraj)));
        ctx->h_traj_cap = B;
    } else {
        CK(cudaStreamSynchronize(st));   // the staging buffer may still feed a previous copy
    }
    for (int t = 0; t < B; ++t) {
        EngineTraj tr = b.traj[t];
        const double h = (grids[t].hi - grids[t].lo) / grids[t].n[0];
        tr.x0 = grids[t].lo + 0.5 * h;
        tr.hx = (float)h;
        tr.rho = at<float>(ctx, b.o_rho[t]);
        tr.coords = at<float>(ctx, b.o_coords[t]);
        tr.eta = eta[t];
        tr.alpha = proj[t].alpha; tr.beta = proj[t].beta; tr.box = proj[t].box;
        for (int c = 0; c < 3; ++c) tr.pin[c] = proj[t].pin[c];
        tr.pin_index = proj[t].pin_index < 0 ? -1 : proj[t].pin_index;
        tr.n_iter = proj[t].n_iter;
        ctx->h_traj[t] = tr;
    }
    CK(cudaMemcpyAsync(at<EngineTraj>(ctx, b.o_traj), ctx->h_traj, (size_t)B * sizeof(EngineTraj),
                       cudaMemcpyHostToDevice, st));

    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cap));
    if (!b.one_launch && ctx->autotune && ctx->engine_choice[acc][K_dtype] < 0 &&
        cap == cudaStreamCaptureStatusNone)
        if ((s = tune_engine(ctx, K, K_dtype, grids, acc, st))) return s;
    const int variant = b.one_launch ? kEngineOneLaunch
                        : ctx->engine_choice[acc][K_dtype] < 0 ? 0 : ctx->engine_choice[acc][K_dtype];

    // Graph replay when asked for and the call matches the captured one.
    std::vector<const void *> key;
    key.push_back(K);
    key.push_back(ctx->ws);
    for (int t = 0; t < B; ++t) key.push_back(grids[t].rho);
    const bool use_graph = (flags & SPARKLING_BATCH_GRAPH) && cap == cudaStreamCaptureStatusNone;
    LaunchScope ls(ctx, SPARKLING_KERNEL_ENGINE, st);
    if (use_graph && b.exec && b.graph_key == key && b.graph_variant == variant &&
        b.graph_eps2 == eps2_of(ctx) && b.graph_proj == ctx->proj_mode) {
        CK(cudaGraphLaunch(b.exec, st));
    } else if (use_graph && b.eager_calls > 0) {
        // Capture (which records without executing) on a private stream --
        // the legacy default stream cannot be captured -- and launch the
        // graph on the caller's stream.
        if (b.exec) { cudaGraphExecDestroy(b.exec); b.exec = nullptr; }
        if (!ctx->cap_stream)
            CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int w = batch_device_work(ctx, K, K_dtype, grids, acc, variant, ctx->cap_stream);
        cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
        if (w) { if (g) cudaGraphDestroy(g); return w; }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&b.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { b.exec = nullptr; return cuda_fail(ctx, e, "cudaGraphInstantiate"); }
        b.graph_key = key;
        b.graph_variant = variant;
        b.graph_eps2 = eps2_of(ctx);
        b.graph_proj = ctx->proj_mode;
        CK(cudaGraphLaunch(b.exec, st));
    } else {
        if ((s = batch_device_work(ctx, K, K_dtype, grids, acc, variant, st))) return s;
        ++b.eager_calls;
    }
    ls.done((int)b.kernels_per_step);
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_step_host(sparkling_ctx *ctx, void *K_host, int K_dtype, int64_t Nc,
                                      int64_t Ns, const sparkling_grid *grid, const float *rho_host,
                                      int acc, double eta, const sparkling_proj *proj, void *stream)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    int s;
    if (!K_host || !rho_host) return fail(ctx, SPARKLING_E_INVAL, "K_host and rho_host are required");
    if ((s = validate_dtype(ctx, K_dtype, "K"))) return s;
    if ((s = check_shots(ctx, Nc, Ns))) return s;
    if ((s = validate_grid(ctx, grid, false))) return s;
    if ((s = lazy_init(ctx))) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t kb = (size_t)Nc * Ns * 3 * (K_dtype == SPARKLING_F32 ? 4 : 8);
    const size_t rb = (size_t)grid->n[0] * grid->n[1] * grid->n[2] * sizeof(float);
    if (kb > ctx->h_K_bytes) {
        if ((s = check_limit(ctx, held_bytes(ctx) - ctx->h_K_bytes, kb, "device copy of K"))) return s;
        CK(cudaDeviceSynchronize());
        cudaFree(ctx->h_K);
        ctx->h_K = nullptr;
        ctx->h_K_bytes = 0;
        if (cudaMalloc(&ctx->h_K, kb) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, SPARKLING_E_NOMEM, "device copy of K (%zu bytes) failed", kb);
        }
        ctx->h_K_bytes = kb;
    }
    if (rb > ctx->h_rho_bytes) {
        if ((s = check_limit(ctx, held_bytes(ctx) - ctx->h_rho_bytes, rb, "device copy of rho")))
            return s;
        CK(cudaDeviceSynchronize());
        cudaFree(ctx->h_rho);
        ctx->h_rho = nullptr;
        ctx->h_rho_bytes = 0;
        if (cudaMalloc(&ctx->h_rho, rb) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, SPARKLING_E_NOMEM, "device copy of rho (%zu bytes) failed", rb);
        }
        ctx->h_rho_bytes = rb;
    }
    CK(cudaMemcpyAsync(ctx->h_K, K_host, kb, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->h_rho, rho_host, rb, cudaMemcpyHostToDevice, st));
    sparkling_grid g = *grid;
    g.rho = ctx->h_rho;
    if (ctx->field_rho == ctx->h_rho) ctx->field_valid = false;   // new density values
    if ((s = sparkling_step(ctx, ctx->h_K, K_dtype, Nc, Ns, &g, acc, eta, proj, stream))) return s;
    CK(cudaMemcpyAsync(K_host, ctx->h_K, kb, cudaMemcpyDeviceToHost, st));
    return read_status(ctx, st);
}

SPARKLING_API int sparkling_status(sparkling_ctx *ctx, void *stream)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    if (!ctx->inited) return SPARKLING_OK;
    int s;
    if ((s = lazy_init(ctx))) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    return read_status(ctx, st);
}

SPARKLING_API int sparkling_set_timing(sparkling_ctx *ctx, int enable)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    ctx->timing = enable != 0;
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_kernel_times(sparkling_ctx *ctx, double *ms_out, int64_t *launches_out,
                                         int n, int reset)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    if (n < 0) return fail(ctx, SPARKLING_E_INVAL, "n < 0");
    for (auto &p : ctx->pending) {
        cudaError_t e = cudaEventSynchronize(p.b);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventSynchronize");
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) ctx->ms[p.kind] += ms;
        ctx->pool.push_back(p.a);
        ctx->pool.push_back(p.b);
    }
    ctx->pending.clear();
    for (int k = 0; k < n && k < SPARKLING_KERNEL_COUNT; ++k) {
        if (ms_out) ms_out[k] = ctx->ms[k];
        if (launches_out) launches_out[k] = ctx->nlaunch[k];
    }
    if (reset)
        for (int k = 0; k < SPARKLING_KERNEL_COUNT; ++k) { ctx->ms[k] = 0; ctx->nlaunch[k] = 0; }
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_set_autotune(sparkling_ctx *ctx, int enable)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    ctx->autotune = enable != 0;
    if (enable < 0) {   // forget the choices made so far
        ctx->attr_choice.clear();
        ctx->rep_choice[0] = ctx->rep_choice[1] = -1;
        for (auto &row : ctx->engine_choice) row[0] = row[1] = -1;
        ctx->sym_choice = -1;
        ctx->pin_attr = -1;
        ctx->tune_log.clear();
        ctx->autotune = true;
    }
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_set_shape(sparkling_ctx *ctx, int kernel, int variant)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    if (kernel == SPARKLING_KERNEL_ATTRACTION) {
        if (variant < -1 || variant >= kAttrVariants)
            return fail(ctx, SPARKLING_E_INVAL, "attraction shape %d not in -1..%d", variant,
                        kAttrVariants - 1);
        ctx->pin_attr = variant;
        return SPARKLING_OK;
    }
    if (kernel == SPARKLING_KERNEL_REPULSION) {
        if (variant < -1 || variant >= kSymVariants)
            return fail(ctx, SPARKLING_E_INVAL, "repulsion shape %d not in -1..%d", variant,
                        kSymVariants - 1);
        ctx->sym_choice = variant;
        return SPARKLING_OK;
    }
    return fail(ctx, SPARKLING_E_INVAL, "kernel %d has no selectable shape", kernel);
}

SPARKLING_API int sparkling_set_projection(sparkling_ctx *ctx, int mode)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    if (mode != SPARKLING_PROJECTION_FP64 && mode != SPARKLING_PROJECTION_MIXED)
        return fail(ctx, SPARKLING_E_INVAL, "projection mode %d is not FP64/MIXED", mode);
    ctx->proj_mode = mode;
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_set_step_path(sparkling_ctx *ctx, int path)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    if (path != SPARKLING_STEP_AUTO && path != SPARKLING_STEP_KERNELS && path != SPARKLING_STEP_ENGINE)
        return fail(ctx, SPARKLING_E_INVAL, "step path %d is not AUTO/KERNELS/ENGINE", path);
    ctx->step_path = path;
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_set_wait_budget(sparkling_ctx *ctx, int64_t cycles)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    if (cycles < 0) cycles = kWaitCycles;
    if (cycles > ((int64_t)1 << 40))
        return fail(ctx, SPARKLING_E_INVAL, "wait budget %lld cycles is too large", (long long)cycles);
    ctx->wait_cycles = cycles;
    if (ctx->inited) {
        // kernels read the budget from the control block: wait until none
        // is running, then replace it
        CK(cudaSetDevice(ctx->device));
        CK(cudaDeviceSynchronize());
        const long long v = cycles;
        CK(cudaMemcpy(reinterpret_cast<char *>(ctx->d_status) + offsetof(DevCtl, wait_cycles), &v,
                      sizeof v, cudaMemcpyHostToDevice));
    }
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_set_memory_limit(sparkling_ctx *ctx, int64_t bytes)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    if (bytes < 0) return fail(ctx, SPARKLING_E_INVAL, "memory limit must be >= 0");
    ctx->mem_limit = (size_t)bytes;
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_set_attraction(sparkling_ctx *ctx, int mode)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    if (mode != SPARKLING_ATTRACTION_DIRECT && mode != SPARKLING_ATTRACTION_FIELD)
        return fail(ctx, SPARKLING_E_INVAL, "attraction mode %d is not DIRECT/FIELD", mode);
    ctx->attr_mode = mode;
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_set_regularisation(sparkling_ctx *ctx, double eps)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    if (!(eps >= 0.0) || !std::isfinite(eps) || eps > 1e3)
        return fail(ctx, SPARKLING_E_INVAL, "eps = %g must be finite, in [0, 1e3]", eps);
    ctx->eps = eps;
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_set_repulsion(sparkling_ctx *ctx, int mode, const sparkling_mesh *mesh)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    if (mode == SPARKLING_REPULSION_DIRECT) {
        ctx->rep_mode = mode;
        return SPARKLING_OK;
    }
    if (mode != SPARKLING_REPULSION_MESH)
        return fail(ctx, SPARKLING_E_INVAL, "repulsion mode %d is not DIRECT/MESH", mode);
    if (!mesh) return fail(ctx, SPARKLING_E_INVAL, "mesh is NULL");
    if (!(std::isfinite(mesh->lo) && std::isfinite(mesh->hi) && mesh->hi > mesh->lo))
        return fail(ctx, SPARKLING_E_INVAL, "mesh needs finite lo < hi");
    if (mesh->n_cells < 8 || mesh->n_cells > 1024)
        return fail(ctx, SPARKLING_E_INVAL, "mesh n_cells = %d must be in [8, 1024]", mesh->n_cells);
    if (!(mesh->sigma_cells > 0) || !std::isfinite(mesh->sigma_cells) || mesh->sigma_cells > 64)
        return fail(ctx, SPARKLING_E_INVAL, "mesh sigma_cells must be in (0, 64]");
    if (!(mesh->rc_sigmas >= 2) || !std::isfinite(mesh->rc_sigmas) || mesh->rc_sigmas > 16)
        return fail(ctx, SPARKLING_E_INVAL, "mesh rc_sigmas must be in [2, 16]");
    ctx->rep_mode = mode;
    ctx->mesh_params = *mesh;
    return SPARKLING_OK;
}

SPARKLING_API int sparkling_attraction_field(sparkling_ctx *ctx, const sparkling_grid *grid,
                                             void *stream)
{
    if (!ctx) return fail(nullptr, SPARKLING_E_INVAL, "ctx is NULL");
    int s;
    if ((s = validate_grid(ctx, grid, true))) return s;
    if ((s = lazy_init(ctx))) return s;
    if (!is_device_ptr(grid->rho)) return fail(ctx, SPARKLING_E_INVAL, "grid->rho must be device memory");
    return build_field(ctx, grid, static_cast<cudaStream_t>(stream));
}

SPARKLING_API int sparkling_tuning_report(const sparkling_ctx *ctx, char *buf, int64_t len)
{
    if (!ctx || !buf || len < 1) return SPARKLING_E_INVAL;
    std::string r = ctx->tune_log;
    for (const auto &kv : ctx->attr_choice) {
        char line[128];
        snprintf(line, sizeof line, "chosen attraction acc=%d gxp=%d: threads=%d\n",
                 (int)(kv.first >> 20), (int)(kv.first & ((1 << 20) - 1)),
                 attr_variant_threads(kv.second));
        r += line;
    }
    for (int acc = 0; acc < 2; ++acc)
        if (ctx->rep_choice[acc] >= 0) {
            char line[128];
            snprintf(line, sizeof line, "chosen repulsion acc=%d: threads=%d unroll=%d\n", acc,
                     rep_variant_threads(ctx->rep_choice[acc]),
                     rep_variant_unroll(ctx->rep_choice[acc]));
            r += line;
        }
    if (ctx->sym_choice >= 0) {
        char line[128];
        snprintf(line, sizeof line, "chosen repulsion symmetric: threads=%d sources/lane=%d %s-paired\n",
                 sym_variant_threads(ctx->sym_choice), sym_variant_sources(ctx->sym_choice),
                 sym_variant_source_paired(ctx->sym_choice) ? "source" : "target");
        r += line;
    }
    const size_t n = std::min<size_t>(r.size(), (size_t)len - 1);
    std::memcpy(buf, r.data(), n);
    buf[n] = 0;
    return SPARKLING_OK;
}

SPARKLING_API int64_t sparkling_launch_count(const sparkling_ctx *ctx)
{
    return ctx ? ctx->launches : 0;
}

} // extern "C"
