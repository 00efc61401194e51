// C ABI of the SPARKLING GB300 library (declared in include/sparkling.h).
//
// Host-side orchestration only: argument validation, the device workspace,
// the even work split of the pair kernels, launch bookkeeping (counts and
// optional CUDA-event timing) and status reporting.  All arithmetic of the
// hot path runs in the kernels of pairs.cu and project.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/sparkling.h"
#include "kernels.h"

using namespace sparkling;

struct sparkling_ctx {
    int device = 0;
    bool inited = false;
    int sms = 0;
    int *d_status = nullptr;    // device status word
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
    // occupancy cache
    int occ_attr[2][2] = {{-1, -1}, {-1, -1}};
    int occ_attr_gxp[2][2] = {{-1, -1}, {-1, -1}};
    int occ_rep[2][2] = {{-1, -1}, {-1, -1}};
};

namespace {

thread_local std::string g_err = "no error";

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
    CK(cudaMalloc(&ctx->d_status, sizeof(int)));
    CK(cudaMemset(ctx->d_status, 0, sizeof(int)));
    CK(cudaMalloc(&ctx->d_small, 8 * sizeof(double)));
    CK(cudaMemset(ctx->d_small, 0, 8 * sizeof(double)));
    ctx->inited = true;
    return SPARKLING_OK;
}

// Device (or managed) memory the current device can dereference.
bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
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

int ensure_ws(sparkling_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->ws_bytes) return SPARKLING_OK;
    // Growth is rare (first call of a larger problem): synchronise so that no
    // queued kernel still uses the old buffer, then reallocate with headroom.
    CK(cudaDeviceSynchronize());
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    const size_t want = align_up(bytes + bytes / 8, 1 << 20);
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
    void done(int nkernels = 1)
    {
        ctx->launches += nkernels;
        ctx->nlaunch[kind] += nkernels;
        if (a && b) {
            cudaEventRecord(b, st);
            ctx->pending.push_back({kind, a, b});
        }
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
    Split spa, spr;
    size_t o_pos, o_rho, o_coords, o_parta, o_partr, o_eblocks, o_g64, end;
};

int plan_pairs(sparkling_ctx *ctx, int64_t N, const sparkling_grid *g, int acc, bool energy,
               bool need_g64, PairPlan &P, Carve &cv)
{
    P.N = N;
    P.nx = g->n[0]; P.ny = g->n[1]; P.nz = g->n[2];
    P.gxp = (P.nx + 3) / 4 * 4;
    P.tiles = (N + kTile - 1) / kTile;
    const int e = energy ? 1 : 0;
    if (ctx->occ_attr[acc][e] < 0 || ctx->occ_attr_gxp[acc][e] != P.gxp) {
        ctx->occ_attr[acc][e] = attraction_ctas_per_sm(acc, energy, P.gxp);
        ctx->occ_attr_gxp[acc][e] = P.gxp;
    }
    if (ctx->occ_rep[acc][e] < 0) ctx->occ_rep[acc][e] = repulsion_ctas_per_sm(acc, energy);
    if (ctx->occ_attr[acc][e] < 1 || ctx->occ_rep[acc][e] < 1) {
        cudaGetLastError();
        return fail(ctx, SPARKLING_E_CUDA, "pair kernels cannot be resident (occupancy 0)");
    }
    const int64_t rows = (int64_t)P.ny * P.nz;
    const int64_t nblocks = (N + kSrcBlock - 1) / kSrcBlock;
    P.spa = make_split(P.tiles, rows, (int64_t)ctx->sms * ctx->occ_attr[acc][e]);
    P.spr = make_split(P.tiles, nblocks, (int64_t)ctx->sms * ctx->occ_rep[acc][e]);
    P.o_pos = cv.take((size_t)N * sizeof(float4));
    P.o_rho = cv.take((size_t)rows * P.gxp * sizeof(float));
    P.o_coords = cv.take(((size_t)P.gxp + P.ny + P.nz) * sizeof(float));
    P.o_parta = cv.take((size_t)P.tiles * P.spa.slots * kTile * sizeof(dacc4));
    P.o_partr = cv.take((size_t)P.tiles * P.spr.slots * kTile * sizeof(dacc4));
    P.o_eblocks = cv.take((size_t)energy_blocks(N) * sizeof(double2));
    P.o_g64 = need_g64 ? cv.take((size_t)N * 3 * sizeof(double)) : 0;
    P.end = cv.off;
    return SPARKLING_OK;
}

template <typename T> T *at(sparkling_ctx *ctx, size_t off)
{
    return reinterpret_cast<T *>(static_cast<char *>(ctx->ws) + off);
}

// pack -> attraction -> repulsion -> combine (gradient) or energy reduction.
int run_pairs(sparkling_ctx *ctx, const void *K, int K_dtype, const sparkling_grid *g, int acc,
              bool energy, const PairPlan &P, void *G, int G_dtype, void *A, void *R, bool g64,
              cudaStream_t st, double scale = 1.0, const double *scale_dev = nullptr)
{
    float4 *pos = at<float4>(ctx, P.o_pos);
    float *rho = at<float>(ctx, P.o_rho);
    float *coords = at<float>(ctx, P.o_coords);
    {
        LaunchScope ls(ctx, SPARKLING_KERNEL_PACK, st);
        CK(launch_pack_positions(K, K_dtype, P.N, pos, ctx->d_status, ctx->sms, st));
        CK(launch_pack_grid(g->rho, P.nx, P.ny, P.nz, P.gxp, g->lo, g->hi, rho, coords,
                            ctx->d_status, ctx->sms, st));
        ls.done(2);
    }
    AttrArgs aa;
    aa.tgt = pos; aa.N = P.N; aa.rho = rho; aa.coords = coords;
    aa.gxp = P.gxp; aa.ny = P.ny; aa.nz = P.nz;
    aa.rows_per_stage = kStageFloats / P.gxp;
    aa.hx = (float)((g->hi - g->lo) / P.nx);
    aa.x0 = g->lo + 0.5 * ((g->hi - g->lo) / P.nx);
    aa.sp = P.spa; aa.part = at<dacc4>(ctx, P.o_parta); aa.status = ctx->d_status;
    {
        LaunchScope ls(ctx, SPARKLING_KERNEL_ATTRACTION, st);
        CK(launch_attraction(aa, acc, energy, st));
        ls.done();
    }
    RepArgs ra;
    ra.pos = pos; ra.N = P.N; ra.sp = P.spr; ra.part = at<dacc4>(ctx, P.o_partr);
    ra.status = ctx->d_status;
    {
        LaunchScope ls(ctx, SPARKLING_KERNEL_REPULSION, st);
        CK(launch_repulsion(ra, acc, energy, st));
        ls.done();
    }
    CombineArgs cb;
    cb.N = P.N; cb.part_a = aa.part; cb.part_r = ra.part; cb.spa = P.spa; cb.spr = P.spr;
    cb.G = G; cb.A = A; cb.R = R;
    cb.G64 = g64 ? at<double>(ctx, P.o_g64) : nullptr;
    cb.scale = scale;
    cb.scale_dev = scale_dev;
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
    if (acc != SPARKLING_ACC_KAHAN32 && acc != SPARKLING_ACC_FP64)
        return fail(ctx, SPARKLING_E_INVAL, "acc %d is not KAHAN32/FP64", acc);
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
    ProjArgs p;
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
        cudaFree(ctx->ws);
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
    PairPlan P;
    Carve cv;
    if ((s = plan_pairs(ctx, Nc * Ns, grid, acc, false, true, P, cv))) return s;
    ProjPlan L;
    if ((s = plan_project(ctx, K_dtype, Nc, Ns, cv, L))) return s;
    if ((s = ensure_ws(ctx, cv.off))) return s;
    if ((s = run_pairs(ctx, K, K_dtype, grid, acc, false, P, nullptr, K_dtype, nullptr, nullptr, true,
                       st)))
        return s;
    if ((s = run_project(ctx, K, K_dtype, Nc, Ns, proj, at<double>(ctx, P.o_g64), eta, L, false, st)))
        return s;
    if (proj->tol > 0) return finish_project(ctx, proj, nullptr, st);
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

SPARKLING_API int64_t sparkling_launch_count(const sparkling_ctx *ctx)
{
    return ctx ? ctx->launches : 0;
}

} // extern "C"
