// sparkling_grad_noalloc: the attraction-repulsion gradient without any
// device allocation.
//
// Some callers cannot let a library call cudaMalloc: processes whose device
// memory is handed out by their own pool or arena (a framework allocator, a
// serving runtime with a fixed memory budget), code running where a new
// allocation would synchronise the device or fail (latency-critical loops,
// some driver-level contexts), or deployments that must know every byte a
// library holds up front.  For them this entry point uses one fixed scratch
// array compiled into the library instead of a context workspace.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes
// (32 MiB).  Every GPU that loads this library holds it until the process
// exits.  Host code may not use the array's name as a device address (on the
// host it names a host-side shadow), so the first call on each device looks
// up the real device address with cudaGetSymbolAddress, with that device
// current, and caches it; kernels receive that pointer.  Because the first
// call on a device performs this lookup, make it before capturing any CUDA
// stream.
//
// All calls on a device share the one array and it keeps the previous call's
// contents.  The control block (status word and wait budget) is reset at the
// start of every call; every other byte a call reads it has written first.
// Calls whose kernels overlap on the GPU (different streams, or different
// host threads) race on the array: serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/sparkling.h"
#include "kernels.h"

using namespace sparkling;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

int noalloc_fail(int code, const char *fmt, ...);

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Device address of the scratch array on the current device (set up once per
// device, with that device current).
int scratch_for_current_device(void **out, int *sms)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return noalloc_fail(SPARKLING_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(SPARKLING_E_CUDA, "device %d outside the supported range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(SPARKLING_E_CUDA, "cudaGetSymbolAddress of the scratch array: %s",
                                cudaGetErrorString(e));
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return noalloc_fail(SPARKLING_E_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
        g_sms[dev] = n;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    *sms = g_sms[dev];
    return SPARKLING_OK;
}

// Device memory of device `dev` (the current one), or managed memory.
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged;
}

// The control block every call starts from: status clear, default wait
// budget.  Static storage, so the asynchronous copy always reads it.
const DevCtl kFreshCtl = {0, 0, kWaitCycles};

} // namespace

// Failures are reported through the thread-local message that
// sparkling_last_error(NULL) returns; api.cu owns it.
void sparkling_set_thread_error(const char *msg);

namespace {
int noalloc_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    sparkling_set_thread_error(buf);
    return code;
}
} // namespace

extern "C" SPARKLING_API int sparkling_grad_noalloc(const void *K, int K_dtype, int64_t N,
                                                    const sparkling_grid *grid, int acc, void *G,
                                                    int G_dtype, void *stream)
{
    if (!K || !G) return noalloc_fail(SPARKLING_E_INVAL, "K and G are required");
    if ((K_dtype != SPARKLING_F32 && K_dtype != SPARKLING_F64) ||
        (G_dtype != SPARKLING_F32 && G_dtype != SPARKLING_F64))
        return noalloc_fail(SPARKLING_E_INVAL, "K_dtype and G_dtype must be SPARKLING_F32/F64");
    if (N < 2 || N > ((int64_t)1 << 31) - kTile)
        return noalloc_fail(SPARKLING_E_INVAL, "N = %lld out of range", (long long)N);
    if (acc != SPARKLING_ACC_KAHAN32 && acc != SPARKLING_ACC_FP64)
        return noalloc_fail(SPARKLING_E_INVAL, "acc %d is not KAHAN32/FP64", acc);
    if (!grid || !grid->rho) return noalloc_fail(SPARKLING_E_INVAL, "grid and grid->rho are required");
    for (int a = 0; a < 3; ++a)
        if (grid->n[a] < 1) return noalloc_fail(SPARKLING_E_INVAL, "grid n[%d] < 1", a);
    if (grid->n[0] > kMaxNx) return noalloc_fail(SPARKLING_E_INVAL, "grid nx exceeds %d", kMaxNx);
    if (!(std::isfinite(grid->lo) && std::isfinite(grid->hi) && grid->hi > grid->lo))
        return noalloc_fail(SPARKLING_E_INVAL, "grid needs finite lo < hi");

    // Scratch layout: status word, packed samples, padded density rows,
    // coordinate tables, attraction and repulsion partial sums.
    const int nx = grid->n[0], ny = grid->n[1], nz = grid->n[2];
    const int gxp = (nx + 3) / 4 * 4;
    const int64_t rows = (int64_t)ny * nz;
    const int64_t tiles = (N + kTile - 1) / kTile;
    const int64_t nblocks = (N + kSrcBlock - 1) / kSrcBlock;
    const size_t fixed = up256(256) + up256((size_t)N * sizeof(float4)) +
                         up256((size_t)rows * gxp * sizeof(float)) +
                         up256(((size_t)gxp + ny + nz) * sizeof(float));
    auto need = [&](const Split &a, const Split &r) {
        return fixed + up256((size_t)tiles * a.slots * kTile * sizeof(dacc4)) +
               up256((size_t)tiles * r.slots * kTile * sizeof(dacc4));
    };
    // Smallest possible footprint: one CTA per tile (two partial slots).
    const Split amin = make_split(tiles, rows, tiles), rmin = make_split(tiles, nblocks, tiles);
    if (need(amin, rmin) > kNoAllocScratchBytes)
        return noalloc_fail(SPARKLING_E_INVAL,
                            "problem needs %zu bytes of scratch (N = %lld, grid %dx%dx%d) but the "
                            "fixed scratch array holds %zu bytes; use sparkling_grad",
                            need(amin, rmin), (long long)N, nx, ny, nz, kNoAllocScratchBytes);

    int s;
    void *base = nullptr;
    int sms = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((s = scratch_for_current_device(&base, &sms))) return s;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_fail(SPARKLING_E_CUDA, "cudaGetDevice failed");
    if (!on_device(K, dev) || !on_device(G, dev) || !on_device(grid->rho, dev))
        return noalloc_fail(SPARKLING_E_INVAL,
                            "K, G and grid->rho must be device memory of the current device (%d)", dev);
    const int occ_a = attraction_ctas_per_sm(acc, false, kAttrDefault);
    const int occ_r = repulsion_ctas_per_sm(acc, false, kRepDefault);
    if (occ_a < 1 || occ_r < 1) {
        cudaGetLastError();
        return noalloc_fail(SPARKLING_E_CUDA, "pair kernels cannot be resident");
    }
    // One full wave when it fits, otherwise fewer CTAs (fewer partial slots).
    int64_t ca = (int64_t)sms * occ_a, cr = (int64_t)sms * occ_r;
    Split spa = make_split(tiles, rows, ca), spr = make_split(tiles, nblocks, cr);
    while (need(spa, spr) > kNoAllocScratchBytes && (ca > tiles || cr > tiles)) {
        ca = ca / 2 > tiles ? ca / 2 : tiles;
        cr = cr / 2 > tiles ? cr / 2 : tiles;
        spa = make_split(tiles, rows, ca);
        spr = make_split(tiles, nblocks, cr);
    }

    char *p = static_cast<char *>(base);
    int *status = reinterpret_cast<int *>(p);
    p += up256(256);
    float4 *pos = reinterpret_cast<float4 *>(p);
    p += up256((size_t)N * sizeof(float4));
    float *rho = reinterpret_cast<float *>(p);
    p += up256((size_t)rows * gxp * sizeof(float));
    float *coords = reinterpret_cast<float *>(p);
    p += up256(((size_t)gxp + ny + nz) * sizeof(float));
    dacc4 *part_a = reinterpret_cast<dacc4 *>(p);
    p += up256((size_t)tiles * spa.slots * kTile * sizeof(dacc4));
    dacc4 *part_r = reinterpret_cast<dacc4 *>(p);

    cudaError_t e;
#define NA_CK(call)                                                                               \
    do {                                                                                          \
        if ((e = (call)) != cudaSuccess)                                                          \
            return noalloc_fail(SPARKLING_E_CUDA, "%s: %s", #call, cudaGetErrorString(e));        \
    } while (0)
    NA_CK(cudaMemcpyAsync(status, &kFreshCtl, sizeof(DevCtl), cudaMemcpyHostToDevice, st));
    NA_CK(launch_pack_positions(K, K_dtype, N, pos, status, sms, st));
    NA_CK(launch_pack_grid(grid->rho, nx, ny, nz, gxp, grid->lo, grid->hi, rho, coords, status, sms,
                           st));
    AttrArgs aa{};
    aa.tgt = pos; aa.N = N; aa.rho = rho; aa.coords = coords;
    aa.gxp = gxp; aa.ny = ny; aa.nz = nz; aa.rows_per_stage = kStageFloats / gxp;
    aa.hx = (float)((grid->hi - grid->lo) / nx);
    aa.x0 = grid->lo + 0.5 * ((grid->hi - grid->lo) / nx);
    aa.sp = spa; aa.part = part_a; aa.status = status; aa.eps2 = kEps2;
    NA_CK(launch_attraction(aa, acc, false, kAttrDefault, st));
    RepArgs ra{};
    ra.pos = pos; ra.N = N; ra.sp = spr; ra.part = part_r; ra.status = status; ra.eps2 = kEps2;
    NA_CK(launch_repulsion(ra, acc, false, kRepDefault, st));
    CombineArgs cb{};
    cb.N = N; cb.part_a = part_a; cb.part_r = part_r; cb.spa = spa; cb.spr = spr;
    cb.G = G; cb.A = nullptr; cb.R = nullptr; cb.G64 = nullptr;
    cb.scale = 1.0; cb.scale_dev = nullptr; cb.energy_blocks = nullptr; cb.racc = nullptr; cb.a_direct = nullptr;
    cb.eps = 0.0;
    NA_CK(launch_combine(cb, G_dtype, sms, st));
    int h = 0;
    NA_CK(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
    if (h & kDevTimeout)
        return noalloc_fail(SPARKLING_E_TIMEOUT, "a bounded device wait ran out; G is incomplete");
    if (h & kDevNonFinite)
        return noalloc_fail(SPARKLING_E_NONFINITE, "non-finite sample or density value, or negative density");
    return SPARKLING_OK;
}
