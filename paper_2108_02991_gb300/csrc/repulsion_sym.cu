// Symmetric repulsion: R_i = (1/N) sum_j (k_i - k_j)/|k_i - k_j| (paper
// eq. Fr_grad with H' = 1) with every unordered pair evaluated once.  The
// pair term is odd in (i, j), so the term computed for (i, j) is added to
// sample i and subtracted from sample j: half the reciprocal square roots
// and ~35% fewer instructions per directed pair than the directed kernel.
//
// Work: the upper triangle of tile pairs (I, J), I <= J, tiles of 1024
// samples, split evenly over one wave of persistent CTAs (contiguous runs of
// a row share the target tile I).  A CTA of NT threads (256 or 128) holds the
// 1024 targets of tile I, T = 1024/NT per lane (4 or 8): warp w holds 32*T
// of them and, in round r, the 32*S sources of chunk (w + r) mod
// (1024 / 32S) of tile J (S per lane, the tile staged by a TMA bulk copy).  The sources and their accumulators rotate one lane per step
// through the 32 lanes, so after 32 steps every (target, source) pair of the
// two chunks has met once and each source is back home; its accumulator is
// then added to a shared-memory j-accumulator, which no other warp touches
// in that round.  A diagonal pair (I, I) is evaluated directed (targets
// only).  The pair arithmetic is paired FP32 (f32x2): either two targets
// share a 64-bit register (sym_item, S = 2 or 4) or a lane's two sources do
// (sym_item_sp, S = 2).
//
// Totals are kept as fixed-point integers (x * 2^32 in int64) and added with
// 64-bit atomics: integer addition is exact and order-independent, so the
// result does not depend on the schedule.  The per-item sums converted to
// fixed point are FP32 sums of <= 1024 unit-vector components.
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.h"
#include "ptx.cuh"
#include "sym_dev.cuh"

namespace sparkling {

namespace {

constexpr int kSymStages = 2;                  // J tiles in flight
// NT threads per CTA hold one tile of targets, T = kTile / NT per lane.
// S sources per lane: a chunk is 32*S sources, a tile kTile/(32*S) chunks;
// in round r warp w owns chunk (w + r) mod chunks.

// Shared memory: mbarriers | J-tile stages | FP32 j-accumulator [NV][1024] |
// per-thread int64 i-accumulators [T*NV][NT] (T * NT = kTile).
constexpr size_t kSymHead = 64;
constexpr size_t kSymStageBytes = (size_t)kTile * sizeof(float4);
constexpr size_t kSymJaccBytes = 3 * kTile * sizeof(float);
constexpr size_t kSymIaccBytes = (size_t)kTile * 3 * sizeof(long long);

// Resident CTAs asked of the compiler: 2 of 256 threads (<= 128 registers),
// 3 of 128 threads (<= 168 registers, 8 targets per lane).
constexpr int sym_min_ctas(int nt) { return nt >= 256 ? 2 : 3; }

// REG: the regularisation eps^2 is a kernel argument; without it the
// zero-distance guard kEps2 is a compile-time constant of the pair loop.
// BATCHED: the units of a.B trajectories (a.traj), else of one.
// SP: the source-paired item (two sources per lane), else the target-paired
// item with S sources per lane.  NT: threads per CTA (T = 1024/NT targets per
// lane).
template <bool ENERGY, int S, bool SP, bool REG, bool BATCHED, int NT>
__global__ void __launch_bounds__(NT, sym_min_ctas(NT)) repulsion_sym_kernel(const SymArgs a)
{
    const float eps2 = REG ? a.eps2 : kEps2;
    constexpr int T = kTile / NT;
    constexpr int kTargetsPerWarp = 32 * T;
    constexpr int NV = ENERGY ? 1 : 3;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float4 *stage = reinterpret_cast<float4 *>(smem + kSymHead);
    float *jacc = reinterpret_cast<float *>(smem + kSymHead + kSymStages * kSymStageBytes);
    long long *iacc = reinterpret_cast<long long *>(smem + kSymHead + kSymStages * kSymStageBytes +
                                                    kSymJaccBytes);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // Units: the tile pairs of one triangle, or of B triangles one after the
    // other (batched: trajectory b owns units [unit0_b, unit0_{b+1})).
    const int64_t U = BATCHED ? a.units : tri_count(a.tiles);
    const int64_t u0 = U * blockIdx.x / a.ctas, u1 = U * (blockIdx.x + 1) / a.ctas;
    if (u0 >= u1) return;
    auto tr_off = [&](int b) -> int64_t { return BATCHED ? a.traj[b].off : 0; };
    auto tr_n = [&](int b) -> int64_t { return BATCHED ? a.traj[b].N : a.N; };
    auto tr_tiles = [&](int b) -> int64_t { return BATCHED ? a.traj[b].tiles : a.tiles; };
    if (tid == 0) {
        for (int s = 0; s < kSymStages; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto count_of = [&](int b, int64_t J) {
        const int64_t rem = tr_n(b) - J * kTile;
        return rem < kTile ? (int)rem : kTile;
    };
    // next unit; past the last tile pair of trajectory b go to b + 1 (the
    // prefetch cursor may run past the last unit: it then stops at b = B - 1)
    auto advance = [&](int &b, int64_t &I, int64_t &J) {
        if (++J == tr_tiles(b)) {
            ++I;
            J = I;
            if (BATCHED && I == tr_tiles(b) && b + 1 < a.B) { ++b; I = 0; J = 0; }
        }
    };
    auto issue = [&](uint32_t g, int b, int64_t J) {
        bulk_load(stage + (g % kSymStages) * kTile, a.pos + tr_off(b) + J * kTile,
                  (uint32_t)(count_of(b, J) * sizeof(float4)), &bars[g % kSymStages]);
    };
    const uint32_t n = (uint32_t)(u1 - u0);
    int b = 0;
    if (BATCHED) {                       // trajectory of unit u0
        int lo = 0, hi = a.B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.traj[mid].unit0 <= u0) lo = mid;
            else hi = mid - 1;
        }
        b = lo;
    }
    int64_t I, J, qI, qJ;
    tri_pair(u0 - (BATCHED ? a.traj[b].unit0 : 0), tr_tiles(b), I, J);
    int qb = b;
    qI = I; qJ = J;                      // cursor of the next tile to prefetch
    for (uint32_t g = 0; g < n && g < (uint32_t)kSymStages; ++g) {
        if (tid == 0) issue(g, qb, qJ);
        advance(qb, qI, qJ);
    }
    int curB = -1;
    int64_t curI = -1;
    // the thread's targets of tile curI: l = warp*32T + t*32 + lane
    auto flush_i = [&]() {
        const int64_t nb = tr_n(curB), ob = tr_off(curB);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int64_t i = curI * kTile + warp * kTargetsPerWarp + t * 32 + lane;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                long long &x = iacc[(t * NV + v) * NT + tid];
                if (i < nb) add_fix(&a.acc[(ob + i) * NV + v], x);
                x = 0;
            }
        }
    };
    for (uint32_t g = 0; g < n; ++g) {
        if (I != curI || b != curB) {
            if (curI >= 0) flush_i();
            curI = I;
            curB = b;
#pragma unroll
            for (int t = 0; t < T; ++t)
#pragma unroll
                for (int v = 0; v < NV; ++v) iacc[(t * NV + v) * NT + tid] = 0;
        }
        // The targets are read again for every item (from L2): nothing but
        // the loop state stays in registers between items.
        float tx[T], ty[T], tz[T], tm[T];
        {
            const int64_t nb = tr_n(b), ob = tr_off(b);
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const int64_t i = I * kTile + warp * kTargetsPerWarp + t * 32 + lane;
                const bool ok = i < nb;
                const float4 p = ok ? a.pos[ob + i] : make_float4(0.f, 0.f, 0.f, 0.f);
                tx[t] = p.x; ty[t] = p.y; tz[t] = p.z; tm[t] = ok ? 1.f : 0.f;
            }
        }
        const bool ok = mbar_wait_bounded(&bars[g % kSymStages], (g / kSymStages) & 1, a.status);
        if (__syncthreads_or(!ok)) {
            if (tid == 0)
                for (uint32_t h = g; h < n && h < g + kSymStages; ++h)
                    mbar_wait_drain(&bars[h % kSymStages], (h / kSymStages) & 1, a.status);
            __syncthreads();
            return;
        }
        const float4 *src = stage + (g % kSymStages) * kTile;
        const int jvalid = count_of(b, J);
        float ai[T][3];
#pragma unroll
        for (int t = 0; t < T; ++t) ai[t][0] = ai[t][1] = ai[t][2] = 0.f;
        if (I == J) {
            diag_item<ENERGY, NT>(src, jvalid, tx, ty, tz, eps2, ai);
        } else {
            for (int e = tid; e < NV * kTile; e += NT) jacc[e] = 0.f;
            __syncthreads();
            if (SP) {
                if (jvalid < kTile)
                    sym_item_sp<ENERGY, true, NT>(src, jvalid, tx, ty, tz, tm, eps2, ai, jacc);
                else
                    sym_item_sp<ENERGY, false, NT>(src, jvalid, tx, ty, tz, tm, eps2, ai, jacc);
            } else {
                if (jvalid < kTile)
                    sym_item<ENERGY, true, S, NT>(src, jvalid, tx, ty, tz, tm, eps2, ai, jacc);
                else
                    sym_item<ENERGY, false, S, NT>(src, jvalid, tx, ty, tz, tm, eps2, ai, jacc);
            }
            for (int l = tid; l < jvalid; l += NT)
#pragma unroll
                for (int v = 0; v < NV; ++v)
                    add_fix(&a.acc[(tr_off(b) + J * kTile + l) * NV + v], to_fix(jacc[v * kTile + l]));
        }
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int v = 0; v < NV; ++v) iacc[(t * NV + v) * NT + tid] += to_fix(ai[t][v]);
        __syncthreads();   // stage g consumed, jacc flushed
        if (g + kSymStages < n) {
            if (tid == 0) {
                fence_proxy_async_smem();
                issue(g + kSymStages, qb, qJ);
            }
            advance(qb, qI, qJ);
        }
        advance(b, I, J);
    }
    flush_i();
}

template <bool E, bool REG, bool BATCHED>
void *sym_fn_reg(int variant)
{
    if (variant == 1) return reinterpret_cast<void *>(repulsion_sym_kernel<E, 4, false, REG, BATCHED, 256>);
    if (variant == 2) return reinterpret_cast<void *>(repulsion_sym_kernel<E, 2, true, REG, BATCHED, 256>);
    if (variant == 3) return reinterpret_cast<void *>(repulsion_sym_kernel<E, 2, true, REG, BATCHED, 128>);
    return reinterpret_cast<void *>(repulsion_sym_kernel<E, 2, false, REG, BATCHED, 256>);
}

template <bool E>
void *sym_fn(int variant, bool reg = true, bool batched = false)
{
    if (batched) return reg ? sym_fn_reg<E, true, true>(variant) : sym_fn_reg<E, false, true>(variant);
    return reg ? sym_fn_reg<E, true, false>(variant) : sym_fn_reg<E, false, false>(variant);
}

} // namespace

int sym_variant_sources(int v) { return v == 1 ? 4 : 2; }
bool sym_variant_source_paired(int v) { return v >= 2; }
int sym_variant_threads(int v) { return v == 3 ? 128 : 256; }

size_t repulsion_sym_smem_bytes()
{
    return kSymHead + kSymStages * kSymStageBytes + kSymJaccBytes + kSymIaccBytes;
}

int repulsion_sym_ctas_per_sm(bool energy, int variant)
{
    // the instances (eps^2 argument or constant, one trajectory or a batch)
    // take about the same resources; the smallest occupancy sizes the grid
    int best = 1 << 30;
    for (int k = 0; k < 4; ++k) {
        const bool reg = (k & 1) != 0, batched = (k & 2) != 0;
        void *fn = energy ? sym_fn<true>(variant, reg, batched) : sym_fn<false>(variant, reg, batched);
        const size_t smem = repulsion_sym_smem_bytes();
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, sym_variant_threads(variant), smem) !=
            cudaSuccess)
            return 0;
        best = n < best ? n : best;
    }
    return best;
}

cudaError_t launch_repulsion_sym(const SymArgs &a, bool energy, int variant, cudaStream_t st)
{
    const bool reg = a.eps2 > kEps2, batched = a.traj != nullptr;
    void *fn = energy ? sym_fn<true>(variant, reg, batched) : sym_fn<false>(variant, reg, batched);
    void *args[] = {const_cast<SymArgs *>(&a)};
    return cudaLaunchKernel(fn, dim3((unsigned)a.ctas), dim3(sym_variant_threads(variant)), args,
                            repulsion_sym_smem_bytes(), st);
}

} // namespace sparkling
