// Persistent engine: one launch of a whole projected-gradient step (eq.
// proj_grad_descent, the inner loop of Algorithm 1) for a batch of
// independent trajectories of uneven size.
//
// The host builds a work list (api.cu): for every trajectory and every tile
// of 1024 targets, attraction items (a run of grid rows), then one
// projection item per shot.  The repulsion of every trajectory is summed
// with each unordered pair once, into exact fixed-point totals per sample
// (EngineArgs::racc): in the one-launch shape by symmetric repulsion items
// of the same work list (a target tile against a run of source tiles),
// otherwise by the batched symmetric kernel before the launch; contexts
// where that kernel cannot be resident get directed repulsion items (a run
// of source blocks) interleaved with the attraction items instead.  Every
// CTA of a single wave pulls the next item from a global counter -- in the
// one-launch shape from the counter of its role's part of the list (one CTA
// in three per SM takes symmetric items first, the others attraction items
// first: see next_item), so each SM runs SFU-bound and FP32-bound items side
// by side.
//
// A pair item writes the FP64 partial sums of its tile into its own slot and
// then bumps its trajectory's completion counter.  A projection item waits
// (bounded) until its trajectory's counter reaches the number of pair items,
// adds the slots of each sample in a fixed order (A - R/N, R from racc when
// set), steps k = K - eta G and projects the shot in place.  Because every
// item owns its slot and the slots are added in a fixed order, results do
// not depend on which CTA ran which item.
//
// Items are dispensed in list order (role dispatch: part by part) and a
// projection item is dispensed only after all pair items of its trajectory,
// so when a CTA waits on a trajectory every item it waits for is already
// running on another CTA: the wait always ends.
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.h"
#include "pair_dev.cuh"
#include "project_dev.cuh"
#include "ptx.cuh"
#include "sym_dev.cuh"

namespace sparkling {

namespace {

constexpr size_t kUnionBytes = (size_t)kAccBytes + (size_t)kStages * kStageFloats * sizeof(float);
constexpr size_t kHeadBytes = 128;   // mbarriers + item broadcast

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Every thread's partial writes are made visible device-wide, then one
// thread counts the item as done.
__device__ __forceinline__ void mark_done(unsigned int *done)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        atomicAdd(done, 1u);
}

// Bounded wait until *done >= target; false (and the timeout status bit) if
// it does not happen within `scale` times the context's wait budget: the
// items waited for may have started just before, and one item can take a
// large part of a copy wait's budget (an attraction item over a whole 256^3
// density: ~3.5e9 cycles of one CTA), so the host sizes the scale from the
// work list's largest item.
__device__ bool wait_done(const unsigned int *done, unsigned int target, int scale, int *status,
                          int *flag)
{
    if (threadIdx.x == 0) {
        int ok = 1;
        if (ld_acquire(done) < target) {
            const long long budget = scale * wait_budget(status);
            const long long t0 = clock64();
            while (ld_acquire(done) < target) {
                if (clock64() - t0 > budget) {
                    atomicOr(status, kDevTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(200);
            }
        }
        *flag = ok;
    }
    __syncthreads();
    const bool ok = *flag != 0;
    __syncthreads();
    __threadfence();
    return ok;
}

__device__ __forceinline__ AttrArgs attr_args(const EngineTraj &t, const EngineArgs &e)
{
    AttrArgs a;
    a.tgt = e.pos + t.off;
    a.N = t.N;
    a.rho = t.rho;
    a.coords = t.coords;
    a.gxp = t.gxp; a.ny = t.ny; a.nz = t.nz;
    a.rows_per_stage = t.rows_per_stage;
    a.x0 = t.x0;
    a.hx = t.hx;
    a.sp.units = 0; a.sp.per_tile = 0; a.sp.ctas = 1;
    a.sp.slots = t.slots;
    a.part = e.part + t.part_off;
    a.eps2 = e.eps2;
    a.status = e.status;
    return a;
}

__device__ __forceinline__ RepArgs rep_args(const EngineTraj &t, const EngineArgs &e)
{
    RepArgs r;
    r.pos = e.pos + t.off;
    r.N = t.N;
    r.sp.units = 0; r.sp.per_tile = 0; r.sp.ctas = 1;
    r.sp.slots = t.slots;
    r.part = e.part + t.part_off;
    r.eps2 = e.eps2;
    r.status = e.status;
    return r;
}

// NT threads per CTA: 256 (4 targets per thread, repulsion unroll 4, three
// CTAs per SM) or 512 (2 targets per thread, unroll 2, two CTAs per SM).
// A projection item (one shot), out of line so that its registers do not
// crowd the attraction loop of the kernel: wait (bounded) for the
// trajectory's pair items, form k = K - eta G from the slots and the
// symmetric repulsion totals, and project the shot in place.
template <typename KT>
__device__ __noinline__ bool project_item(const EngineArgs &e, const EngineItem &item,
                                          const EngineTraj &tr, unsigned char *region, int *bcast)
{
    if (!wait_done(e.done + item.traj, (unsigned int)tr.n_pair_items, e.wait_scale, e.status,
                   bcast + 1))
        return false;
    const int Ns = tr.Ns;
    double *base = e.proj_in_smem ? reinterpret_cast<double *>(region)
                                  : e.gstate + (size_t)blockIdx.x * 18 * (size_t)Ns;
    const Arrays A = carve(base, Ns);
    ShotParams sp;
    sp.Ns = Ns;
    sp.alpha = tr.alpha; sp.beta = tr.beta; sp.box = tr.box;
    sp.tol = 0.0; sp.margin = 0.0;
    for (int c = 0; c < 3; ++c) sp.pin[c] = tr.pin[c];
    sp.pin_index = tr.pin_index; sp.n_iter = tr.n_iter; sp.check_every = 0;
    sp.viol = nullptr; sp.notconv = nullptr;
    const int64_t first = (int64_t)item.tile * Ns;          // local sample index
    KT *K = static_cast<KT *>(e.K) + 3 * (tr.off + first);
    const dacc4 *part = e.part + tr.part_off;
    const double invN = 1.0 / (double)tr.N;
    const double eta = tr.eta;
    const int slots = tr.slots, ach = tr.a_chunks;
    auto loadk = [&](int m, double *kv) {
        const int64_t i = first + m;
        const int64_t tile = i / kTile, l = i - tile * kTile;
        const dacc4 *p = part + tile * slots * kTile + l;
        double g[3] = {0.0, 0.0, 0.0}, r[3] = {0.0, 0.0, 0.0};
        for (int s = 0; s < slots; ++s) {
            const double2 xy = __ldcg(reinterpret_cast<const double2 *>(p + s * kTile));
            const double zz = __ldcg(reinterpret_cast<const double *>(p + s * kTile) + 2);
            if (s < ach) { g[0] += xy.x; g[1] += xy.y; g[2] += zz; }
            else { r[0] += xy.x; r[1] += xy.y; r[2] += zz; }
        }
        if (e.racc) {   // symmetric repulsion totals (fixed point), complete once the pair items are
            const unsigned long long *q = e.racc + 3 * (tr.off + i);
            for (int c = 0; c < 3; ++c) r[c] = (double)(long long)__ldcg(q + c) / kFixScale;
        }
        for (int c = 0; c < 3; ++c)
            kv[c] = (double)K[3 * m + c] - eta * (g[c] - r[c] * invN);
    };
    if (sizeof(KT) == 4 && e.proj_mixed)
        project_shot_mixed<KT>(carve_f(reinterpret_cast<float *>(base), Ns), K, sp, loadk);
    else
        project_shot<KT>(A, K, sp, loadk);
    // The projection state may share memory with the stage buffers: order its
    // ordinary stores before later bulk copies (async proxy).
    fence_proxy_async_smem();
    __syncthreads();
    return true;
}

// A symmetric repulsion item: the tile pairs (I, J), J in [J0, J1), of one
// trajectory (I <= J0), the J tiles streamed through the stage buffers by
// bulk copies.  Each pair's source sums (jacc, shared) and target sums are
// added to the fixed-point totals e.racc with 64-bit atomics -- the
// integers of the standalone kernel, so the totals are the same bit for bit.
template <int NT>
__device__ bool sym_item_run(const EngineArgs &e, const EngineTraj &tr, int64_t I, int64_t J0,
                             int64_t J1, float4 *stage, uint64_t *bars, float *jacc,
                             uint32_t &consumed)
{
    constexpr int T = kTile / NT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float4 *pos = e.pos + tr.off;
    unsigned long long *acc = e.racc + 3 * tr.off;
    const int64_t N = tr.N;
    const uint32_t n = (uint32_t)(J1 - J0);
    auto count_of = [&](int64_t J) {
        const int64_t rem = N - J * kTile;
        return rem < kTile ? (int)rem : kTile;
    };
    auto issue = [&](uint32_t s) {
        const uint32_t g = consumed + s;
        const int64_t J = J0 + s;
        bulk_load(stage + (g % kStages) * kTile, pos + J * kTile,
                  (uint32_t)(count_of(J) * sizeof(float4)), &bars[g % kStages]);
    };
    if (tid == 0) {
        fence_proxy_async_smem();     // the buffers last held generic-proxy data
        for (uint32_t s = 0; s < n && s < (uint32_t)kStages; ++s) issue(s);
    }
    // the thread's targets l = warp*32T + t*32 + lane of tile I
    float tx[T], ty[T], tz[T], tm[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t i = I * kTile + warp * 32 * T + t * 32 + lane;
        const bool ok = i < N;
        const float4 p = ok ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        tx[t] = p.x; ty[t] = p.y; tz[t] = p.z; tm[t] = ok ? 1.f : 0.f;
    }
    for (uint32_t s = 0; s < n; ++s) {
        const uint32_t g = consumed + s;
        const bool ok = mbar_wait_bounded(&bars[g % kStages], (g / kStages) & 1, e.status);
        if (__syncthreads_or(!ok)) {
            const uint32_t left = n - s;
            drain_stages(bars, g, left < (uint32_t)kStages ? left : (uint32_t)kStages, e.status);
            return false;
        }
        const float4 *src = stage + (g % kStages) * kTile;
        const int64_t J = J0 + s;
        const int jvalid = count_of(J);
        float ai[T][3];
#pragma unroll
        for (int t = 0; t < T; ++t) ai[t][0] = ai[t][1] = ai[t][2] = 0.f;
        if (J == I) {
            diag_item<false, NT>(src, jvalid, tx, ty, tz, e.eps2, ai);
        } else {
            for (int q = tid; q < 3 * kTile; q += NT) jacc[q] = 0.f;
            __syncthreads();
            if (jvalid < kTile)
                sym_item_sp<false, true, NT>(src, jvalid, tx, ty, tz, tm, e.eps2, ai, jacc);
            else
                sym_item_sp<false, false, NT>(src, jvalid, tx, ty, tz, tm, e.eps2, ai, jacc);
            for (int l = tid; l < jvalid; l += NT)
#pragma unroll
                for (int v = 0; v < 3; ++v)
                    add_fix(&acc[(J * kTile + l) * 3 + v], to_fix(jacc[v * kTile + l]));
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int64_t i = I * kTile + warp * 32 * T + t * 32 + lane;
            if (i < N)
#pragma unroll
                for (int v = 0; v < 3; ++v) add_fix(&acc[i * 3 + v], to_fix(ai[t][v]));
        }
        __syncthreads();   // this stage and jacc are free again
        if (tid == 0 && s + kStages < n) {
            fence_proxy_async_smem();
            issue(s + kStages);
        }
    }
    consumed += n;
    return true;
}

// Index of the next item for this CTA (thread 0), n_items when none is left.
// Role dispatch: the next projection item if its trajectory's pair items
// are all done (claimed only then, so it never waits), else the CTA's own
// pair part, then the other pair part, then any projection item -- taken
// only once every pair item has been dispensed to a running CTA, so its
// wait ends.
template <bool SYM>
__device__ __forceinline__ int next_item(const EngineArgs &e, int role)
{
    if (!SYM || !e.roles) return (int)atomicAdd(e.queue, 1u);
    const int base_p = e.n_attr + e.n_sym;
    const unsigned int n_p = (unsigned int)(e.n_items - base_p);
    const unsigned int p = *(volatile unsigned int *)(e.queue + 2);
    if (p < n_p) {
        const int t = e.items[base_p + p].traj;
        if (ld_acquire(e.done + t) >= (unsigned int)e.traj[t].n_pair_items &&
            atomicCAS(e.queue + 2, p, p + 1) == p)
            return base_p + (int)p;
    }
    for (int k = 0; k < 2; ++k) {
        const int q = k == 0 ? role : 1 - role;
        const unsigned int n = (unsigned int)(q == 0 ? e.n_attr : e.n_sym);
        if (*(volatile unsigned int *)(e.queue + q) >= n) continue;
        const unsigned int i = atomicAdd(e.queue + q, 1u);
        if (i < n) return (q == 0 ? 0 : e.n_attr) + (int)i;
    }
    const unsigned int i = atomicAdd(e.queue + 2, 1u);
    return i < n_p ? base_p + (int)i : e.n_items;
}

// REP: the work list may hold directed repulsion items (only when the
// batched symmetric kernel cannot run); without them the kernel carries no
// repulsion code.  SYM: the one-launch shape, whose work list holds the
// symmetric repulsion items.
template <int ACC, typename KT, int NT, bool REP, bool SYM>
__global__ void __launch_bounds__(NT, NT >= 512 ? 2 : 3) engine_kernel(const EngineArgs e)
{
    extern __shared__ __align__(128) unsigned char esm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(esm);
    int *bcast = reinterpret_cast<int *>(esm + 64);
    unsigned char *region = esm + kHeadBytes;
    void *accbase = region;
    float *stage = reinterpret_cast<float *>(region + kAccBytes);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s)
            mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t consumed = 0;
    int role = 0;   // role dispatch: 0 attraction items first, 1 symmetric items first
    if (SYM && e.roles) {
        if (threadIdx.x == 0) {
            unsigned int smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            bcast[2] = atomicAdd(e.sm_slots + (smid & (kSmSlots - 1)), 1u) % 3u == 2u ? 1 : 0;
        }
        __syncthreads();
        role = bcast[2];
    }
    for (;;) {
        if (threadIdx.x == 0)
            bcast[0] = next_item<SYM>(e, role);
        __syncthreads();
        const int idx = bcast[0];
        __syncthreads();
        if (idx >= e.n_items)
            break;
        const EngineItem item = e.items[idx];
        const EngineTraj &tr = e.traj[item.traj];
        if (item.kind == kItemAttraction) {
            const AttrArgs a = attr_args(tr, e);
            if (!attraction_segment<ACC, false, NT>(a, item.tile, item.u0, item.u1, item.slot, stage,
                                                bars, accbase, consumed))
                return;
            mark_done(e.done + item.traj);
        } else if (SYM && item.kind == kItemSym) {
            if (!sym_item_run<NT>(e, tr, item.tile, item.u0, item.u1,
                                  reinterpret_cast<float4 *>(stage), bars,
                                  static_cast<float *>(accbase), consumed))
                return;
            mark_done(e.done + item.traj);
        } else if (REP && item.kind == kItemRepulsion) {
            const RepArgs r = rep_args(tr, e);
            if (!repulsion_segment<ACC, false, NT, (NT >= 512 ? 2 : 4)>(r, item.tile, item.u0, item.u1, item.slot,
                                               reinterpret_cast<float4 *>(stage), bars, accbase,
                                               consumed))
                return;
            mark_done(e.done + item.traj);
        } else {
            if (!project_item<KT>(e, item, tr, region, bcast))
                return;
        }
    }
}

template <int ACC, typename KT, int NT, bool REP, bool SYM>
void *engine_fn() { return reinterpret_cast<void *>(engine_kernel<ACC, KT, NT, REP, SYM>); }

template <int NT, bool REP, bool SYM>
void *pick_engine_nt(int acc, int dtype)
{
    if (acc == 0)
        return dtype == 0 ? engine_fn<0, float, NT, REP, SYM>() : engine_fn<0, double, NT, REP, SYM>();
    return dtype == 0 ? engine_fn<1, float, NT, REP, SYM>() : engine_fn<1, double, NT, REP, SYM>();
}

// rep: directed repulsion items (not in the one-launch shape, which has the
// symmetric items instead)
void *pick_engine(int acc, int dtype, int variant, bool rep)
{
    if (variant == kEngineOneLaunch) return pick_engine_nt<128, false, true>(acc, dtype);
    if (rep)
        return variant == 1 ? pick_engine_nt<512, true, false>(acc, dtype)
                            : pick_engine_nt<256, true, false>(acc, dtype);
    return variant == 1 ? pick_engine_nt<512, false, false>(acc, dtype)
                        : pick_engine_nt<256, false, false>(acc, dtype);
}

} // namespace

size_t engine_smem_bytes() { return kHeadBytes + kUnionBytes; }

size_t engine_proj_smem_limit() { return kUnionBytes; }

int engine_variant_threads(int v) { return v == kEngineOneLaunch ? 128 : v == 1 ? 512 : 256; }

int engine_ctas_per_sm(int acc, int dtype, int variant)
{
    int best = 1 << 30;
    for (int rep = 0; rep < (variant == kEngineOneLaunch ? 1 : 2); ++rep) {
        void *fn = pick_engine(acc, dtype, variant, rep != 0);
        const size_t smem = engine_smem_bytes();
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, engine_variant_threads(variant),
                                                          smem) != cudaSuccess)
            return 0;
        best = n < best ? n : best;
    }
    return best;
}

cudaError_t launch_engine(const EngineArgs &e, int acc, int dtype, int variant, int ctas,
                          cudaStream_t st)
{
    void *fn = pick_engine(acc, dtype, variant, e.racc == nullptr);
    void *args[] = {const_cast<EngineArgs *>(&e)};
    return cudaLaunchKernel(fn, dim3((unsigned)ctas), dim3(engine_variant_threads(variant)), args,
                            engine_smem_bytes(), st);
}

} // namespace sparkling
