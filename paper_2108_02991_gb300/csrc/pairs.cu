// Direct attraction and repulsion sums of full-3D SPARKLING on sm_103a.
//
// For every sample i (paper Sec. II-C, eqs. attraction_derivative_basic and
// Fr_grad with H = |.|_2, the attraction summed directly over the density
// grid instead of the paper's FFT + trilinear interpolation):
//   A_i = sum_q rho_q (k_i - x_q) / |k_i - x_q|
//   R_i = (1/N) sum_j (k_i - k_j) / |k_i - k_j|
// and, in energy mode, sum_q rho_q |k_i - x_q| and sum_j |k_i - k_j|.
//
// Design (FP32-issue / SFU bound, not memory bound):
// - a CTA holds kTile = 1024 targets in registers (4 per thread);
// - sources stream through shared memory in 16 KB stages filled by 1-D TMA
//   bulk copies (cp.async.bulk + mbarrier), three stages deep;
// - the attraction exploits the Cartesian grid: along a grid row dy, dz are
//   constant, so a pair costs dx = kx - x_q, r2 = fma(dx, dx, dy^2+dz^2+eps),
//   MUFU.RSQ, w = rho * rinv, sum w, fma(w, dx) -- the y and z components
//   are dy * sum w and dz * sum w, added once per row;
// - a repulsion pair is 3 FADD + 3 FFMA (r2 with eps folded in) + MUFU.RSQ +
//   3 FFMA;
// - eps = 1e-30 added to r^2 makes a zero difference contribute exactly 0
//   without a branch (the minimum-norm subgradient of |.| at 0);
// - row / block sums are FP32 and folded per target into a compensated FP32
//   (TwoSum) or an FP64 accumulator;
// - the flattened (tile, unit) space is split evenly over one wave of
//   persistent CTAs; each CTA writes one FP64 partial per tile it touches and
//   a combine kernel adds the partials in a fixed order (deterministic).
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.h"
#include "ptx.cuh"

namespace sparkling {

namespace {

template <typename KT>
__global__ void pack_positions_kernel(const KT *__restrict__ K, int64_t N, float4 *__restrict__ out,
                                      int *status)
{
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        float x = (float)K[3 * i], y = (float)K[3 * i + 1], z = (float)K[3 * i + 2];
        bad |= !(isfinite(x) && isfinite(y) && isfinite(z));
        out[i] = make_float4(x, y, z, 0.f);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(status, kDevNonFinite);
}

// Density rows padded to gxp (multiple of 4) with zeros, and the cell-centre
// coordinate tables computed in double and rounded once to float.
__global__ void pack_grid_kernel(const float *__restrict__ rho, int nx, int ny, int nz, int gxp,
                                 double lo, double hi, float *__restrict__ rho_out,
                                 float *__restrict__ coords, int *status)
{
    const int64_t rows = (int64_t)ny * nz;
    const int64_t total = rows * gxp;
    int bad = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / gxp;
        const int x = (int)(e - r * gxp);
        float v = 0.f;
        if (x < nx) {
            v = rho[r * nx + x];
            bad |= !(isfinite(v) && v >= 0.f);
        }
        rho_out[e] = v;
    }
    const int64_t nc = (int64_t)gxp + ny + nz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc;
         e += (int64_t)gridDim.x * blockDim.x) {
        int q, n;
        if (e < gxp) { q = (int)e; n = nx; }
        else if (e < gxp + ny) { q = (int)(e - gxp); n = ny; }
        else { q = (int)(e - gxp - ny); n = nz; }
        coords[e] = (q < n) ? (float)(lo + ((double)q + 0.5) * ((hi - lo) / (double)n)) : 0.f;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(status, kDevNonFinite);
}

// Wait for the stages a CTA issued but did not consume, so that no bulk copy
// is still writing into shared memory when the CTA exits early.
__device__ void drain_stages(uint64_t *bars, uint32_t first, uint32_t count, int *status)
{
    if (threadIdx.x == 0)
        for (uint32_t g = first; g < first + count; ++g)
            mbar_wait_bounded(&bars[g % kStages], (g / kStages) & 1, status);
    __syncthreads();
}

// Per-thread accumulators in shared memory, one column per thread (a warp
// touches consecutive words).  ACC 0: compensated FP32 (value + TwoSum error
// term); ACC 1: FP64.  Both take 8 bytes per accumulated value.
template <int ACC> struct SmemAcc;

template <> struct SmemAcc<0> {
    float *p;
    __device__ SmemAcc(void *base, int tid) : p(static_cast<float *>(base) + tid) {}
    __device__ void zero(int nv)
    {
        for (int v = 0; v < 2 * nv; ++v) p[v * kThreads] = 0.f;
    }
    __device__ __forceinline__ void add(int v, float x)
    {
        float s = p[(2 * v) * kThreads], c = p[(2 * v + 1) * kThreads], t, e;
        two_sum(s, x, t, e);
        p[(2 * v) * kThreads] = t;
        p[(2 * v + 1) * kThreads] = c + e;
    }
    __device__ double value(int v) const
    {
        return (double)p[(2 * v) * kThreads] + (double)p[(2 * v + 1) * kThreads];
    }
};

template <> struct SmemAcc<1> {
    double *p;
    __device__ SmemAcc(void *base, int tid) : p(static_cast<double *>(base) + tid) {}
    __device__ void zero(int nv)
    {
        for (int v = 0; v < nv; ++v) p[v * kThreads] = 0.0;
    }
    __device__ __forceinline__ void add(int v, float x) { p[v * kThreads] += (double)x; }
    __device__ double value(int v) const { return p[v * kThreads]; }
};

constexpr int kAccBytes = kTargetsPerThread * 3 * 8 * kThreads;   // 24 KB per CTA

// NR grid rows (1 or 2) against the thread's T targets.  The rows share the
// x coordinates, so one dx = kx - x_q feeds NR pairs.  x_q is rebuilt as
// lo + (q + 1/2) h: kxp = kx - lo - h/2 (rounded once from double) and
// dx = kxp - q h with one FFMA per group of 4 points.  Row sums are FP32 and
// are added into the stage accumulators st[t][0..NV).
template <bool ENERGY, int NR>
__device__ __forceinline__ void attr_rows(const float *rows, int gxp, const float *kxp,
                                          const float *ky, const float *kz, const float *yr,
                                          const float *zr, float h, float (*st)[3])
{
    constexpr int T = kTargetsPerThread;
    float s2[NR][T], sw[NR][T], sx[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const float dy = ky[t] - yr[r], dz = kz[t] - zr[r];
            s2[r][t] = fmaf(dy, dy, fmaf(dz, dz, kEps2));
            sw[r][t] = 0.f;
        }
        sx[t] = 0.f;
    }
    const float mh = -h, h2 = 2.f * h, h3 = 3.f * h;
    const int n4 = gxp >> 2;
    float qf = 0.f;
#pragma unroll (NR == 1 ? 2 : 1)
    for (int g4 = 0; g4 < n4; ++g4) {
        float4 w[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r)
            w[r] = reinterpret_cast<const float4 *>(rows + r * gxp)[g4];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            float dx[4];
            dx[0] = fmaf(qf, mh, kxp[t]);
            dx[1] = dx[0] - h;
            dx[2] = dx[0] - h2;
            dx[3] = dx[0] - h3;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float rho = j == 0 ? w[r].x : j == 1 ? w[r].y : j == 2 ? w[r].z : w[r].w;
                    const float r2 = fmaf(dx[j], dx[j], s2[r][t]);
                    const float wt = rho * rsqrt_sfu(r2);
                    if (ENERGY) {
                        sw[r][t] = fmaf(wt, r2, sw[r][t]);     // rho * |d|
                    } else {
                        sw[r][t] += wt;
                        sx[t] = fmaf(wt, dx[j], sx[t]);
                    }
                }
            }
        }
        qf += 4.f;
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        if (ENERGY) {
#pragma unroll
            for (int r = 0; r < NR; ++r) st[t][0] += sw[r][t];
        } else {
            st[t][0] += sx[t];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                st[t][1] = fmaf(ky[t] - yr[r], sw[r][t], st[t][1]);
                st[t][2] = fmaf(kz[t] - zr[r], sw[r][t], st[t][2]);
            }
        }
    }
}

template <int ACC, bool ENERGY>
__device__ bool attraction_segment(const AttrArgs &a, int64_t tile, int64_t r0, int64_t r1,
                                   int slot, float *stage, uint64_t *bars, void *accbase,
                                   uint32_t &consumed)
{
    constexpr int T = kTargetsPerThread;
    constexpr int NV = ENERGY ? 1 : 3;
    const int tid = threadIdx.x;
    float kxp[T], ky[T], kz[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t i = tile * kTile + t * kThreads + tid;
        const float4 p = i < a.N ? a.tgt[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        kxp[t] = (float)((double)p.x - a.x0);
        ky[t] = p.y;
        kz[t] = p.z;
    }
    SmemAcc<ACC> acc(accbase, tid);
    acc.zero(T * NV);
    const int R = a.rows_per_stage;
    const uint32_t nst = (uint32_t)((r1 - r0 + R - 1) / R);
    const int gxp = a.gxp;

    auto issue = [&](uint32_t s) {
        const int64_t rs = r0 + (int64_t)s * R;
        const int64_t re = rs + R < r1 ? rs + R : r1;
        const uint32_t g = consumed + s;
        bulk_load(stage + (g % kStages) * kStageFloats, a.rho + rs * gxp,
                  (uint32_t)((re - rs) * gxp * sizeof(float)), &bars[g % kStages]);
    };
    if (tid == 0)
        for (uint32_t s = 0; s < nst && s < (uint32_t)kStages; ++s)
            issue(s);

    const float *ys = a.coords + gxp;
    const float *zs = ys + a.ny;
    for (uint32_t s = 0; s < nst; ++s) {
        const uint32_t g = consumed + s;
        const bool ok = mbar_wait_bounded(&bars[g % kStages], (g / kStages) & 1, a.status);
        if (__syncthreads_or(!ok)) {
            // Stage s and the ones issued after it may still be in flight.
            const uint32_t left = nst - s;
            drain_stages(bars, g, left < (uint32_t)kStages ? left : (uint32_t)kStages, a.status);
            return false;
        }
        const float *buf = stage + (g % kStages) * kStageFloats;
        const int64_t rs = r0 + (int64_t)s * R;
        const int nrows = (int)((rs + R < r1 ? rs + R : r1) - rs);
        int iy = (int)(rs % a.ny), iz = (int)(rs / a.ny);
        float st[T][3];
#pragma unroll
        for (int t = 0; t < T; ++t) st[t][0] = st[t][1] = st[t][2] = 0.f;
        int rr = 0;
        for (; rr + 1 < nrows; rr += 2) {
            float yr[2], zr[2];
            yr[0] = ys[iy]; zr[0] = zs[iz];
            if (++iy == a.ny) { iy = 0; ++iz; }
            yr[1] = ys[iy]; zr[1] = zs[iz];
            if (++iy == a.ny) { iy = 0; ++iz; }
            attr_rows<ENERGY, 2>(buf + rr * gxp, gxp, kxp, ky, kz, yr, zr, a.hx, st);
        }
        if (rr < nrows) {
            float yr[1] = {ys[iy]}, zr[1] = {zs[iz]};
            attr_rows<ENERGY, 1>(buf + rr * gxp, gxp, kxp, ky, kz, yr, zr, a.hx, st);
        }
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int v = 0; v < NV; ++v) acc.add(t * NV + v, st[t][v]);
        __syncthreads();   // every thread is done with this buffer
        if (tid == 0 && s + kStages < nst) {
            fence_proxy_async_smem();
            issue(s + kStages);
        }
    }
    consumed += nst;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int l = t * kThreads + tid;
        if (tile * kTile + l < a.N) {
            dacc4 v = ENERGY ? make_dacc4(0.0, 0.0, 0.0, acc.value(t))
                             : make_dacc4(acc.value(3 * t), acc.value(3 * t + 1),
                                          acc.value(3 * t + 2), 0.0);
            a.part[(tile * a.sp.slots + slot) * kTile + l] = v;
        }
    }
    return true;
}

template <int ACC, bool ENERGY>
__global__ void __launch_bounds__(kThreads, 3) attraction_kernel(const AttrArgs a)
{
    extern __shared__ __align__(128) float smem[];
    void *accbase = smem;                                     // kAccBytes
    float *stage = smem + kAccBytes / sizeof(float);          // kStages * kStageFloats
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage + kStages * kStageFloats);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s)
            mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const int64_t rows = a.sp.per_tile;
    int64_t u = split_begin(a.sp, blockIdx.x);
    const int64_t uend = split_begin(a.sp, blockIdx.x + 1);
    uint32_t consumed = 0;
    while (u < uend) {
        const int64_t tile = u / rows;
        const int64_t r0 = u - tile * rows;
        const int64_t r1 = rows < r0 + (uend - u) ? rows : r0 + (uend - u);
        const int slot = (int)(blockIdx.x - split_cta_of(a.sp, tile * rows));
        if (!attraction_segment<ACC, ENERGY>(a, tile, r0, r1, slot, stage, bars, accbase,
                                             consumed))
            return;
        u += r1 - r0;
    }
}

template <bool ENERGY>
__device__ __forceinline__ void rep_pair(float kx, float ky, float kz, const float4 q, float &rx,
                                         float &ry, float &rz)
{
    const float dx = kx - q.x, dy = ky - q.y, dz = kz - q.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, kEps2)));
    const float ri = rsqrt_sfu(r2);
    if (ENERGY) {
        rx = fmaf(r2, ri, rx);           // |d|
    } else {
        rx = fmaf(dx, ri, rx);
        ry = fmaf(dy, ri, ry);
        rz = fmaf(dz, ri, rz);
    }
}

template <int ACC, bool ENERGY>
__device__ bool repulsion_segment(const RepArgs &a, int64_t tile, int64_t b0, int64_t b1, int slot,
                                  float4 *stage, uint64_t *bars, void *accbase,
                                  uint32_t &consumed)
{
    constexpr int T = kTargetsPerThread;
    constexpr int NV = ENERGY ? 1 : 3;
    const int tid = threadIdx.x;
    float kx[T], ky[T], kz[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t i = tile * kTile + t * kThreads + tid;
        const float4 p = i < a.N ? a.pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        kx[t] = p.x; ky[t] = p.y; kz[t] = p.z;
    }
    SmemAcc<ACC> acc(accbase, tid);
    acc.zero(T * NV);
    const uint32_t nst = (uint32_t)(b1 - b0);
    auto count_of = [&](int64_t b) -> int {
        const int64_t rem = a.N - b * kSrcBlock;
        return rem < kSrcBlock ? (int)rem : kSrcBlock;
    };
    auto issue = [&](uint32_t s) {
        const int64_t b = b0 + s;
        const uint32_t g = consumed + s;
        bulk_load(stage + (g % kStages) * kSrcBlock, a.pos + b * kSrcBlock,
                  (uint32_t)(count_of(b) * sizeof(float4)), &bars[g % kStages]);
    };
    if (tid == 0)
        for (uint32_t s = 0; s < nst && s < (uint32_t)kStages; ++s)
            issue(s);
    for (uint32_t s = 0; s < nst; ++s) {
        const uint32_t g = consumed + s;
        const bool ok = mbar_wait_bounded(&bars[g % kStages], (g / kStages) & 1, a.status);
        if (__syncthreads_or(!ok)) {
            // Stage s and the ones issued after it may still be in flight.
            const uint32_t left = nst - s;
            drain_stages(bars, g, left < (uint32_t)kStages ? left : (uint32_t)kStages, a.status);
            return false;
        }
        const float4 *buf = stage + (g % kStages) * kSrcBlock;
        const int cnt = count_of(b0 + s);
        float rx[T], ry[T], rz[T];
#pragma unroll
        for (int t = 0; t < T; ++t) { rx[t] = 0.f; ry[t] = 0.f; rz[t] = 0.f; }
        if (cnt == kSrcBlock) {
#pragma unroll 2
            for (int j = 0; j < kSrcBlock; ++j) {
                const float4 q = buf[j];
#pragma unroll
                for (int t = 0; t < T; ++t)
                    rep_pair<ENERGY>(kx[t], ky[t], kz[t], q, rx[t], ry[t], rz[t]);
            }
        } else {
            for (int j = 0; j < cnt; ++j) {
                const float4 q = buf[j];
#pragma unroll
                for (int t = 0; t < T; ++t)
                    rep_pair<ENERGY>(kx[t], ky[t], kz[t], q, rx[t], ry[t], rz[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            acc.add(t * NV, rx[t]);
            if (!ENERGY) {
                acc.add(t * NV + 1, ry[t]);
                acc.add(t * NV + 2, rz[t]);
            }
        }
        __syncthreads();
        if (tid == 0 && s + kStages < nst) {
            fence_proxy_async_smem();
            issue(s + kStages);
        }
    }
    consumed += nst;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int l = t * kThreads + tid;
        if (tile * kTile + l < a.N) {
            dacc4 v = ENERGY ? make_dacc4(0.0, 0.0, 0.0, acc.value(t))
                             : make_dacc4(acc.value(3 * t), acc.value(3 * t + 1),
                                          acc.value(3 * t + 2), 0.0);
            a.part[(tile * a.sp.slots + slot) * kTile + l] = v;
        }
    }
    return true;
}

template <int ACC, bool ENERGY>
__global__ void __launch_bounds__(kThreads, 3) repulsion_kernel(const RepArgs a)
{
    extern __shared__ __align__(128) float4 smem4[];
    void *accbase = smem4;
    float4 *stage = smem4 + kAccBytes / sizeof(float4);
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage + kStages * kSrcBlock);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s)
            mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const int64_t per = a.sp.per_tile;
    int64_t u = split_begin(a.sp, blockIdx.x);
    const int64_t uend = split_begin(a.sp, blockIdx.x + 1);
    uint32_t consumed = 0;
    while (u < uend) {
        const int64_t tile = u / per;
        const int64_t b0 = u - tile * per;
        const int64_t b1 = per < b0 + (uend - u) ? per : b0 + (uend - u);
        const int slot = (int)(blockIdx.x - split_cta_of(a.sp, tile * per));
        if (!repulsion_segment<ACC, ENERGY>(a, tile, b0, b1, slot, stage, bars, accbase, consumed))
            return;
        u += b1 - b0;
    }
}

__device__ __forceinline__ dacc4 sum_slots(const dacc4 *part, const Split &sp, int64_t i)
{
    const int64_t tile = i / kTile, l = i - tile * kTile;
    const int64_t lo = split_cta_of(sp, tile * sp.per_tile);
    const int64_t hi = split_cta_of(sp, (tile + 1) * sp.per_tile - 1);
    dacc4 s = make_dacc4(0.0, 0.0, 0.0, 0.0);
    for (int64_t j = 0; j <= hi - lo; ++j) {
        const dacc4 v = part[(tile * sp.slots + j) * kTile + l];
        s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
    }
    return s;
}

template <typename OT>
__global__ void combine_kernel(const CombineArgs c)
{
    const double invN = 1.0 / (double)c.N;
    const double sc = c.scale_dev ? c.scale * c.scale_dev[0] : c.scale;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        dacc4 a = sum_slots(c.part_a, c.spa, i);
        const dacc4 r = sum_slots(c.part_r, c.spr, i);
        double rx = r.x * invN, ry = r.y * invN, rz = r.z * invN;
        double gx = a.x - rx, gy = a.y - ry, gz = a.z - rz;
        if (sc != 1.0) {
            gx *= sc; gy *= sc; gz *= sc;
            a.x *= sc; a.y *= sc; a.z *= sc;
            rx *= sc; ry *= sc; rz *= sc;
        }
        OT *G = static_cast<OT *>(c.G);
        if (G) { G[3 * i] = (OT)gx; G[3 * i + 1] = (OT)gy; G[3 * i + 2] = (OT)gz; }
        if (c.G64) { c.G64[3 * i] = gx; c.G64[3 * i + 1] = gy; c.G64[3 * i + 2] = gz; }
        OT *A = static_cast<OT *>(c.A);
        if (A) { A[3 * i] = (OT)a.x; A[3 * i + 1] = (OT)a.y; A[3 * i + 2] = (OT)a.z; }
        OT *R = static_cast<OT *>(c.R);
        if (R) { R[3 * i] = (OT)rx; R[3 * i + 1] = (OT)ry; R[3 * i + 2] = (OT)rz; }
    }
}

constexpr int kEnergyThreads = 256;
constexpr int kEnergyPerThread = 4;
constexpr int kEnergyBlock = kEnergyThreads * kEnergyPerThread;

// Fixed-shape tree reduction of two doubles over a block.
__device__ double2 block_sum2(double a, double b)
{
    __shared__ double sa[kEnergyThreads], sb[kEnergyThreads];
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = kEnergyThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    return make_double2(sa[0], sb[0]);
}

// Per block: sum of the per-target energy sums of kEnergyBlock targets.
__global__ void __launch_bounds__(kEnergyThreads) energy_block_kernel(const CombineArgs c)
{
    double ea = 0.0, er = 0.0;
    for (int k = 0; k < kEnergyPerThread; ++k) {
        const int64_t i = (int64_t)blockIdx.x * kEnergyBlock + k * kEnergyThreads + threadIdx.x;
        if (i < c.N) {
            ea += sum_slots(c.part_a, c.spa, i).w;
            er += sum_slots(c.part_r, c.spr, i).w;
        }
    }
    const double2 s = block_sum2(ea, er);
    if (threadIdx.x == 0)
        c.energy_blocks[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kEnergyThreads) energy_final_kernel(const double2 *blocks, int nb,
                                                                      int64_t N, double *out2)
{
    double ea = 0.0, er = 0.0;
    for (int b = threadIdx.x; b < nb; b += kEnergyThreads) {
        ea += blocks[b].x;
        er += blocks[b].y;
    }
    const double2 s = block_sum2(ea, er);
    if (threadIdx.x == 0) {
        const double n = (double)N;
        out2[0] = s.x / n;               // F^a
        out2[1] = s.y / (2.0 * n * n);   // F^r
    }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int ACC, bool E>
void *attraction_fn() { return reinterpret_cast<void *>(attraction_kernel<ACC, E>); }
template <int ACC, bool E>
void *repulsion_fn() { return reinterpret_cast<void *>(repulsion_kernel<ACC, E>); }

void *pick_attraction(int acc, bool energy)
{
    if (acc == 0) return energy ? attraction_fn<0, true>() : attraction_fn<0, false>();
    return energy ? attraction_fn<1, true>() : attraction_fn<1, false>();
}

void *pick_repulsion(int acc, bool energy)
{
    if (acc == 0) return energy ? repulsion_fn<0, true>() : repulsion_fn<0, false>();
    return energy ? repulsion_fn<1, true>() : repulsion_fn<1, false>();
}

int grid_for(int64_t n, int threads, int sms)
{
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)sms * 8;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

} // namespace

cudaError_t launch_pack_positions(const void *K, int dtype, int64_t N, float4 *out, int *status,
                                  int sms, cudaStream_t st)
{
    const int g = grid_for(N, 256, sms);
    if (dtype == 0)
        pack_positions_kernel<float><<<g, 256, 0, st>>>(static_cast<const float *>(K), N, out, status);
    else
        pack_positions_kernel<double><<<g, 256, 0, st>>>(static_cast<const double *>(K), N, out, status);
    return cudaGetLastError();
}

cudaError_t launch_pack_grid(const float *rho, int nx, int ny, int nz, int gxp, double lo,
                             double hi, float *rho_out, float *coords, int *status, int sms,
                             cudaStream_t st)
{
    const int g = grid_for((int64_t)ny * nz * gxp, 256, sms);
    pack_grid_kernel<<<g, 256, 0, st>>>(rho, nx, ny, nz, gxp, lo, hi, rho_out, coords, status);
    return cudaGetLastError();
}

size_t attraction_smem_bytes(int)
{
    return (size_t)kAccBytes + (size_t)kStages * kStageFloats * sizeof(float) +
           kStages * sizeof(uint64_t);
}

size_t repulsion_smem_bytes()
{
    return (size_t)kAccBytes + (size_t)kStages * kSrcBlock * sizeof(float4) +
           kStages * sizeof(uint64_t);
}

int attraction_ctas_per_sm(int acc, bool energy, int gxp)
{
    void *fn = pick_attraction(acc, energy);
    const size_t smem = attraction_smem_bytes(gxp);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kThreads, smem) != cudaSuccess)
        return 0;
    return n;
}

int repulsion_ctas_per_sm(int acc, bool energy)
{
    void *fn = pick_repulsion(acc, energy);
    const size_t smem = repulsion_smem_bytes();
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kThreads, smem) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_attraction(const AttrArgs &a, int acc, bool energy, cudaStream_t st)
{
    void *fn = pick_attraction(acc, energy);
    void *args[] = {const_cast<AttrArgs *>(&a)};
    return cudaLaunchKernel(fn, dim3((unsigned)a.sp.ctas), dim3(kThreads), args,
                            attraction_smem_bytes(a.gxp), st);
}

cudaError_t launch_repulsion(const RepArgs &a, int acc, bool energy, cudaStream_t st)
{
    void *fn = pick_repulsion(acc, energy);
    void *args[] = {const_cast<RepArgs *>(&a)};
    return cudaLaunchKernel(fn, dim3((unsigned)a.sp.ctas), dim3(kThreads), args,
                            repulsion_smem_bytes(), st);
}

cudaError_t launch_combine(const CombineArgs &c, int out_dtype, int sms, cudaStream_t st)
{
    const int g = grid_for(c.N, 256, sms);
    if (out_dtype == 0)
        combine_kernel<float><<<g, 256, 0, st>>>(c);
    else
        combine_kernel<double><<<g, 256, 0, st>>>(c);
    return cudaGetLastError();
}

int energy_blocks(int64_t N) { return (int)((N + kEnergyBlock - 1) / kEnergyBlock); }

cudaError_t launch_combine_energy(const CombineArgs &c, double *out2, cudaStream_t st)
{
    const int nb = energy_blocks(c.N);
    energy_block_kernel<<<nb, kEnergyThreads, 0, st>>>(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    energy_final_kernel<<<1, kEnergyThreads, 0, st>>>(c.energy_blocks, nb, c.N, out2);
    return cudaGetLastError();
}

} // namespace sparkling
