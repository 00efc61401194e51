// Device code of the pair sums shared by the standalone kernels (pairs.cu)
// and the persistent engine (engine.cu): per-target shared-memory
// accumulators, and one "segment" of attraction (a tile of targets against a
// run of grid rows) or repulsion (a tile against a run of source blocks),
// streamed through shared memory by 1-D TMA bulk copies.  See pairs.cu for
// the design notes.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.h"
#include "ptx.cuh"

namespace sparkling {
namespace {

// Wait for the stages a CTA issued but did not consume, so that no bulk copy
// is still writing into shared memory when the CTA exits early.
__device__ void drain_stages(uint64_t *bars, uint32_t first, uint32_t count, int *status)
{
    if (threadIdx.x == 0)
        for (uint32_t g = first; g < first + count; ++g)
            mbar_wait_drain(&bars[g % kStages], (g / kStages) & 1, status);
    __syncthreads();
}

// Per-thread accumulators in shared memory, one column per thread (a warp
// touches consecutive words).  ACC 0: compensated FP32 (value + TwoSum error
// term); ACC 1: FP64.  Both take 8 bytes per accumulated value.
template <int ACC, int NT> struct SmemAcc;

template <int NT> struct SmemAcc<0, NT> {
    float *p;
    __device__ SmemAcc(void *base, int tid) : p(static_cast<float *>(base) + tid) {}
    __device__ void zero(int nv)
    {
        for (int v = 0; v < 2 * nv; ++v) p[v * NT] = 0.f;
    }
    __device__ __forceinline__ void add(int v, float x)
    {
        float s = p[(2 * v) * NT], c = p[(2 * v + 1) * NT], t, e;
        two_sum(s, x, t, e);
        p[(2 * v) * NT] = t;
        p[(2 * v + 1) * NT] = c + e;
    }
    __device__ double value(int v) const
    {
        return (double)p[(2 * v) * NT] + (double)p[(2 * v + 1) * NT];
    }
};

template <int NT> struct SmemAcc<1, NT> {
    double *p;
    __device__ SmemAcc(void *base, int tid) : p(static_cast<double *>(base) + tid) {}
    __device__ void zero(int nv)
    {
        for (int v = 0; v < nv; ++v) p[v * NT] = 0.0;
    }
    __device__ __forceinline__ void add(int v, float x) { p[v * NT] += (double)x; }
    __device__ double value(int v) const { return p[v * NT]; }
};

// ACC 2: the plain FP64-accumulate form.  The pair terms are added to FP64
// row sums one by one (no FP32 partial sums), and the row sums go to FP64
// accumulators.
template <int NT> struct SmemAcc<2, NT> {
    double *p;
    __device__ SmemAcc(void *base, int tid) : p(static_cast<double *>(base) + tid) {}
    __device__ void zero(int nv)
    {
        for (int v = 0; v < nv; ++v) p[v * NT] = 0.0;
    }
    __device__ __forceinline__ void add(int v, double x) { p[v * NT] += x; }
    __device__ double value(int v) const { return p[v * NT]; }
};

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// Type of the row sums: FP32 for the compensated and FP64 folds, FP64 for
// the plain FP64-accumulate form.
template <int ACC> struct RowSum { typedef float type; };
template <> struct RowSum<2> { typedef double type; };

constexpr int kAccBytes = kTile * 3 * 8;   // 24 KB per CTA: 3 values x 8 bytes per target

// NR grid rows (1 or 2) against the thread's T targets.  The rows share the
// x coordinates, so one dx = kx - x_q feeds NR pairs.  x_q is rebuilt as
// lo + (q + 1/2) h: kxp = kx - lo - h/2 (rounded once from double) and
// dx = kxp - q h with one FFMA per group of 4 points.  Row sums are FP32 and
// are added into the stage accumulators st[t][0..NV).  AT is the type the
// pair terms are summed in: float (row sums in FP32), or double (every pair
// term converted and added in FP64: the plain FP64-accumulate form).
template <bool ENERGY, int NR, int T, typename AT>
__device__ __forceinline__ void attr_rows(const float *rows, int gxp, const float *kxp,
                                          const float *ky, const float *kz, const float *yr,
                                          const float *zr, float h, float eps2, AT (*st)[3])
{
    float s2[NR][T];
    AT sw[NR][T], sx[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const float dy = ky[t] - yr[r], dz = kz[t] - zr[r];
            s2[r][t] = fmaf(dy, dy, fmaf(dz, dz, eps2));
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
                        sw[r][t] = fma_t((AT)wt, (AT)r2, sw[r][t]);     // rho * |d|
                    } else {
                        sw[r][t] += (AT)wt;
                        sx[t] = fma_t((AT)wt, (AT)dx[j], sx[t]);
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
                st[t][1] = fma_t((AT)(ky[t] - yr[r]), sw[r][t], st[t][1]);
                st[t][2] = fma_t((AT)(kz[t] - zr[r]), sw[r][t], st[t][2]);
            }
        }
    }
}

template <int ACC, bool ENERGY, int NT>
__device__ bool attraction_segment(const AttrArgs &a, int64_t tile, int64_t r0, int64_t r1,
                                   int slot, float *stage, uint64_t *bars, void *accbase,
                                   uint32_t &consumed)
{
    constexpr int T = kTile / NT;
    constexpr int NV = ENERGY ? 1 : 3;
    const int tid = threadIdx.x;
    float kxp[T], ky[T], kz[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t i = tile * kTile + t * NT + tid;
        const float4 p = i < a.N ? a.tgt[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        kxp[t] = (float)((double)p.x - a.x0);
        ky[t] = p.y;
        kz[t] = p.z;
    }
    SmemAcc<ACC, NT> acc(accbase, tid);
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
        typedef typename RowSum<ACC>::type AT;
        AT st[T][3];
#pragma unroll
        for (int t = 0; t < T; ++t) st[t][0] = st[t][1] = st[t][2] = (AT)0;
        int rr = 0;
        for (; rr + 1 < nrows; rr += 2) {
            float yr[2], zr[2];
            yr[0] = ys[iy]; zr[0] = zs[iz];
            if (++iy == a.ny) { iy = 0; ++iz; }
            yr[1] = ys[iy]; zr[1] = zs[iz];
            if (++iy == a.ny) { iy = 0; ++iz; }
            attr_rows<ENERGY, 2, T, AT>(buf + rr * gxp, gxp, kxp, ky, kz, yr, zr, a.hx, a.eps2, st);
        }
        if (rr < nrows) {
            float yr[1] = {ys[iy]}, zr[1] = {zs[iz]};
            attr_rows<ENERGY, 1, T, AT>(buf + rr * gxp, gxp, kxp, ky, kz, yr, zr, a.hx, a.eps2, st);
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
        const int l = t * NT + tid;
        if (tile * kTile + l < a.N) {
            dacc4 v = ENERGY ? make_dacc4(0.0, 0.0, 0.0, acc.value(t))
                             : make_dacc4(acc.value(3 * t), acc.value(3 * t + 1),
                                          acc.value(3 * t + 2), 0.0);
            a.part[(tile * a.sp.slots + slot) * kTile + l] = v;
        }
    }
    return true;
}

template <bool ENERGY>
__device__ __forceinline__ void rep_pair(float kx, float ky, float kz, const float4 q, float eps2,
                                         float &rx, float &ry, float &rz)
{
    const float dx = kx - q.x, dy = ky - q.y, dz = kz - q.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    const float ri = rsqrt_sfu(r2);
    if (ENERGY) {
        rx = fmaf(r2, ri, rx);           // |d|
    } else {
        rx = fmaf(dx, ri, rx);
        ry = fmaf(dy, ri, ry);
        rz = fmaf(dz, ri, rz);
    }
}

template <int ACC, bool ENERGY, int NT, int UNROLL>
__device__ __forceinline__ bool repulsion_segment(const RepArgs &a, int64_t tile, int64_t b0, int64_t b1, int slot,
                                  float4 *stage, uint64_t *bars, void *accbase,
                                  uint32_t &consumed)
{
    constexpr int T = kTile / NT;
    constexpr int NV = ENERGY ? 1 : 3;
    const int tid = threadIdx.x;
    float kx[T], ky[T], kz[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t i = tile * kTile + t * NT + tid;
        const float4 p = i < a.N ? a.pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        kx[t] = p.x; ky[t] = p.y; kz[t] = p.z;
    }
    SmemAcc<ACC, NT> acc(accbase, tid);
    acc.zero(T * NV);
    const float eps2 = a.eps2;
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
#pragma unroll (UNROLL)
            for (int j = 0; j < kSrcBlock; ++j) {
                const float4 q = buf[j];
#pragma unroll
                for (int t = 0; t < T; ++t)
                    rep_pair<ENERGY>(kx[t], ky[t], kz[t], q, eps2, rx[t], ry[t], rz[t]);
            }
        } else {
            for (int j = 0; j < cnt; ++j) {
                const float4 q = buf[j];
#pragma unroll
                for (int t = 0; t < T; ++t)
                    rep_pair<ENERGY>(kx[t], ky[t], kz[t], q, eps2, rx[t], ry[t], rz[t]);
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
        const int l = t * NT + tid;
        if (tile * kTile + l < a.N) {
            dacc4 v = ENERGY ? make_dacc4(0.0, 0.0, 0.0, acc.value(t))
                             : make_dacc4(acc.value(3 * t), acc.value(3 * t + 1),
                                          acc.value(3 * t + 2), 0.0);
            a.part[(tile * a.sp.slots + slot) * kTile + l] = v;
        }
    }
    return true;
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

} // namespace
} // namespace sparkling
