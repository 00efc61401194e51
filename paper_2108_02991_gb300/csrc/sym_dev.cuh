// Device code of the symmetric repulsion shared by the standalone kernel
// (repulsion_sym.cu) and the persistent engine (engine.cu): one item is a
// tile of 1024 targets against a tile of 1024 sources, every unordered pair
// evaluated once (paper eq. Fr_grad with H' = 1; the pair term is odd, so the
// term of (i, j) goes to i and, negated, to j).  See repulsion_sym.cu for the
// work split and the rotation of sources through the lanes of a warp.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.h"
#include "ptx.cuh"

namespace sparkling {
namespace {

__device__ __forceinline__ long long to_fix(float x)
{
    return __float2ll_rn(x * 4294967296.0f);
}

__device__ __forceinline__ void add_fix(unsigned long long *p, long long v)
{
    if (v != 0) atomicAdd(p, (unsigned long long)v);
}

// One off-diagonal item: the thread's T = kTile/NT targets against tile J (in src,
// jvalid valid sources).  Target sums go to ai (registers), source sums to
// jacc ([NV][kTile], shared).  RAGGED: the last tile is partial; tm/sm mask
// the missing targets/sources to zero.
template <bool ENERGY, bool RAGGED, int S, int NT>
__device__ __forceinline__ void sym_item(const float4 *src, int jvalid, const float *tx,
                                         const float *ty, const float *tz, const float *tm,
                                         float eps2, float (*ai)[3], float *jacc)
{
    constexpr int T = kTile / NT;
    constexpr int P = T / 2;                    // target pairs (paired FP32 lanes)
    constexpr int kSymChunk = 32 * S, kChunks = kTile / kSymChunk;
    static_assert(kChunks >= NT / 32 && (kChunks & (kChunks - 1)) == 0, "chunk count");
    static_assert(T % 2 == 0, "targets are processed in pairs");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int from = (lane + 1) & 31;
    // targets (2p, 2p+1) and their sums in the two halves of 64-bit registers
    f2 TX[P], TY[P], TZ[P], AX[P], AY[P], AZ[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        TX[p] = f2_pack(tx[2 * p], tx[2 * p + 1]);
        TY[p] = f2_pack(ty[2 * p], ty[2 * p + 1]);
        TZ[p] = f2_pack(tz[2 * p], tz[2 * p + 1]);
        AX[p] = AY[p] = AZ[p] = f2_pack(0.f, 0.f);
    }
    const f2 E2 = f2_pack(eps2, eps2);
    for (int r = 0; r < kChunks; ++r) {
        const int c = (warp + r) & (kChunks - 1);
        float sx[S], sy[S], sz[S], sm[S], bx[S], by[S], bz[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int j = c * kSymChunk + s * 32 + lane;
            const bool ok = !RAGGED || j < jvalid;
            // a missing source (stale shared memory, possibly NaN) becomes a
            // finite point whose terms the zero mask then removes
            const float4 q = ok ? src[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            sx[s] = q.x; sy[s] = q.y; sz[s] = q.z;
            sm[s] = ok ? 1.f : 0.f;
            bx[s] = 0.f; by[s] = 0.f; bz[s] = 0.f;
        }
        for (int step = 0; step < 32; ++step) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const f2 SX = f2_pack(sx[s], sx[s]), SY = f2_pack(sy[s], sy[s]),
                         SZ = f2_pack(sz[s], sz[s]);
                f2 QX, QY, QZ;                  // the source's share, summed over the pairs
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const f2 DX = f2_sub(TX[p], SX), DY = f2_sub(TY[p], SY),
                             DZ = f2_sub(TZ[p], SZ);
                    const f2 R2 = f2_fma(DX, DX, f2_fma(DY, DY, f2_fma(DZ, DZ, E2)));
                    float r2a, r2b;
                    f2_unpack(R2, r2a, r2b);
                    f2 RI = f2_pack(rsqrt_sfu(r2a), rsqrt_sfu(r2b));
                    if (RAGGED) RI = f2_mul(RI, f2_pack(tm[2 * p] * sm[s], tm[2 * p + 1] * sm[s]));
                    if (ENERGY) {
                        const f2 E = f2_mul(R2, RI);     // |d|, counted for both samples
                        AX[p] = f2_add(AX[p], E);
                        QX = p == 0 ? E : f2_add(QX, E);
                    } else {
                        AX[p] = f2_fma(DX, RI, AX[p]);
                        AY[p] = f2_fma(DY, RI, AY[p]);
                        AZ[p] = f2_fma(DZ, RI, AZ[p]);
                        QX = p == 0 ? f2_mul(DX, RI) : f2_fma(DX, RI, QX);
                        QY = p == 0 ? f2_mul(DY, RI) : f2_fma(DY, RI, QY);
                        QZ = p == 0 ? f2_mul(DZ, RI) : f2_fma(DZ, RI, QZ);
                    }
                }
                float u, v;
                if (ENERGY) {
                    f2_unpack(QX, u, v);
                    bx[s] += u + v;
                } else {                        // the pair term is odd: the source gets -term
                    f2_unpack(QX, u, v);
                    bx[s] -= u + v;
                    f2_unpack(QY, u, v);
                    by[s] -= u + v;
                    f2_unpack(QZ, u, v);
                    bz[s] -= u + v;
                }
            }
            // the sources and their sums move one lane down
#pragma unroll
            for (int s = 0; s < S; ++s) {
                sx[s] = __shfl_sync(0xffffffffu, sx[s], from);
                sy[s] = __shfl_sync(0xffffffffu, sy[s], from);
                sz[s] = __shfl_sync(0xffffffffu, sz[s], from);
                if (RAGGED) sm[s] = __shfl_sync(0xffffffffu, sm[s], from);
                bx[s] = __shfl_sync(0xffffffffu, bx[s], from);
                if (!ENERGY) {
                    by[s] = __shfl_sync(0xffffffffu, by[s], from);
                    bz[s] = __shfl_sync(0xffffffffu, bz[s], from);
                }
            }
        }
        // 32 steps later every source is back in its lane: this warp alone
        // owns chunk c in round r
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int j = c * kSymChunk + s * 32 + lane;
            jacc[j] += bx[s];
            if (!ENERGY) {
                jacc[kTile + j] += by[s];
                jacc[2 * kTile + j] += bz[s];
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        float u, v;
        f2_unpack(AX[p], u, v);
        ai[2 * p][0] += u;
        ai[2 * p + 1][0] += v;
        if (!ENERGY) {
            f2_unpack(AY[p], u, v);
            ai[2 * p][1] += u;
            ai[2 * p + 1][1] += v;
            f2_unpack(AZ[p], u, v);
            ai[2 * p][2] += u;
            ai[2 * p + 1][2] += v;
        }
    }
}

// The same item with the pairing turned around: a lane's two sources
// (c*64 + lane and c*64 + 32 + lane of chunk c) share the 64-bit registers,
// and each target is copied into both halves once per item.  A step then
// needs no packing and no folding: per target, 3 differences, 3 squared-
// distance steps and 3 + 3 accumulations, all paired -- 12 FP32 lane
// operations per unordered pair -- and the source sums stay paired while
// they rotate.  The target sums are folded once per item.
template <bool ENERGY, bool RAGGED, int NT>
__device__ __forceinline__ void sym_item_sp(const float4 *src, int jvalid, const float *tx,
                                            const float *ty, const float *tz, const float *tm,
                                            float eps2, float (*ai)[3], float *jacc)
{
    constexpr int T = kTile / NT;
    constexpr int kChunk = 64, kChunks = kTile / kChunk;
    static_assert(kChunks >= NT / 32 && (kChunks & (kChunks - 1)) == 0, "chunk count");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int from = (lane + 1) & 31;
    f2 TX[T], TY[T], TZ[T], TM[T], AX[T], AY[T], AZ[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        TX[t] = f2_pack(tx[t], tx[t]);
        TY[t] = f2_pack(ty[t], ty[t]);
        TZ[t] = f2_pack(tz[t], tz[t]);
        TM[t] = f2_pack(tm[t], tm[t]);
        AX[t] = AY[t] = AZ[t] = f2_pack(0.f, 0.f);
    }
    const f2 E2 = f2_pack(eps2, eps2);
    for (int r = 0; r < kChunks; ++r) {
        const int c = (warp + r) & (kChunks - 1);
        const int j0 = c * kChunk + lane, j1 = j0 + 32;
        // a missing source (stale shared memory, possibly NaN) becomes a
        // finite point whose terms the zero mask then removes
        const bool ok0 = !RAGGED || j0 < jvalid, ok1 = !RAGGED || j1 < jvalid;
        const float4 q0 = ok0 ? src[j0] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 q1 = ok1 ? src[j1] : make_float4(0.f, 0.f, 0.f, 0.f);
        f2 SX = f2_pack(q0.x, q1.x), SY = f2_pack(q0.y, q1.y), SZ = f2_pack(q0.z, q1.z);
        f2 SM = f2_pack(ok0 ? 1.f : 0.f, ok1 ? 1.f : 0.f);
        f2 BX = f2_pack(0.f, 0.f), BY = BX, BZ = BX;     // + the pair terms of the two sources
        for (int step = 0; step < 32; ++step) {
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const f2 DX = f2_sub(TX[t], SX), DY = f2_sub(TY[t], SY), DZ = f2_sub(TZ[t], SZ);
                const f2 R2 = f2_fma(DX, DX, f2_fma(DY, DY, f2_fma(DZ, DZ, E2)));
                float r2a, r2b;
                f2_unpack(R2, r2a, r2b);
                f2 RI = f2_pack(rsqrt_sfu(r2a), rsqrt_sfu(r2b));
                if (RAGGED) RI = f2_mul(RI, f2_mul(SM, TM[t]));
                if (ENERGY) {
                    const f2 E = f2_mul(R2, RI);      // |d|, counted for both samples
                    AX[t] = f2_add(AX[t], E);
                    BX = f2_add(BX, E);
                } else {
                    AX[t] = f2_fma(DX, RI, AX[t]);
                    AY[t] = f2_fma(DY, RI, AY[t]);
                    AZ[t] = f2_fma(DZ, RI, AZ[t]);
                    BX = f2_fma(DX, RI, BX);
                    BY = f2_fma(DY, RI, BY);
                    BZ = f2_fma(DZ, RI, BZ);
                }
            }
            // the sources and their sums move one lane down
            SX = __shfl_sync(0xffffffffu, SX, from);
            SY = __shfl_sync(0xffffffffu, SY, from);
            SZ = __shfl_sync(0xffffffffu, SZ, from);
            if (RAGGED) SM = __shfl_sync(0xffffffffu, SM, from);
            BX = __shfl_sync(0xffffffffu, BX, from);
            if (!ENERGY) {
                BY = __shfl_sync(0xffffffffu, BY, from);
                BZ = __shfl_sync(0xffffffffu, BZ, from);
            }
        }
        // back home after 32 steps; this warp alone owns chunk c in round r.
        // The pair term is odd: a source's force share is minus the sum.
        float u, v;
        f2_unpack(BX, u, v);
        jacc[j0] += ENERGY ? u : -u;
        jacc[j1] += ENERGY ? v : -v;
        if (!ENERGY) {
            f2_unpack(BY, u, v);
            jacc[kTile + j0] -= u;
            jacc[kTile + j1] -= v;
            f2_unpack(BZ, u, v);
            jacc[2 * kTile + j0] -= u;
            jacc[2 * kTile + j1] -= v;
        }
        __syncthreads();
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        float u, v;
        f2_unpack(AX[t], u, v);
        ai[t][0] += u + v;
        if (!ENERGY) {
            f2_unpack(AY[t], u, v);
            ai[t][1] += u + v;
            f2_unpack(AZ[t], u, v);
            ai[t][2] += u + v;
        }
    }
}

// A diagonal item (I, I): the thread's targets against every source of the
// tile, directed (each ordered pair once, target side only; the self term
// contributes nothing to the force and eps to the energy, which the energy
// reduction removes).
template <bool ENERGY, int NT>
__device__ __forceinline__ void diag_item(const float4 *src, int jvalid, const float *tx,
                                          const float *ty, const float *tz, float eps2,
                                          float (*ai)[3])
{
    constexpr int T = kTile / NT;
#pragma unroll 2
    for (int j = 0; j < jvalid; ++j) {
        const float4 q = src[j];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float dx = tx[t] - q.x, dy = ty[t] - q.y, dz = tz[t] - q.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
            const float ri = rsqrt_sfu(r2);
            if (ENERGY) {
                ai[t][0] = fmaf(r2, ri, ai[t][0]);
            } else {
                ai[t][0] = fmaf(dx, ri, ai[t][0]);
                ai[t][1] = fmaf(dy, ri, ai[t][1]);
                ai[t][2] = fmaf(dz, ri, ai[t][2]);
            }
        }
    }
}

} // namespace
} // namespace sparkling
