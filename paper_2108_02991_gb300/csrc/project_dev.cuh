// Device code of the per-shot projection shared by the standalone kernel
// (project.cu) and the persistent engine (engine.cu).  See project.cu for the
// algorithm (FISTA on the Fenchel dual, FP64).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.h"
#include "ptx.cuh"

namespace sparkling {
namespace {


struct Arrays {
    double *k[3], *s[3], *y1[3], *y2[3], *q1[3], *q2[3];
};

__device__ __forceinline__ Arrays carve(double *base, int Ns)
{
    Arrays a;
    for (int c = 0; c < 3; ++c) {
        a.k[c] = base + (0 + c) * (size_t)Ns;
        a.s[c] = base + (3 + c) * (size_t)Ns;
        a.y1[c] = base + (6 + c) * (size_t)Ns;
        a.y2[c] = base + (9 + c) * (size_t)Ns;
        a.q1[c] = base + (12 + c) * (size_t)Ns;
        a.q2[c] = base + (15 + c) * (size_t)Ns;
    }
    return a;
}

// Phase S: s = pin(clip(k - D1^T d1 - D2^T d2)) for the dual pair (d1, d2).
__device__ __forceinline__ void primal_phase(const Arrays &A, double *const d1[3],
                                             double *const d2[3], int Ns, double box,
                                             int pin_index, const double *pin)
{
    for (int m = threadIdx.x; m < Ns; m += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double t1 = 0.0, t2 = 0.0;
            if (m >= 1) t1 += d1[c][m - 1];
            if (m < Ns - 1) t1 -= d1[c][m];
            if (m >= 2) t2 += d2[c][m - 2];
            if (m >= 1 && m < Ns - 1 - 0 && m - 1 < Ns - 2) t2 -= 2.0 * d2[c][m - 1];
            if (m < Ns - 2) t2 += d2[c][m];
            double v = A.k[c][m] - t1 - t2;
            v = v > box ? box : v;
            v = v < -box ? -box : v;
            A.s[c][m] = (m == pin_index) ? pin[c] : v;
        }
    }
}

__device__ __forceinline__ double norm3(double a, double b, double c)
{
    return sqrt(a * a + b * b + c * c);
}

// Phase Z: dual proximal-gradient step and FISTA extrapolation.
__device__ __forceinline__ void dual_phase(const Arrays &A, int Ns, double r1, double r2,
                                           double mom)
{
    constexpr double tau = 1.0 / 20.0;
    for (int n = threadIdx.x; n < Ns - 1; n += blockDim.x) {
        double z[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            z[c] = A.y1[c][n] + tau * (A.s[c][n + 1] - A.s[c][n]);
        // q = z - P_ball(r1)(z) = z * max(0, 1 - r1/|z|), one rsqrt when |z| > r1
        const double zz = z[0] * z[0] + z[1] * z[1] + z[2] * z[2];
        const double f = zz > r1 * r1 ? 1.0 - r1 * rsqrt(zz) : 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double qn = z[c] * f;
            A.y1[c][n] = qn + mom * (qn - A.q1[c][n]);
            A.q1[c][n] = qn;
        }
        if (n < Ns - 2) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                z[c] = A.y2[c][n] + tau * (A.s[c][n + 2] - 2.0 * A.s[c][n + 1] + A.s[c][n]);
            const double zz2 = z[0] * z[0] + z[1] * z[1] + z[2] * z[2];
            const double f2 = zz2 > r2 * r2 ? 1.0 - r2 * rsqrt(zz2) : 0.0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double qn = z[c] * f2;
                A.y2[c][n] = qn + mom * (qn - A.q2[c][n]);
                A.q2[c][n] = qn;
            }
        }
    }
}

// Block-wide max of four values and sum of one (all threads get the result).
__device__ void block_reduce(double v[4], double &g)
{
    __shared__ double red[32][5];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            v[e] = fmax(v[e], __shfl_xor_sync(0xffffffffu, v[e], o));
        g += __shfl_xor_sync(0xffffffffu, g, o);
    }
    __syncthreads();
    if (lane == 0) {
        for (int e = 0; e < 4; ++e) red[warp][e] = v[e];
        red[warp][4] = g;
    }
    __syncthreads();
    for (int e = 0; e < 4; ++e) v[e] = red[0][e];
    g = red[0][4];
    for (int w = 1; w < nw; ++w) {
        for (int e = 0; e < 4; ++e) v[e] = fmax(v[e], red[w][e]);
        g += red[w][4];
    }
    __syncthreads();
}

// Violations (amplitude, slew, box, pin) of s against (ra, rb, box, pin) and
// the duality gap of (q1, q2) at s, reduced over the block.
__device__ void check_phase(const Arrays &A, int Ns, double ra, double rb, double box,
                            int pin_index, const double *pin, double v[4], double &gap)
{
    v[0] = v[1] = v[2] = v[3] = 0.0;
    gap = 0.0;
    for (int n = threadIdx.x; n < Ns; n += blockDim.x) {
        if (n < Ns - 1) {
            double d[3];
            for (int c = 0; c < 3; ++c) d[c] = A.s[c][n + 1] - A.s[c][n];
            v[0] = fmax(v[0], norm3(d[0], d[1], d[2]) - ra);
            gap += ra * norm3(A.q1[0][n], A.q1[1][n], A.q1[2][n]) -
                   (A.q1[0][n] * d[0] + A.q1[1][n] * d[1] + A.q1[2][n] * d[2]);
        }
        if (n < Ns - 2) {
            double d[3];
            for (int c = 0; c < 3; ++c) d[c] = A.s[c][n + 2] - 2.0 * A.s[c][n + 1] + A.s[c][n];
            v[1] = fmax(v[1], norm3(d[0], d[1], d[2]) - rb);
            gap += rb * norm3(A.q2[0][n], A.q2[1][n], A.q2[2][n]) -
                   (A.q2[0][n] * d[0] + A.q2[1][n] * d[1] + A.q2[2][n] * d[2]);
        }
        for (int c = 0; c < 3; ++c) v[2] = fmax(v[2], fabs(A.s[c][n]) - box);
        if (n == pin_index)
            for (int c = 0; c < 3; ++c) v[3] = fmax(v[3], fabs(A.s[c][n] - pin[c]));
    }
    block_reduce(v, gap);
}

// Constraint set and iteration control of one shot's projection.
struct ShotParams {
    int Ns;
    double alpha, beta, box, tol, margin;
    double pin[3];
    int pin_index, n_iter, check_every;
    unsigned long long *viol;   // optional [4]
    int *notconv;               // optional
};

// Project one shot (called by every thread of the block).  loadk(m, k)
// writes the FP64 input coordinates k[0..2] of sample m (the stepped
// K - eta G);
// the result is written to Kshot ([Ns][3], KT).  A holds the 18 FP64 state
// arrays (shared or global memory).
template <typename KT, class LoadK>
__device__ void project_shot(const Arrays &A, KT *Kshot, const ShotParams &p, LoadK loadk)
{
    const int Ns = p.Ns;
    double *const y1[3] = {A.y1[0], A.y1[1], A.y1[2]};
    double *const y2[3] = {A.y2[0], A.y2[1], A.y2[2]};
    double *const q1[3] = {A.q1[0], A.q1[1], A.q1[2]};
    double *const q2[3] = {A.q2[0], A.q2[1], A.q2[2]};
    const bool converge = p.tol > 0.0;
    const double a_eff = converge ? p.alpha * (1.0 - p.margin) : p.alpha;
    const double b_eff = converge ? p.beta * (1.0 - p.margin) : p.beta;
    const double tau = 1.0 / 20.0;
    for (int m = threadIdx.x; m < Ns; m += blockDim.x) {
        double kv[3];
        loadk(m, kv);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            A.k[c][m] = kv[c];
            A.y1[c][m] = 0.0; A.y2[c][m] = 0.0;
            A.q1[c][m] = 0.0; A.q2[c][m] = 0.0;
        }
    }
    __syncthreads();
    double t = 1.0;
    bool certified = !converge;
    for (int it = 0; it < p.n_iter; ++it) {
        primal_phase(A, y1, y2, Ns, p.box, p.pin_index, p.pin);
        __syncthreads();
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const double mom = (t - 1.0) / tn;
        dual_phase(A, Ns, tau * a_eff, tau * b_eff, mom);
        t = tn;
        __syncthreads();
        if (converge && p.check_every > 0 && (it + 1) % p.check_every == 0) {
            primal_phase(A, q1, q2, Ns, p.box, p.pin_index, p.pin);
            __syncthreads();
            double v[4], gap;
            check_phase(A, Ns, a_eff, b_eff, p.box, p.pin_index, p.pin, v, gap);
            if (v[0] <= p.tol && v[1] <= p.tol && v[2] <= p.tol && v[3] <= p.tol &&
                gap <= p.tol) {
                certified = true;
                break;
            }
        }
    }
    primal_phase(A, q1, q2, Ns, p.box, p.pin_index, p.pin);
    __syncthreads();
    if (converge && !certified) {
        double v[4], gap;
        check_phase(A, Ns, a_eff, b_eff, p.box, p.pin_index, p.pin, v, gap);
        certified = v[0] <= p.tol && v[1] <= p.tol && v[2] <= p.tol && v[3] <= p.tol &&
                    gap <= p.tol;
        if (!certified && threadIdx.x == 0 && p.notconv)
            atomicAdd(p.notconv, 1);
    }
    for (int m = threadIdx.x; m < Ns; m += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Kshot[3 * m + c] = (KT)A.s[c][m];
    }
    if (p.viol) {
        // Violations of the rounded output against the requested set.
        __syncthreads();
        for (int m = threadIdx.x; m < Ns; m += blockDim.x)
            for (int c = 0; c < 3; ++c)
                A.s[c][m] = (double)Kshot[3 * m + c];
        __syncthreads();
        double v[4], gap;
        check_phase(A, Ns, p.alpha, p.beta, p.box, p.pin_index, p.pin, v, gap);
        if (threadIdx.x == 0)
            for (int e = 0; e < 4; ++e)
                atomicMax(&p.viol[e], (unsigned long long)__double_as_longlong(fmax(v[e], 0.0)));
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Mixed-precision form for FP32 outputs (fixed iterations).  The iteration is
// the same dual FISTA, rewritten on small quantities: the displacement
// e = s - k instead of s, with the large terms computed once per shot in
// FP64 and stored as FP32 differences:
//   e(q)  = clamp(-(D1^T q1 + D2^T q2), lo, hi),  lo = -box - k, hi = box - k
//           (lo = hi = v - k at the pinned sample)
//   D s   = D k + D e   (D1 k and D2 k precomputed in FP64)
// Every FP32 operand is then of the size of a displacement or a dual, so the
// rounding is ~1e-7 of those (~1e-10 absolute for the workloads), far below
// the FP32 rounding of the output s = k + e, which is formed in FP64.  On
// GB300, FP64 runs at 1/64 of the FP32 rate, which this form avoids.

constexpr int kMixedFloats = 27;   // per sample: e, lo, hi, D1k, D2k, q1, y1, q2, y2 (x3)

struct ArraysF {
    float *e[3], *lo[3], *hi[3], *d1k[3], *d2k[3], *q1[3], *y1[3], *q2[3], *y2[3];
};

__device__ __forceinline__ ArraysF carve_f(float *base, int Ns)
{
    ArraysF a;
    for (int c = 0; c < 3; ++c) {
        a.e[c] = base + (0 + c) * (size_t)Ns;
        a.lo[c] = base + (3 + c) * (size_t)Ns;
        a.hi[c] = base + (6 + c) * (size_t)Ns;
        a.d1k[c] = base + (9 + c) * (size_t)Ns;
        a.d2k[c] = base + (12 + c) * (size_t)Ns;
        a.q1[c] = base + (15 + c) * (size_t)Ns;
        a.y1[c] = base + (18 + c) * (size_t)Ns;
        a.q2[c] = base + (21 + c) * (size_t)Ns;
        a.y2[c] = base + (24 + c) * (size_t)Ns;
    }
    return a;
}

__device__ __forceinline__ void primal_phase_f(const ArraysF &A, float *const d1[3],
                                               float *const d2[3], int Ns)
{
    for (int m = threadIdx.x; m < Ns; m += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float t1 = 0.f, t2 = 0.f;
            if (m >= 1) t1 += d1[c][m - 1];
            if (m < Ns - 1) t1 -= d1[c][m];
            if (m >= 2) t2 += d2[c][m - 2];
            if (m >= 1 && m <= Ns - 2) t2 -= 2.f * d2[c][m - 1];
            if (m < Ns - 2) t2 += d2[c][m];
            const float v = -t1 - t2;
            A.e[c][m] = fminf(fmaxf(v, A.lo[c][m]), A.hi[c][m]);
        }
    }
}

__device__ __forceinline__ void dual_phase_f(const ArraysF &A, int Ns, float r1, float r2,
                                             float mom)
{
    constexpr float tau = 1.0f / 20.0f;
    const float r1s = r1 * r1, r2s = r2 * r2;
    for (int n = threadIdx.x; n < Ns - 1; n += blockDim.x) {
        float z[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            z[c] = fmaf(tau, A.d1k[c][n] + (A.e[c][n + 1] - A.e[c][n]), A.y1[c][n]);
        float zz = z[0] * z[0] + z[1] * z[1] + z[2] * z[2];
        float f = zz > r1s ? 1.f - r1 * rsqrtf(zz) : 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float qn = z[c] * f;
            A.y1[c][n] = fmaf(mom, qn - A.q1[c][n], qn);
            A.q1[c][n] = qn;
        }
        if (n < Ns - 2) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                z[c] = fmaf(tau, A.d2k[c][n] + (A.e[c][n + 2] - 2.f * A.e[c][n + 1] + A.e[c][n]),
                            A.y2[c][n]);
            zz = z[0] * z[0] + z[1] * z[1] + z[2] * z[2];
            f = zz > r2s ? 1.f - r2 * rsqrtf(zz) : 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float qn = z[c] * f;
                A.y2[c][n] = fmaf(mom, qn - A.q2[c][n], qn);
                A.q2[c][n] = qn;
            }
        }
    }
}

// Fixed-iteration projection of one shot in the mixed form; same contract as
// project_shot (loadk gives the FP64 stepped input; it is called twice per
// sample: for the set-up and for the output s = k + e).
template <typename KT, class LoadK>
__device__ void project_shot_mixed(const ArraysF &A, KT *Kshot, const ShotParams &p, LoadK loadk)
{
    const int Ns = p.Ns;
    float *const y1[3] = {A.y1[0], A.y1[1], A.y1[2]};
    float *const y2[3] = {A.y2[0], A.y2[1], A.y2[2]};
    float *const q1[3] = {A.q1[0], A.q1[1], A.q1[2]};
    float *const q2[3] = {A.q2[0], A.q2[1], A.q2[2]};
    // set-up: lo/hi (FP64 differences, rounded once), duals to zero
    for (int m = threadIdx.x; m < Ns; m += blockDim.x) {
        double kv[3];
        loadk(m, kv);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (m == p.pin_index) {
                A.lo[c][m] = A.hi[c][m] = (float)(p.pin[c] - kv[c]);
            } else {
                A.lo[c][m] = (float)(-p.box - kv[c]);
                A.hi[c][m] = (float)(p.box - kv[c]);
            }
            A.q1[c][m] = 0.f; A.y1[c][m] = 0.f; A.q2[c][m] = 0.f; A.y2[c][m] = 0.f;
        }
    }
    // D1 k and D2 k in FP64: each sample needs its two right neighbours.
    for (int n = threadIdx.x; n < Ns - 1; n += blockDim.x) {
        double k0[3], k1[3], k2[3];
        loadk(n, k0);
        loadk(n + 1, k1);
        if (n < Ns - 2) loadk(n + 2, k2);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            A.d1k[c][n] = (float)(k1[c] - k0[c]);
            if (n < Ns - 2) A.d2k[c][n] = (float)(k2[c] - 2.0 * k1[c] + k0[c]);
        }
    }
    __syncthreads();
    const float tau = 1.0f / 20.0f;
    const float r1 = (float)(tau * p.alpha), r2 = (float)(tau * p.beta);
    double t = 1.0;
    for (int it = 0; it < p.n_iter; ++it) {
        primal_phase_f(A, y1, y2, Ns);
        __syncthreads();
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const float mom = (float)((t - 1.0) / tn);
        dual_phase_f(A, Ns, r1, r2, mom);
        t = tn;
        __syncthreads();
    }
    primal_phase_f(A, q1, q2, Ns);
    __syncthreads();
    // s = k + e in FP64, with the box and the pin applied exactly (e itself
    // only reaches them up to its FP32 rounding).
    for (int m = threadIdx.x; m < Ns; m += blockDim.x) {
        double kv[3];
        loadk(m, kv);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double v = kv[c] + (double)A.e[c][m];
            v = v > p.box ? p.box : (v < -p.box ? -p.box : v);
            Kshot[3 * m + c] = (KT)(m == p.pin_index ? p.pin[c] : v);
        }
    }
    __syncthreads();
}

// Violations of an output shot already written to Kshot (device memory),
// evaluated in FP64 and max-reduced into viol[4] (amplitude, slew, box, pin).
template <typename KT>
__device__ void record_violation(const KT *Kshot, const ShotParams &p)
{
    __syncthreads();
    double v[4] = {0.0, 0.0, 0.0, 0.0}, unused = 0.0;
    const int Ns = p.Ns;
    for (int n = threadIdx.x; n < Ns; n += blockDim.x) {
        double s0[3], s1[3], s2[3];
        for (int c = 0; c < 3; ++c) {
            s0[c] = (double)Kshot[3 * n + c];
            v[2] = fmax(v[2], fabs(s0[c]) - p.box);
            if (n == p.pin_index) v[3] = fmax(v[3], fabs(s0[c] - p.pin[c]));
        }
        if (n < Ns - 1) {
            for (int c = 0; c < 3; ++c) s1[c] = (double)Kshot[3 * (n + 1) + c];
            v[0] = fmax(v[0], norm3(s1[0] - s0[0], s1[1] - s0[1], s1[2] - s0[2]) - p.alpha);
        }
        if (n < Ns - 2) {
            for (int c = 0; c < 3; ++c) s2[c] = (double)Kshot[3 * (n + 2) + c];
            v[1] = fmax(v[1], norm3(s2[0] - 2.0 * s1[0] + s0[0], s2[1] - 2.0 * s1[1] + s0[1],
                                    s2[2] - 2.0 * s1[2] + s0[2]) - p.beta);
        }
    }
    block_reduce(v, unused);
    if (threadIdx.x == 0)
        for (int e = 0; e < 4; ++e)
            atomicMax(&p.viol[e], (unsigned long long)__double_as_longlong(fmax(v[e], 0.0)));
    __syncthreads();
}

} // namespace
} // namespace sparkling
