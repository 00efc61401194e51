// Per-shot projection onto the gradient-amplitude / slew-rate / box / pin
// constraint set (paper eq. constraints, Sec. II-D, Suppl. Sec. I) by FISTA on
// the Fenchel dual of min 1/2 |s - k|^2, in FP64:
//   D1 s[n] = s[n+1] - s[n]                 (n < Ns-1)
//   D2 s[n] = s[n+2] - 2 s[n+1] + s[n]      (n < Ns-2)
//   s(q)    = pin(clip_box(k - D1^T q1 - D2^T q2))
//   z       = y + tau D s(y),  tau = 1/20 (|D1|^2 <= 4, |D2|^2 <= 16)
//   q+      = z * max(0, 1 - tau*radius/|z|)        (row-wise, radius alpha/beta)
//   t+      = (1 + sqrt(1 + 4 t^2))/2,  y = q+ + ((t-1)/t+)(q+ - q)
// The output is s(q).  With a gradient G the shot is first stepped:
// k = K - eta G (eq. proj_grad_descent).
//
// One CTA per shot (grid-stride over shots).  The 18 per-sample FP64 arrays
// (k, s, y1, y2, q1, q2; x, y, z each, structure of arrays so that a warp
// touches consecutive doubles) live in shared memory when they fit and in a
// per-CTA global scratch region otherwise; the code is the same through
// generic pointers.  Each iteration is two phases separated by barriers:
// S computes s from the duals, Z updates the duals from s.
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.h"
#include "ptx.cuh"

namespace sparkling {

namespace {

constexpr int kProjMaxThreads = 1024;
constexpr size_t kProjSmemMax = 200 * 1024;

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
        const double nz = norm3(z[0], z[1], z[2]);
        const double f = nz > r1 ? 1.0 - r1 / nz : 0.0;
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
            const double nz2 = norm3(z[0], z[1], z[2]);
            const double f2 = nz2 > r2 ? 1.0 - r2 / nz2 : 0.0;
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

template <typename KT>
__global__ void __launch_bounds__(kProjMaxThreads) project_kernel(const ProjArgs p)
{
    extern __shared__ __align__(16) double psm[];
    const int Ns = p.Ns;
    double *base = p.gstate ? p.gstate + (size_t)blockIdx.x * 18 * (size_t)Ns : psm;
    const Arrays A = carve(base, Ns);
    double *const y1[3] = {A.y1[0], A.y1[1], A.y1[2]};
    double *const y2[3] = {A.y2[0], A.y2[1], A.y2[2]};
    double *const q1[3] = {A.q1[0], A.q1[1], A.q1[2]};
    double *const q2[3] = {A.q2[0], A.q2[1], A.q2[2]};
    const bool converge = p.tol > 0.0;
    const double a_eff = converge ? p.alpha * (1.0 - p.margin) : p.alpha;
    const double b_eff = converge ? p.beta * (1.0 - p.margin) : p.beta;
    const double tau = 1.0 / 20.0;
    KT *K = static_cast<KT *>(p.K);

    for (int64_t shot = blockIdx.x; shot < p.Nc; shot += gridDim.x) {
        const int64_t off = shot * (int64_t)Ns;
        for (int m = threadIdx.x; m < Ns; m += blockDim.x) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double kv = (double)K[3 * (off + m) + c];
                if (p.G) kv -= p.eta * p.G[3 * (off + m) + c];
                A.k[c][m] = kv;
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
                K[3 * (off + m) + c] = (KT)A.s[c][m];
        }
        if (p.viol) {
            // Violations of the rounded output against the requested set.
            __syncthreads();
            for (int m = threadIdx.x; m < Ns; m += blockDim.x)
                for (int c = 0; c < 3; ++c)
                    A.s[c][m] = (double)K[3 * (off + m) + c];
            __syncthreads();
            double v[4], gap;
            check_phase(A, Ns, p.alpha, p.beta, p.box, p.pin_index, p.pin, v, gap);
            if (threadIdx.x == 0)
                for (int e = 0; e < 4; ++e)
                    atomicMax(&p.viol[e], (unsigned long long)__double_as_longlong(fmax(v[e], 0.0)));
        }
        __syncthreads();
    }
}

} // namespace

size_t project_state_bytes(int Ns) { return (size_t)18 * Ns * sizeof(double); }

bool project_state_in_smem(int Ns) { return project_state_bytes(Ns) <= kProjSmemMax; }

int project_block(int Ns)
{
    int b = ((Ns + 31) / 32) * 32;
    if (b > kProjMaxThreads) b = kProjMaxThreads;
    if (b < 32) b = 32;
    return b;
}

int project_ctas_per_sm(int dtype, int Ns)
{
    void *fn = dtype == 0 ? reinterpret_cast<void *>(project_kernel<float>)
                          : reinterpret_cast<void *>(project_kernel<double>);
    const size_t smem = project_state_in_smem(Ns) ? project_state_bytes(Ns) : 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProjSmemMax) !=
        cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, project_block(Ns), smem) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_project(const ProjArgs &p, int dtype, int grid, cudaStream_t st)
{
    void *fn = dtype == 0 ? reinterpret_cast<void *>(project_kernel<float>)
                          : reinterpret_cast<void *>(project_kernel<double>);
    const size_t smem = p.gstate ? 0 : project_state_bytes(p.Ns);
    void *args[] = {const_cast<ProjArgs *>(&p)};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(project_block(p.Ns)), args, smem, st);
}

} // namespace sparkling
