// Device side of the multi-resolution driver (Algorithm 1): the linear
// interpolator between levels and the reductions of the Barzilai-Borwein
// step (Sec. II-C, choice of step size).  The level and iteration loop is
// host code in api.cu; every arithmetic step runs here or in the pair and
// projection kernels.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace sparkling {

namespace {

template <typename KT> __device__ __forceinline__ double ld(const KT *p, int64_t i) { return (double)p[i]; }

// L_{2d}: sample n of a d-sample shot goes to fine index 2n; fine index
// 2n + 1 is the midpoint of coarse samples n and n + 1, and the last fine
// sample continues the last coarse segment (a one-sample shot repeats).
// One thread per fine coordinate, arithmetic in double, one rounding to KT.
template <typename KT>
__global__ void upsample_kernel(const KT *__restrict__ Kc, KT *__restrict__ Kf, int64_t Nc,
                                int64_t d)
{
    const int64_t total = Nc * 2 * d * 3;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e % 3);
        const int64_t m = (e / 3) % (2 * d), s = e / (3 * 2 * d);
        const int64_t n = m >> 1;
        const KT *c = Kc + 3 * d * s;
        const double here = ld(c, 3 * n + a);
        double v;
        if ((m & 1) == 0) v = here;
        else if (n + 1 < d) v = 0.5 * (here + ld(c, 3 * (n + 1) + a));
        else if (d > 1) v = here + 0.5 * (here - ld(c, 3 * (n - 1) + a));
        else v = here;
        Kf[e] = (KT)v;
    }
}

constexpr int kBBThreads = 256;

// Per block: sum of s.s and s.y over its coordinates (s = K - Kp,
// y = G - Gp), then Kp <- K and Gp <- G.  dots = 0 only copies.
template <typename KT>
__global__ void __launch_bounds__(kBBThreads) bb_partial_kernel(const KT *__restrict__ K,
                                                                double *__restrict__ Kp,
                                                                const double *__restrict__ G,
                                                                double *__restrict__ Gp, int64_t n,
                                                                int dots, double2 *__restrict__ part)
{
    double ss = 0.0, sy = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)kBBThreads + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * kBBThreads) {
        const double k = (double)K[e], g = G[e];
        if (dots) {
            const double s = k - Kp[e], y = g - Gp[e];
            ss = fma(s, s, ss);
            sy = fma(s, y, sy);
        }
        Kp[e] = k;
        Gp[e] = g;
    }
    __shared__ double a[kBBThreads], b[kBBThreads];
    a[threadIdx.x] = ss;
    b[threadIdx.x] = sy;
    __syncthreads();
    for (int w = kBBThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            a[threadIdx.x] += a[threadIdx.x + w];
            b[threadIdx.x] += b[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(a[0], b[0]);
}

// The block partials in a fixed order (deterministic): out = (s.s, s.y).
__global__ void __launch_bounds__(kBBThreads) bb_final_kernel(const double2 *__restrict__ part,
                                                              int nb, double *__restrict__ out)
{
    __shared__ double a[kBBThreads], b[kBBThreads];
    double ss = 0.0, sy = 0.0;
    for (int i = threadIdx.x; i < nb; i += kBBThreads) {
        ss += part[i].x;
        sy += part[i].y;
    }
    a[threadIdx.x] = ss;
    b[threadIdx.x] = sy;
    __syncthreads();
    for (int w = kBBThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            a[threadIdx.x] += a[threadIdx.x + w];
            b[threadIdx.x] += b[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = a[0];
        out[1] = b[0];
    }
}

int blocks_for(int64_t n, int sms)
{
    const int64_t b = (n + kBBThreads - 1) / kBBThreads, cap = (int64_t)sms * 8;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

} // namespace

cudaError_t launch_upsample(const void *Kc, void *Kf, int dtype, int64_t Nc, int64_t d, int sms,
                            cudaStream_t st)
{
    const int nb = blocks_for(Nc * 2 * d * 3, sms);
    if (dtype == 0)
        upsample_kernel<float><<<nb, kBBThreads, 0, st>>>(static_cast<const float *>(Kc),
                                                          static_cast<float *>(Kf), Nc, d);
    else
        upsample_kernel<double><<<nb, kBBThreads, 0, st>>>(static_cast<const double *>(Kc),
                                                           static_cast<double *>(Kf), Nc, d);
    return cudaGetLastError();
}

int bb_blocks(int64_t n, int sms) { return blocks_for(n, sms); }

cudaError_t launch_bb(const void *K, int dtype, double *Kp, const double *G, double *Gp, int64_t n,
                      bool dots, double2 *part, double *out, int sms, cudaStream_t st)
{
    const int nb = blocks_for(n, sms);
    if (dtype == 0)
        bb_partial_kernel<float><<<nb, kBBThreads, 0, st>>>(static_cast<const float *>(K), Kp, G,
                                                            Gp, n, dots ? 1 : 0, part);
    else
        bb_partial_kernel<double><<<nb, kBBThreads, 0, st>>>(static_cast<const double *>(K), Kp,
                                                             G, Gp, n, dots ? 1 : 0, part);
    if (dots) bb_final_kernel<<<1, kBBThreads, 0, st>>>(part, nb, out);
    return cudaGetLastError();
}

} // namespace sparkling
