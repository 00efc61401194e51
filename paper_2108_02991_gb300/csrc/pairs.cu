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
//   (TwoSum) or an FP64 accumulator; the plain FP64-accumulate form of the
//   attraction (acc 2) adds every pair term in FP64 instead, for comparison;
// - the flattened (tile, unit) space is split evenly over one wave of
//   persistent CTAs; each CTA writes one FP64 partial per tile it touches and
//   a combine kernel adds the partials in a fixed order (deterministic).
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.h"
#include "pair_dev.cuh"
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

// Resident CTAs the launch bounds ask for: three at 128 or 256 threads per
// CTA (shared memory holds no more: registers <= 168 and <= 80), two at 512
// (registers <= 64).
constexpr int min_ctas(int nt) { return nt >= 512 ? 2 : 3; }

template <int ACC, bool ENERGY, int NT>
__global__ void __launch_bounds__(NT, min_ctas(NT)) attraction_kernel(const AttrArgs a)
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
        if (!attraction_segment<ACC, ENERGY, NT>(a, tile, r0, r1, slot, stage, bars, accbase,
                                             consumed))
            return;
        u += r1 - r0;
    }
}

template <typename OT>
__global__ void combine_kernel(const CombineArgs c)
{
    const double invN = 1.0 / (double)c.N;
    const double sc = c.scale_dev ? c.scale * c.scale_dev[0] : c.scale;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        dacc4 a = c.a_direct ? c.a_direct[i] : sum_slots(c.part_a, c.spa, i);
        dacc4 r;
        if (c.r_direct) {
            r = c.r_direct[i];
        } else if (c.racc) {
            r.x = (double)(long long)c.racc[3 * i] / kFixScale;
            r.y = (double)(long long)c.racc[3 * i + 1] / kFixScale;
            r.z = (double)(long long)c.racc[3 * i + 2] / kFixScale;
            r.w = 0.0;
        } else {
            r = sum_slots(c.part_r, c.spr, i);
        }
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
            ea += c.a_direct ? c.a_direct[i].w : sum_slots(c.part_a, c.spa, i).w;
            er += c.r_direct ? c.r_direct[i].w
                             : c.racc ? (double)(long long)c.racc[i] / kFixScale
                                      : sum_slots(c.part_r, c.spr, i).w;
        }
    }
    const double2 s = block_sum2(ea, er);
    if (threadIdx.x == 0)
        c.energy_blocks[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kEnergyThreads) energy_final_kernel(const double2 *blocks, int nb,
                                                                      int64_t N, double eps,
                                                                      double *out2)
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
        // the directed sums include the N self pairs, |0|_eps = eps each
        out2[1] = (s.y - n * eps) / (2.0 * n * n);   // F^r
    }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int ACC, bool E, int NT>
void *attraction_fn() { return reinterpret_cast<void *>(attraction_kernel<ACC, E, NT>); }

template <int NT>
void *pick_attraction_nt(int acc, bool energy)
{
    if (acc == 0) return energy ? attraction_fn<0, true, NT>() : attraction_fn<0, false, NT>();
    if (acc == 2) return energy ? attraction_fn<2, true, NT>() : attraction_fn<2, false, NT>();
    return energy ? attraction_fn<1, true, NT>() : attraction_fn<1, false, NT>();
}

void *pick_attraction(int acc, bool energy, int variant)
{
    switch (variant) {
    case 0: return pick_attraction_nt<128>(acc, energy);
    case 2: return pick_attraction_nt<512>(acc, energy);
    default: return pick_attraction_nt<256>(acc, energy);
    }
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

int attr_variant_threads(int v) { return v == 0 ? 128 : (v == 2 ? 512 : 256); }

size_t attraction_smem_bytes(int)
{
    return (size_t)kAccBytes + (size_t)kStages * kStageFloats * sizeof(float) +
           kStages * sizeof(uint64_t);
}

int attraction_ctas_per_sm(int acc, bool energy, int variant)
{
    void *fn = pick_attraction(acc, energy, variant);
    const size_t smem = attraction_smem_bytes(0);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, attr_variant_threads(variant), smem) !=
        cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_attraction(const AttrArgs &a, int acc, bool energy, int variant, cudaStream_t st)
{
    void *fn = pick_attraction(acc, energy, variant);
    void *args[] = {const_cast<AttrArgs *>(&a)};
    return cudaLaunchKernel(fn, dim3((unsigned)a.sp.ctas), dim3(attr_variant_threads(variant)), args,
                            attraction_smem_bytes(a.gxp), st);
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
    energy_final_kernel<<<1, kEnergyThreads, 0, st>>>(c.energy_blocks, nb, c.N, c.eps, out2);
    return cudaGetLastError();
}

} // namespace sparkling
