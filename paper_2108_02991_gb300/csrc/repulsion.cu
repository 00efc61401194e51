// Standalone repulsion kernels of every tile shape: the persistent even split
// of (target tile, source block) units over one wave of CTAs, each CTA
// streaming 1024-sample source blocks through shared memory (see pairs.cu and
// pair_dev.cuh).  Kept in its own translation unit so that the variants
// compile in parallel with the attraction ones.
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.h"
#include "pair_dev.cuh"
#include "ptx.cuh"

namespace sparkling {

namespace {

constexpr int min_ctas(int nt) { return nt >= 512 ? 2 : 768 / nt; }

template <int ACC, bool ENERGY, int NT, int UNROLL>
__global__ void __launch_bounds__(NT, min_ctas(NT)) repulsion_kernel(const RepArgs a)
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
        if (!repulsion_segment<ACC, ENERGY, NT, UNROLL>(a, tile, b0, b1, slot, stage, bars, accbase,
                                                        consumed))
            return;
        u += b1 - b0;
    }
}

template <int NT, int U>
void *pick(int acc, bool energy)
{
    if (acc == 0)
        return energy ? reinterpret_cast<void *>(repulsion_kernel<0, true, NT, U>)
                      : reinterpret_cast<void *>(repulsion_kernel<0, false, NT, U>);
    return energy ? reinterpret_cast<void *>(repulsion_kernel<1, true, NT, U>)
                  : reinterpret_cast<void *>(repulsion_kernel<1, false, NT, U>);
}

void *pick_repulsion(int acc, bool energy, int variant)
{
    switch (variant) {
    case 0: return pick<128, 2>(acc, energy);
    case 1: return pick<256, 1>(acc, energy);
    case 3: return pick<256, 4>(acc, energy);
    case 4: return pick<512, 2>(acc, energy);
    default: return pick<256, 2>(acc, energy);
    }
}

} // namespace

int rep_variant_threads(int v) { return v == 0 ? 128 : (v == 4 ? 512 : 256); }

int rep_variant_unroll(int v) { return v == 1 ? 1 : (v == 3 ? 4 : 2); }

size_t repulsion_smem_bytes()
{
    return (size_t)kAccBytes + (size_t)kStages * kSrcBlock * sizeof(float4) +
           kStages * sizeof(uint64_t);
}

int repulsion_ctas_per_sm(int acc, bool energy, int variant)
{
    void *fn = pick_repulsion(acc, energy, variant);
    const size_t smem = repulsion_smem_bytes();
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, rep_variant_threads(variant), smem) !=
        cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_repulsion(const RepArgs &a, int acc, bool energy, int variant, cudaStream_t st)
{
    void *fn = pick_repulsion(acc, energy, variant);
    void *args[] = {const_cast<RepArgs *>(&a)};
    return cudaLaunchKernel(fn, dim3((unsigned)a.sp.ctas), dim3(rep_variant_threads(variant)), args,
                            repulsion_smem_bytes(), st);
}

} // namespace sparkling
