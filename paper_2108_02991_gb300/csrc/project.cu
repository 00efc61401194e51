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
// FP32 samples may instead (an opt-in of the context) iterate in FP32 on the
// displacement s - k and the duals (project_shot_mixed); FP64 is the default
// for every sample type.
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
#include "project_dev.cuh"
#include "ptx.cuh"

namespace sparkling {

namespace {

constexpr int kProjMaxThreads = 1024;
constexpr size_t kProjSmemMax = 200 * 1024;

template <typename KT>
__global__ void __launch_bounds__(kProjMaxThreads) project_kernel(const ProjArgs p)
{
    extern __shared__ __align__(16) double psm[];
    const int Ns = p.Ns;
    double *base = p.gstate ? p.gstate + (size_t)blockIdx.x * 18 * (size_t)Ns : psm;
    const Arrays A = carve(base, Ns);
    ShotParams sp;
    sp.Ns = Ns;
    sp.alpha = p.alpha; sp.beta = p.beta; sp.box = p.box; sp.tol = p.tol; sp.margin = p.margin;
    for (int c = 0; c < 3; ++c) sp.pin[c] = p.pin[c];
    sp.pin_index = p.pin_index; sp.n_iter = p.n_iter; sp.check_every = p.check_every;
    sp.viol = p.viol; sp.notconv = p.notconv;
    KT *K = static_cast<KT *>(p.K);
    for (int64_t shot = blockIdx.x; shot < p.Nc; shot += gridDim.x) {
        const int64_t off = shot * (int64_t)Ns;
        const double *G = p.G;
        const double eta = p.eta;
        auto loadk = [&](int m, double *kv) {
            for (int c = 0; c < 3; ++c) {
                kv[c] = (double)K[3 * (off + m) + c];
                if (G) kv[c] -= eta * G[3 * (off + m) + c];
            }
        };
        if (sizeof(KT) == 4 && p.tol <= 0.0 && p.mixed) {
            // FP32 output, fixed iterations, asked for: the mixed-precision form
            project_shot_mixed<KT>(carve_f(reinterpret_cast<float *>(base), Ns), K + 3 * off, sp,
                                   loadk);
            if (p.viol) record_violation<KT>(K + 3 * off, sp);
        } else {
            project_shot<KT>(A, K + 3 * off, sp, loadk);
        }
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
