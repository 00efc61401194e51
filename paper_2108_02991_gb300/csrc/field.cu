// Fast attraction, the paper's own method (Sec. II-C.1, eq.
// attraction_derivative_basic): the attraction field
//   E(y) = sum_q rho_q (y - x_q)/|y - x_q|      and potential
//   phi(y) = sum_q rho_q |y - x_q|
// are computed once per density on the nodes of the density grid extended by
// one node on each side (nodes lo + (m + 1/2) h, m = -1 .. n), as exact
// discrete convolutions of rho with the kernels d/|d| and |d| -- done with
// real-to-complex FFTs in FP64 (cuFFT) on a periodic box of L >= 2n + 1
// points per axis, so that every offset m - q in [-n, n] has its own residue
// and the circular convolution equals the linear one.  Each iteration then
// interpolates E (and phi) trilinearly at the samples: O(N) work instead of
// O(N P).  The result approximates the direct sum; its error against the
// direct sum is measured, not assumed.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>

#include "kernels.h"

namespace sparkling {

namespace {

// Kernel samples on the periodic box: component c of k(d) at the offset
// d = (dx, dy, dz) (in cells) whose residue is the array index.  With
// |p|_eps = sqrt(|p|^2 + eps^2) and p = d h: c 0..2: p_c / |p|_eps (0 at
// d = 0); c 3: |p|_eps.
__global__ void fill_kernel_kernel(double *out, int Lx, int Ly, int Lz, double hx, double hy,
                                   double hz, double eps2, int c)
{
    const int64_t total = (int64_t)Lx * Ly * Lz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(e % Lx), iy = (int)((e / Lx) % Ly), iz = (int)(e / ((int64_t)Lx * Ly));
        // residue -> signed offset in (-L/2, L/2]
        const int dx = ix <= Lx / 2 ? ix : ix - Lx;
        const int dy = iy <= Ly / 2 ? iy : iy - Ly;
        const int dz = iz <= Lz / 2 ? iz : iz - Lz;
        const double px = dx * hx, py = dy * hy, pz = dz * hz;
        const double r = sqrt(px * px + py * py + pz * pz + eps2);
        double v;
        if (c == 3) v = r;
        else v = r > 0.0 ? (c == 0 ? px : (c == 1 ? py : pz)) / r : 0.0;
        out[e] = v;
    }
}

// rho (float, [nz][ny][nx]) placed at box index q + 1 (zero elsewhere).
__global__ void fill_density_kernel(double *out, const float *rho, int nx, int ny, int nz, int Lx,
                                    int Ly, int Lz)
{
    const int64_t total = (int64_t)Lx * Ly * Lz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(e % Lx) - 1, iy = (int)((e / Lx) % Ly) - 1,
                  iz = (int)(e / ((int64_t)Lx * Ly)) - 1;
        double v = 0.0;
        if (ix >= 0 && ix < nx && iy >= 0 && iy < ny && iz >= 0 && iz < nz)
            v = (double)rho[((int64_t)iz * ny + iy) * nx + ix];
        out[e] = v;
    }
}

// khat <- khat * rhohat / (Lx Ly Lz)
__global__ void spectral_product_kernel(cufftDoubleComplex *k, const cufftDoubleComplex *r,
                                        int64_t n, double scale)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const cufftDoubleComplex a = k[e], b = r[e];
        k[e].x = (a.x * b.x - a.y * b.y) * scale;
        k[e].y = (a.x * b.y + a.y * b.x) * scale;
    }
}

// Node o = (ox, oy, oz) in [0, n+1]^3 of the convolution (node m = o - 1)
// into component c of the float4 field.
__global__ void extract_kernel(float4 *field, const double *conv, int nx, int ny, int nz, int Lx,
                               int Ly, int c)
{
    const int fx = nx + 2, fy = ny + 2, fz = nz + 2;
    const int64_t total = (int64_t)fx * fy * fz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ox = (int)(e % fx), oy = (int)((e / fx) % fy), oz = (int)(e / ((int64_t)fx * fy));
        const float v = (float)conv[((int64_t)oz * Ly + oy) * Lx + ox];
        float *f = reinterpret_cast<float *>(&field[e]);
        f[c] = v;
    }
}

// Trilinear interpolation of (E, phi) at every sample.  Node o along x sits
// at lo + (o - 1/2) hx, o = 0 .. nx + 1, so a sample in [lo, hi] has
// u = (x - lo)/hx + 1/2 in [1/2, nx + 1/2]: cell o0 = floor(u) in [0, nx].
// Samples outside the box are clamped to the outermost cell.
__global__ void interp_kernel(const float4 *__restrict__ pos, int64_t N,
                              const float4 *__restrict__ field, int nx, int ny, int nz, double lo,
                              double hx, double hy, double hz, dacc4 *__restrict__ out)
{
    const int fx = nx + 2, fy = ny + 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = pos[i];
        int o[3];
        float f[3];
        const double u[3] = {((double)p.x - lo) / hx + 0.5, ((double)p.y - lo) / hy + 0.5,
                             ((double)p.z - lo) / hz + 0.5};
        const int nmax[3] = {nx, ny, nz};
        for (int a = 0; a < 3; ++a) {
            double fl = floor(u[a]);
            int oa = (int)fl;
            double fa = u[a] - fl;
            if (oa < 0) { oa = 0; fa = 0.0; }
            if (oa > nmax[a]) { oa = nmax[a]; fa = 1.0; }
            o[a] = oa;
            f[a] = (float)fa;
        }
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int dx = c & 1, dy = (c >> 1) & 1, dz = c >> 2;
            const float w = (dx ? f[0] : 1.f - f[0]) * (dy ? f[1] : 1.f - f[1]) *
                            (dz ? f[2] : 1.f - f[2]);
            const float4 v = __ldg(&field[((int64_t)(o[2] + dz) * fy + (o[1] + dy)) * fx + (o[0] + dx)]);
            acc[0] = fmaf(w, v.x, acc[0]);
            acc[1] = fmaf(w, v.y, acc[1]);
            acc[2] = fmaf(w, v.z, acc[2]);
            acc[3] = fmaf(w, v.w, acc[3]);
        }
        out[i] = make_dacc4(acc[0], acc[1], acc[2], acc[3]);
    }
}

int grid_of(int64_t n, int sms)
{
    int64_t b = (n + 255) / 256;
    const int64_t cap = (int64_t)sms * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// Smallest L >= m whose prime factors are 2, 3, 5, 7 (fast cuFFT sizes).
int nice_size(int m)
{
    for (int L = m;; ++L) {
        int r = L;
        for (int p : {2, 3, 5, 7})
            while (r % p == 0) r /= p;
        if (r == 1) return L;
    }
}

} // namespace

size_t field_bytes(int nx, int ny, int nz)
{
    return (size_t)(nx + 2) * (ny + 2) * (nz + 2) * sizeof(float4);
}

// Build the (E, phi) node field of a density into `field` (field_bytes).
// Allocates its FFT buffers and plans for the duration of the call.
cudaError_t field_build(const float *rho, int nx, int ny, int nz, double lo, double hi, double eps,
                        float4 *field, int sms, cudaStream_t st, const char **what)
{
    const int Lx = nice_size(2 * nx + 1), Ly = nice_size(2 * ny + 1), Lz = nice_size(2 * nz + 1);
    const int64_t nreal = (int64_t)Lx * Ly * Lz;
    const int64_t ncplx = (int64_t)Lz * Ly * (Lx / 2 + 1);
    const double hx = (hi - lo) / nx, hy = (hi - lo) / ny, hz = (hi - lo) / nz;
    double *real = nullptr;
    cufftDoubleComplex *rhat = nullptr, *khat = nullptr;
    cufftHandle fwd = 0, inv = 0;
    bool have_fwd = false, have_inv = false;
    cudaError_t err = cudaSuccess;
    *what = "field buffers";
    auto done = [&](cudaError_t e) {
        if (have_fwd) cufftDestroy(fwd);
        if (have_inv) cufftDestroy(inv);
        cudaFree(real);
        cudaFree(rhat);
        cudaFree(khat);
        return e;
    };
    if ((err = cudaMalloc(&real, nreal * sizeof(double))) != cudaSuccess) return done(err);
    if ((err = cudaMalloc(&rhat, ncplx * sizeof(cufftDoubleComplex))) != cudaSuccess) return done(err);
    if ((err = cudaMalloc(&khat, ncplx * sizeof(cufftDoubleComplex))) != cudaSuccess) return done(err);
    *what = "cuFFT plans";
    if (cufftPlan3d(&fwd, Lz, Ly, Lx, CUFFT_D2Z) != CUFFT_SUCCESS) return done(cudaErrorUnknown);
    have_fwd = true;
    if (cufftPlan3d(&inv, Lz, Ly, Lx, CUFFT_Z2D) != CUFFT_SUCCESS) return done(cudaErrorUnknown);
    have_inv = true;
    if (cufftSetStream(fwd, st) != CUFFT_SUCCESS || cufftSetStream(inv, st) != CUFFT_SUCCESS)
        return done(cudaErrorUnknown);
    *what = "field transforms";
    const int gr = grid_of(nreal, sms), gc = grid_of(ncplx, sms);
    fill_density_kernel<<<gr, 256, 0, st>>>(real, rho, nx, ny, nz, Lx, Ly, Lz);
    if ((err = cudaGetLastError()) != cudaSuccess) return done(err);
    if (cufftExecD2Z(fwd, real, rhat) != CUFFT_SUCCESS) return done(cudaErrorUnknown);
    for (int c = 0; c < 4; ++c) {
        fill_kernel_kernel<<<gr, 256, 0, st>>>(real, Lx, Ly, Lz, hx, hy, hz, eps * eps, c);
        if ((err = cudaGetLastError()) != cudaSuccess) return done(err);
        if (cufftExecD2Z(fwd, real, khat) != CUFFT_SUCCESS) return done(cudaErrorUnknown);
        spectral_product_kernel<<<gc, 256, 0, st>>>(khat, rhat, ncplx, 1.0 / (double)nreal);
        if ((err = cudaGetLastError()) != cudaSuccess) return done(err);
        if (cufftExecZ2D(inv, khat, real) != CUFFT_SUCCESS) return done(cudaErrorUnknown);
        extract_kernel<<<grid_of((int64_t)(nx + 2) * (ny + 2) * (nz + 2), sms), 256, 0, st>>>(
            field, real, nx, ny, nz, Lx, Ly, c);
        if ((err = cudaGetLastError()) != cudaSuccess) return done(err);
    }
    // the buffers are freed only after the stream has consumed them
    if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return done(err);
    *what = "";
    return done(cudaSuccess);
}

cudaError_t launch_interp(const float4 *pos, int64_t N, const float4 *field, int nx, int ny, int nz,
                          double lo, double hi, dacc4 *out, int sms, cudaStream_t st)
{
    interp_kernel<<<grid_of(N, sms), 256, 0, st>>>(pos, N, field, nx, ny, nz, lo, (hi - lo) / nx,
                                                   (hi - lo) / ny, (hi - lo) / nz, out);
    return cudaGetLastError();
}

} // namespace sparkling
