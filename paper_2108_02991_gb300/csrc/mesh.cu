// Fast repulsion: particle-particle particle-mesh (P3M) summation of
// R_i = sum_{j != i} d_ij / |d_ij|_eps, the O(N^2) bottleneck of Sec. II-C.2
// (the paper takes a fast multipole method there; this is the GB300 path).
//
// The kernel splits exactly: d/r = d/r erfc(r/sigma) + d/r erf(r/sigma),
// r = |d|_eps.  The short-range part decays like a Gaussian and is summed
// directly over the pairs closer than rc, found through a cell list (cells
// of side >= rc/2, samples sorted by cell).  The long-range part is smooth and
// is summed on a mesh:
//   1. every sample spreads a unit charge to 4 x 4 x 4 nodes with cubic
//      B-spline weights (64-bit fixed-point atomics: exact, order-free);
//   2. the charge mesh (M^3 nodes, zero-padded to L = 2M per axis) is
//      convolved with the long-range kernel by FP32 real FFTs (cuFFT);
//   3. every sample gathers the four convolved fields (force x, y, z and the
//      potential) from its 64 nodes with the same weights.
// The kernel spectra are built once per mesh and eps: the kernel, tapered to
// zero beyond every offset the mesh can have (a C-infinity step between
// radius sqrt(3) M h and 2 M h), is sampled on a 4M box, transformed (FP64),
// divided by the squared transform of the B-spline window (deconvolution),
// transformed back, cut to the offsets |m| < M and transformed on the L box.
// The taper keeps the deconvolution from amplifying a truncation edge (the
// free-space convolution idea of Vico, Greengard and Ferrando, 2016).
// The erfc of the short-range part is the rational approximation 7.1.26 of
// Abramowitz and Stegun (|error| <= 1.5e-7) times exp(-x^2).
#include <cuda_runtime.h>
#include <cufft.h>
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "kernels.h"
#include "ptx.cuh"

namespace sparkling {

namespace {

constexpr int kMeshThreads = 256;
constexpr double kFix = 4294967296.0;       // charge fixed point: round(w * 2^32)

int grid_for(int64_t n, int sms)
{
    const int64_t b = (n + kMeshThreads - 1) / kMeshThreads, cap = (int64_t)sms * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// C-infinity step: 1 for t <= 0, 0 for t >= 1.
__device__ double taper(double t)
{
    if (t <= 0.0) return 1.0;
    if (t >= 1.0) return 0.0;
    const double a = exp(-1.0 / (1.0 - t)), b = exp(-1.0 / t);
    return a / (a + b);
}

// Component c (0..2 force, 3 potential) of the tapered long-range kernel at
// the offsets of the periodic Lb = 4M box (residue order), planes z0 ..
// z0 + nz - 1 of it: out[z - z0][y][x].
__global__ void fill_slab_kernel(double *out, int Lb, int z0, int nz, double h, double sigma,
                                 double eps2, double r1, double r2, int c)
{
    const int64_t total = (int64_t)nz * Lb * Lb;
    const double spi = sigma * 0.56418958354775628;   // sigma / sqrt(pi)
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(e % Lb), iy = (int)((e / Lb) % Lb);
        const int iz = z0 + (int)(e / ((int64_t)Lb * Lb));
        const double x = (ix <= Lb / 2 ? ix : ix - Lb) * h;
        const double y = (iy <= Lb / 2 ? iy : iy - Lb) * h;
        const double z = (iz <= Lb / 2 ? iz : iz - Lb) * h;
        const double d2 = x * x + y * y + z * z;
        const double r = sqrt(d2 + eps2), q = r / sigma;
        const double chi = taper((sqrt(d2) - r1) / (r2 - r1));
        double v;
        if (c == 3) {
            v = r * erf(q) + spi * exp(-q * q);
        } else {
            const double e_over_r = r > 0.0 ? erf(q) / r : 2.0 * 0.56418958354775628 / sigma;
            v = (c == 0 ? x : (c == 1 ? y : z)) * e_over_r;
        }
        out[e] = v * chi;
    }
}

// One axis of the deconvolution: divide the spectrum of every 1-D line by
// sinc(f)^8, the squared transform of the cubic B-spline window along that
// axis (f = frequency index / Lb in cycles per sample).  Element e holds
// frequency (e / inner) % nf.
__global__ void deconvolve_axis_kernel(cufftDoubleComplex *k, int64_t n, int64_t inner, int nf,
                                       int Lb)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)((e / inner) % nf);
        if (f == 0) continue;
        const double t = 3.14159265358979323846 * f / Lb;
        const double s = sin(t) / t, s2 = s * s, s4 = s2 * s2;
        const double w = s4 * s4;
        k[e].x /= w;
        k[e].y /= w;
    }
}

// Offset index of the L = 2M box (residue order; index M unused) -> index
// of the Lb box, or -1 for the unused index.
__device__ __forceinline__ int small_to_big(int i, int M, int Lb)
{
    if (i == M) return -1;
    const int m = i < M ? i : i - 2 * M;
    return (m + Lb) % Lb;
}

// Pass 1 (x): src[zz][y][x] (x over Lb) -> a1[z0 + zz][y][xs] (xs over 2M).
__global__ void keep_x_kernel(double *a1, const double *src, int z0, int nz, int Lb, int M)
{
    const int L = 2 * M;
    const int64_t total = (int64_t)nz * Lb * L;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int xs = (int)(e % L);
        const int64_t row = e / L;                       // zz * Lb + y
        const int bx = small_to_big(xs, M, Lb);
        a1[((int64_t)z0 * Lb) * L + e] = bx < 0 ? 0.0 : src[row * Lb + bx];
    }
}

// Pass 2 (y): plane src[y][x] (y over Lb, x over 2M) -> a2[z][ys][x].
__global__ void keep_y_kernel(double *a2, const double *src, int z, int Lb, int M)
{
    const int L = 2 * M;
    const int64_t total = (int64_t)L * L;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(e % L), ys = (int)(e / L);
        const int by = small_to_big(ys, M, Lb);
        a2[(int64_t)z * L * L + e] = by < 0 ? 0.0 : src[(int64_t)by * L + x];
    }
}

// Pass 3 (z): plane src[z][x] (z over Lb, x over 2M) for row ys -> the
// float L box out[zs][ys][x], scaled.
__global__ void keep_z_kernel(float *out, const double *src, int ys, int Lb, int M, double scale)
{
    const int L = 2 * M;
    const int64_t total = (int64_t)L * L;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(e % L), zs = (int)(e / L);
        const int bz = small_to_big(zs, M, Lb);
        out[((int64_t)zs * L + ys) * L + x] =
            bz < 0 ? 0.f : (float)(src[(int64_t)bz * L + x] * scale);
    }
}

// Cubic B-spline weights of the 4 nodes first .. first + 3 around mesh
// coordinate u (first = floor(u) - 1); u in double, weights in float.
__device__ __forceinline__ void bspline_weights(double u, int &first, float w[4])
{
    const double fl = floor(u);
    first = (int)fl - 1;
    const float f = (float)(u - fl), g = 1.f - f, f2 = f * f, f3 = f2 * f;
    w[0] = g * g * g * (1.f / 6.f);
    w[1] = (3.f * f3 - 6.f * f2 + 4.f) * (1.f / 6.f);
    w[2] = (-3.f * f3 + 3.f * f2 + 3.f * f + 1.f) * (1.f / 6.f);
    w[3] = f3 * (1.f / 6.f);
}

struct NodeWeights {
    int first[3];
    float w[3][4];
    bool ok;
};

__device__ __forceinline__ NodeWeights node_weights(float4 p, double x0, double inv_h, int M)
{
    NodeWeights nw;
    const double u[3] = {((double)p.x - x0) * inv_h, ((double)p.y - x0) * inv_h,
                         ((double)p.z - x0) * inv_h};
    nw.ok = true;
    for (int a = 0; a < 3; ++a) {
        const bool in = u[a] >= 1.0 && u[a] < (double)(M - 2);
        nw.ok = nw.ok && in;
        bspline_weights(in ? u[a] : 1.0, nw.first[a], nw.w[a]);
    }
    return nw;
}

// Unit charges of the samples on the M^3 charge mesh (fixed point).
__global__ void spread_kernel(const float4 *__restrict__ pos, int64_t N, unsigned long long *Q,
                              double x0, double inv_h, int M, int *status)
{
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const NodeWeights nw = node_weights(pos[i], x0, inv_h, M);
        if (!nw.ok) {
            bad = 1;
            continue;
        }
        for (int c = 0; c < 4; ++c)
            for (int b = 0; b < 4; ++b) {
                const float wzy = nw.w[2][c] * nw.w[1][b];
                unsigned long long *row =
                    Q + ((int64_t)(nw.first[2] + c) * M + (nw.first[1] + b)) * M + nw.first[0];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const long long v = __double2ll_rn((double)(wzy * nw.w[0][a]) * kFix);
                    if (v) atomicAdd(row + a, (unsigned long long)v);
                }
            }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kDevRange);
}

// Fixed-point charges -> the zero-padded real L^3 box.
__global__ void charges_to_box_kernel(const unsigned long long *__restrict__ Q, float *box, int M,
                                      int L)
{
    const int64_t total = (int64_t)L * L * L;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(e % L), iy = (int)((e / L) % L), iz = (int)(e / ((int64_t)L * L));
        float v = 0.f;
        if (ix < M && iy < M && iz < M)
            v = (float)((double)(long long)Q[((int64_t)iz * M + iy) * M + ix] * (1.0 / kFix));
        box[e] = v;
    }
}

// out = a * b (complex), n elements.
__global__ void spectrum_product_kernel(cufftComplex *out, const cufftComplex *__restrict__ a,
                                        const cufftComplex *__restrict__ b, int64_t n)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const cufftComplex x = a[e], y = b[e];
        out[e] = make_cuFloatComplex(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
    }
}

// Long-range sums gathered from the convolved fields (L^3 boxes; node n of
// the mesh is box index n) -- the force x, y, z fields, or the potential
// field alone for the energy -- plus the short-range fixed-point sums
// ([N][3] or [N][1]): out = S + L.
template <bool ENERGY>
__global__ void gather_kernel(const float4 *__restrict__ pos, int64_t N,
                              const float *__restrict__ phi, int64_t box, int L, double x0,
                              double inv_h, int M, const unsigned long long *__restrict__ shortr,
                              dacc4 *out)
{
    constexpr int NC = ENERGY ? 1 : 3;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const NodeWeights nw = node_weights(pos[i], x0, inv_h, M);
        float acc[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) acc[k] = 0.f;
        if (nw.ok) {
            for (int c = 0; c < 4; ++c)
                for (int b = 0; b < 4; ++b) {
                    const float wzy = nw.w[2][c] * nw.w[1][b];
                    const int64_t row = ((int64_t)(nw.first[2] + c) * L + (nw.first[1] + b)) * L +
                                        nw.first[0];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const float w = wzy * nw.w[0][a];
#pragma unroll
                        for (int k = 0; k < NC; ++k)
                            acc[k] = fmaf(w, __ldg(phi + k * box + row + a), acc[k]);
                    }
                }
        }
        dacc4 r;
        if (ENERGY) {
            r.x = r.y = r.z = 0.0;
            r.w = (double)(long long)shortr[i] * (1.0 / kFix) + (double)acc[0];
        } else {
            r.x = (double)(long long)shortr[3 * i] * (1.0 / kFix) + (double)acc[0];
            r.y = (double)(long long)shortr[3 * i + 1] * (1.0 / kFix) + (double)acc[NC > 1 ? 1 : 0];
            r.z = (double)(long long)shortr[3 * i + 2] * (1.0 / kFix) + (double)acc[NC > 2 ? 2 : 0];
            r.w = 0.0;
        }
        out[i] = r;
    }
}

// ---- short-range part ------------------------------------------------------

__device__ __forceinline__ int cell_coord(float x, float x0, float inv_cs, int nc)
{
    int c = (int)floorf((x - x0) * inv_cs);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void cell_keys_kernel(const float4 *__restrict__ pos, int64_t N, float x0, float inv_cs,
                                 int nc, unsigned int *keys, int *vals)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = pos[i];
        const int cx = cell_coord(p.x, x0, inv_cs, nc), cy = cell_coord(p.y, x0, inv_cs, nc),
                  cz = cell_coord(p.z, x0, inv_cs, nc);
        keys[i] = (unsigned int)((cz * nc + cy) * nc + cx);
        vals[i] = (int)i;
    }
}

// Cell ranges [start, end) of the sorted keys (cells without samples keep
// start = end = 0) and the samples' positions in sorted order.
__global__ void cell_ranges_kernel(const unsigned int *__restrict__ keys,
                                   const int *__restrict__ idx, const float4 *__restrict__ pos,
                                   int64_t N, int *start, int *end, float4 *spos)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const unsigned int c = keys[k];
        if (k == 0 || keys[k - 1] != c) start[c] = (int)k;
        if (k == N - 1 || keys[k + 1] != c) end[c] = (int)(k + 1);
        spos[k] = pos[idx[k]];
    }
}

// erfc(x), x >= 0: Abramowitz & Stegun 7.1.26 polynomial in t = 1/(1 + p x)
// times exp(-x^2) (returned separately, the energy needs it too).
__device__ __forceinline__ float erfc_as(float x, float &gauss)
{
    const float t = __frcp_rn(fmaf(0.3275911f, x, 1.f));
    float poly = fmaf(t, 1.061405429f, -1.453152027f);
    poly = fmaf(t, poly, 1.421413741f);
    poly = fmaf(t, poly, -0.284496736f);
    poly = fmaf(t, poly, 0.254829592f);
    gauss = __expf(-x * x);
    return t * poly * gauss;
}

// Cells have side >= rc / kCellReach, so the pairs closer than rc lie in the
// (2 kCellReach + 1)^3 cells around a sample's cell (smaller cells: fewer
// candidate pairs beyond rc).
constexpr int kCellReach = 3;
constexpr int kRowSpan = 2 * kCellReach + 1;
constexpr int kRows = kRowSpan * kRowSpan;

// Sorted range [j0, j1) of the sources in row r (0 .. kRows-1: dz, dy in
// -kCellReach .. kCellReach) of the cells around cell (cx, cy, cz): the
// x-neighbours of a row are consecutive cells, so their samples are one
// contiguous range.
__device__ __forceinline__ bool row_range(int cx, int cy, int cz, int r, int nc,
                                          const int *__restrict__ start,
                                          const int *__restrict__ end, int &j0, int &j1)
{
    const int z = cz + r / kRowSpan - kCellReach, y = cy + r % kRowSpan - kCellReach;
    if (z < 0 || z >= nc || y < 0 || y >= nc) return false;
    const int xa = cx >= kCellReach ? cx - kCellReach : 0;
    const int xb = cx < nc - kCellReach ? cx + kCellReach : nc - 1;
    const int base = (z * nc + y) * nc;
    j0 = -1;
    for (int x = xa; x <= xb; ++x) {
        const int s = start[base + x], e = end[base + x];
        if (s < e) {
            if (j0 < 0) j0 = s;
            j1 = e;
        }
    }
    return j0 >= 0;
}

constexpr int kShortThreads = 128;               // 4 warps, each takes its own items
constexpr int kShortChunk = 64;                  // targets per item (2 per lane of a warp)
constexpr int kShortSlice = 4096;                // sources per item at most

// Items of cell c: ceil(n_c / kShortChunk) target chunks times the source
// slices of its kRows rows.
__global__ void count_items_kernel(const int *__restrict__ start, const int *__restrict__ end,
                                   int nc, int *counts, int *slices)
{
    const int ncell = nc * nc * nc;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        const int n = end[c] - start[c];
        int cnt = 0, sl = 0;
        if (n > 0) {
            const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
            for (int r = 0; r < kRows; ++r) {
                int j0, j1;
                if (row_range(cx, cy, cz, r, nc, start, end, j0, j1))
                    sl += (j1 - j0 + kShortSlice - 1) / kShortSlice;
            }
            cnt = ((n + kShortChunk - 1) / kShortChunk) * sl;
        }
        counts[c] = cnt;
        slices[c] = sl;
    }
}

// The short-range work list, numbered on the device: cell c owns items
// [offsets[c], offsets[c] + counts[c]) (an exclusive scan of the counts),
// ceil(n_c / kShortChunk) target chunks times slices[c] source slices of
// its neighbour rows.  The kernels read its length on the device: the items
// below the stored list's capacity are written by fill_items_kernel (one
// thread per item) and read by the short-range kernel, which decodes any
// item beyond the capacity itself.
// Item u -> (targets t0, tn; sources s0, sn), all sorted positions.
__device__ int4 item_at(int64_t u, const int *__restrict__ offsets, const int *__restrict__ slices,
                        const int *__restrict__ start, const int *__restrict__ end, int nc)
{
    const int ncell = nc * nc * nc;
    int lo = 0, hi = ncell - 1;                // largest c with offsets[c] <= u
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)offsets[mid] <= u) lo = mid;
        else hi = mid - 1;
    }
    const int c = lo;
    const int local = (int)(u - offsets[c]), sl = slices[c];
    int4 it = make_int4(0, 0, 0, 0);
    if (sl <= 0 || local < 0) return it;
    const int k = local / sl;
    int rs = local % sl;
    const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
    it.x = start[c] + k * kShortChunk;
    it.y = min(kShortChunk, end[c] - it.x);
    for (int r = 0; r < kRows; ++r) {
        int j0, j1;
        if (!row_range(cx, cy, cz, r, nc, start, end, j0, j1)) continue;
        const int ns = (j1 - j0 + kShortSlice - 1) / kShortSlice;
        if (rs < ns) {
            it.z = j0 + rs * kShortSlice;
            it.w = min(kShortSlice, j1 - it.z);
            break;
        }
        rs -= ns;
    }
    return it;
}

// The list's length, and its first `cap` items stored (grid-stride).
__global__ void fill_items_kernel(const int *__restrict__ counts, const int *__restrict__ offsets,
                                  const int *__restrict__ slices, const int *__restrict__ start,
                                  const int *__restrict__ end, int nc, int64_t cap, int4 *items,
                                  long long *total_out)
{
    const int ncell = nc * nc * nc;
    const int64_t total = (int64_t)offsets[ncell - 1] + counts[ncell - 1];
    if (blockIdx.x == 0 && threadIdx.x == 0) *total_out = total;
    const int64_t n = total < cap ? total : cap;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x)
        items[u] = item_at(u, offsets, slices, start, end, nc);
}

// Short-range pair term of target p and source q, added to f (force) or
// f[0] (energy): pairs with |d| < rc only; the self pair adds nothing to the
// force and g_short(0) to the energy.
template <bool ENERGY>
__device__ __forceinline__ void short_pair(const float4 p, const float4 q, float rc2,
                                           float inv_sigma, float spi, float eps2, float *f)
{
    const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (d2 < rc2) {
        const float re2 = d2 + eps2;
        const float ri = rsqrt_sfu(fmaxf(re2, kEps2));
        const float r = re2 * ri;
        float gauss;
        const float ec = erfc_as(r * inv_sigma, gauss);
        if (ENERGY) {
            f[0] += fmaf(r, ec, -spi * gauss);
        } else {
            const float w = ec * ri;
            f[0] = fmaf(dx, w, f[0]);
            f[1] = fmaf(dy, w, f[1]);
            f[2] = fmaf(dz, w, f[2]);
        }
    }
}

// One item: targets [it.x, it.x + it.y) (two per lane) against sources
// [it.z, it.z + it.w) of the sorted positions, the sums added to the targets'
// fixed-point accumulators.
template <bool ENERGY>
__device__ __forceinline__ void short_item(const int4 it, int lane, const float4 *__restrict__ spos,
                                           const int *__restrict__ idx, float rc2, float inv_sigma,
                                           float spi, float eps2, unsigned long long *acc)
{
    constexpr int NV = ENERGY ? 1 : 3;
    float4 p[2];
    bool ok[2];
    float f[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    for (int t = 0; t < 2; ++t) {
        const int l = lane + 32 * t;
        ok[t] = l < it.y;
        p[t] = ok[t] ? spos[it.x + l] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float4 *src = spos + it.z;
#pragma unroll 4
    for (int j = 0; j < it.w; ++j) {
        const float4 q = __ldg(src + j);
        short_pair<ENERGY>(p[0], q, rc2, inv_sigma, spi, eps2, f[0]);
        short_pair<ENERGY>(p[1], q, rc2, inv_sigma, spi, eps2, f[1]);
    }
    for (int t = 0; t < 2; ++t) {
        if (!ok[t]) continue;
        unsigned long long *a = acc + (int64_t)idx[it.x + lane + 32 * t] * NV;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const long long x = __float2ll_rn(f[t][v] * 4294967296.0f);
            if (x) atomicAdd(a + v, (unsigned long long)x);
        }
    }
}

// Persistent warps take items from a queue: kShortChunk targets of one cell
// (two per lane) against up to kShortSlice sources of one neighbour row.
// The lanes of a warp read the same source at the same time (one broadcast
// load serves 64 pairs); the item sums are added to the targets' 64-bit
// fixed-point accumulators (exact, order-free).  Small items keep the lanes
// busy where cells hold few samples.  The length of the list is read on the
// device; items below `cap` come from the stored list, the rest are decoded
// here: nothing about the work list goes through the host, so an evaluation
// can be captured in a CUDA graph.
template <bool ENERGY>
__global__ void __launch_bounds__(kShortThreads) short_items_kernel(
    const int4 *__restrict__ items, int64_t cap, const int *__restrict__ counts,
    const int *__restrict__ offsets, const int *__restrict__ slices, const int *__restrict__ start,
    const int *__restrict__ end, int nc, unsigned int *queue, const float4 *__restrict__ spos,
    const int *__restrict__ idx, float rc2, float inv_sigma, float spi, float eps2,
    unsigned long long *acc)
{
    const int lane = threadIdx.x & 31;
    const int ncell = nc * nc * nc;
    const int64_t total = (int64_t)offsets[ncell - 1] + counts[ncell - 1];
    for (;;) {
        int64_t u = 0;
        if (lane == 0) u = atomicAdd(queue, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= total) break;
        int4 it;
        if (u < cap) {
            it = items[u];
        } else {                               // beyond the stored list: decode it here
            if (lane == 0) it = item_at(u, offsets, slices, start, end, nc);
            it.x = __shfl_sync(0xffffffffu, it.x, 0);
            it.y = __shfl_sync(0xffffffffu, it.y, 0);
            it.z = __shfl_sync(0xffffffffu, it.z, 0);
            it.w = __shfl_sync(0xffffffffu, it.w, 0);
        }
        if (it.y > 0 && it.w > 0)
            short_item<ENERGY>(it, lane, spos, idx, rc2, inv_sigma, spi, eps2, acc);
    }
}

} // namespace

// ---- host side ---------------------------------------------------------------

namespace {

bool seven_smooth(int n)
{
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

template <typename T> cudaError_t grow(T *&p, size_t &cap, size_t bytes)
{
    if (bytes <= cap) return cudaSuccess;
    cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
}

} // namespace

struct MeshState {
    MeshConfig cfg;          // the mesh the spectra were built for
    bool built = false;
    int M = 0, L = 0, nc = 0;
    double x0 = 0.0;
    cufftComplex *spectra = nullptr;   // 4 kernel spectra on the L box (scaled by 1/L^3)
    size_t spectra_cap = 0;
    cufftHandle r2c = 0, c2r = 0;
    bool plans = false;
    // evaluation buffers (grow with N)
    unsigned long long *Q = nullptr; size_t Q_cap = 0;
    float *box = nullptr; size_t box_cap = 0;           // charges, then 4 fields
    cufftComplex *qhat = nullptr; size_t qhat_cap = 0;
    cufftComplex *tmp = nullptr; size_t tmp_cap = 0;
    unsigned int *keys = nullptr; size_t keys_cap = 0;   // 2N keys, 2N values
    int *vals = nullptr; size_t vals_cap = 0;
    int *ranges = nullptr; size_t ranges_cap = 0;        // start[nc^3], end[nc^3]
    float4 *spos = nullptr; size_t spos_cap = 0;
    unsigned long long *shortr = nullptr; size_t shortr_cap = 0;   // fixed point [N][3]
    int *cellwork = nullptr; size_t cellwork_cap = 0;   // counts, slices, offsets [ncell] each
    int4 *items = nullptr; size_t items_cap = 0;        // the stored part of the work list
    int64_t items_n = -1;                               // the sample count it was sized for
    unsigned long long *dsmall = nullptr;               // [0]: item queue, [1]: list length
    int short_ctas[2] = {0, 0};                         // persistent CTAs (gradient, energy)
    void *cub = nullptr; size_t cub_cap = 0;
};

MeshState *mesh_state_create() { return new MeshState(); }

void mesh_state_destroy(MeshState *m)
{
    if (!m) return;
    if (m->plans) { cufftDestroy(m->r2c); cufftDestroy(m->c2r); }
    cudaFree(m->spectra); cudaFree(m->Q); cudaFree(m->box); cudaFree(m->qhat); cudaFree(m->tmp);
    cudaFree(m->keys); cudaFree(m->vals); cudaFree(m->ranges); cudaFree(m->spos);
    cudaFree(m->shortr); cudaFree(m->cub); cudaFree(m->cellwork); cudaFree(m->items);
    cudaFree(m->dsmall);
    delete m;
}

int mesh_guard(int n_cells)
{
    int g = 4;
    while (!seven_smooth(n_cells + 2 * g)) ++g;
    return g;
}

bool mesh_matches(const MeshState *m, const MeshConfig &c)
{
    return m->built && m->cfg.n_cells == c.n_cells && m->cfg.lo == c.lo && m->cfg.hi == c.hi &&
           m->cfg.sigma == c.sigma && m->cfg.rc == c.rc && m->cfg.eps == c.eps;
}

// Kernel spectra and FFT plans of mesh c (blocking; allocates the 4M box for
// the duration of the call).
cudaError_t mesh_build(MeshState *m, const MeshConfig &c, int sms, cudaStream_t st,
                       const char **what)
{
    m->built = false;
    const int g = mesh_guard(c.n_cells);
    const int M = c.n_cells + 2 * g, L = 2 * M, Lb = 4 * M, nf = Lb / 2 + 1;
    const double h = (c.hi - c.lo) / c.n_cells;
    const int64_t nl = (int64_t)L * L * L, nlc = (int64_t)L * L * (L / 2 + 1);
    // The deconvolution divides by a product of one factor per axis, so it
    // runs as three passes of 1-D transforms over the Lb = 4M box, each
    // keeping only the offsets |m| < M of its axis: pass 1 (x) on slabs of
    // kSlab planes of the kernel generated on the fly, pass 2 (y) per z
    // plane, pass 3 (z) per y row.  Peak memory: a1 = Lb * Lb * 2M and
    // a2 = Lb * 2M * 2M doubles (the full box would be Lb^3).
    constexpr int kSlab = 8;
    double *a1 = nullptr, *a2 = nullptr, *rbuf = nullptr;
    cufftDoubleComplex *cbuf = nullptr;
    float *small = nullptr;
    void *work = nullptr;
    cufftHandle px_f = 0, px_i = 0, py_f = 0, py_i = 0, pz_f = 0, pz_i = 0, sfwd = 0;
    bool made[7] = {false, false, false, false, false, false, false};
    cufftHandle *handles[7] = {&px_f, &px_i, &py_f, &py_i, &pz_f, &pz_i, &sfwd};
    cudaError_t err = cudaSuccess;
    auto done = [&](cudaError_t e) {
        for (int k = 0; k < 7; ++k)
            if (made[k]) cufftDestroy(*handles[k]);
        cudaFree(a1); cudaFree(a2); cudaFree(rbuf); cudaFree(cbuf); cudaFree(small);
        cudaFree(work);
        return e;
    };
    *what = "mesh kernel buffers";
    const size_t rbuf_n = std::max((size_t)kSlab * Lb * Lb, (size_t)Lb * L);
    const size_t cbuf_n = std::max((size_t)kSlab * Lb * nf, (size_t)nf * L);
    if ((err = grow(m->spectra, m->spectra_cap, (size_t)4 * nlc * sizeof(cufftComplex))) ||
        (err = cudaMalloc(&a1, (size_t)Lb * Lb * L * sizeof(double))) ||
        (err = cudaMalloc(&a2, (size_t)Lb * L * L * sizeof(double))) ||
        (err = cudaMalloc(&rbuf, rbuf_n * sizeof(double))) ||
        (err = cudaMalloc(&cbuf, cbuf_n * sizeof(cufftDoubleComplex))) ||
        (err = cudaMalloc(&small, nl * sizeof(float))))
        return done(err);
    *what = "mesh cuFFT plans";
    // 1-D plans: n = Lb; x: contiguous lines; y, z: lines of stride L (x the batch)
    int n1[1] = {Lb}, nfe[1] = {nf};
    size_t ws[7] = {0, 0, 0, 0, 0, 0, 0};
    auto many = [&](int k, int istride, int idist, int ostride, int odist, int batch, cufftType t,
                    bool real_in) {
        if (cufftCreate(handles[k]) != CUFFT_SUCCESS) return false;
        made[k] = true;
        int *inem = real_in ? n1 : nfe, *onem = real_in ? nfe : n1;
        return cufftSetAutoAllocation(*handles[k], 0) == CUFFT_SUCCESS &&
               cufftMakePlanMany(*handles[k], 1, n1, inem, istride, idist, onem, ostride, odist,
                                 t, batch, &ws[k]) == CUFFT_SUCCESS;
    };
    if (!many(0, 1, Lb, 1, nf, kSlab * Lb, CUFFT_D2Z, true) ||
        !many(1, 1, nf, 1, Lb, kSlab * Lb, CUFFT_Z2D, false) ||
        !many(2, L, 1, L, 1, L, CUFFT_D2Z, true) || !many(3, L, 1, L, 1, L, CUFFT_Z2D, false) ||
        !many(4, L * L, 1, L, 1, L, CUFFT_D2Z, true) || !many(5, L, 1, L, 1, L, CUFFT_Z2D, false))
        return done(cudaErrorUnknown);
    if (cufftCreate(&sfwd) != CUFFT_SUCCESS) return done(cudaErrorUnknown);
    made[6] = true;
    if (cufftSetAutoAllocation(sfwd, 0) != CUFFT_SUCCESS ||
        cufftMakePlan3d(sfwd, L, L, L, CUFFT_R2C, &ws[6]) != CUFFT_SUCCESS)
        return done(cudaErrorUnknown);
    *what = "mesh cuFFT work area";
    size_t wmax = 256;
    for (int k = 0; k < 7; ++k) wmax = std::max(wmax, ws[k]);
    if ((err = cudaMalloc(&work, wmax))) return done(err);
    for (int k = 0; k < 7; ++k)
        if (cufftSetWorkArea(*handles[k], work) != CUFFT_SUCCESS ||
            cufftSetStream(*handles[k], st) != CUFFT_SUCCESS)
            return done(cudaErrorUnknown);
    *what = "mesh kernel spectra";
    const double r1 = std::sqrt(3.0) * M * h, r2 = 2.0 * M * h;
    const double scale = 1.0 / ((double)Lb * Lb * Lb * (double)nl);
    for (int comp = 0; comp < 4; ++comp) {
        // pass 1: x lines of up to kSlab planes at a time (the plan always
        // transforms kSlab planes; rows past the last plane are not kept)
        for (int z0 = 0; z0 < Lb; z0 += kSlab) {
            const int nzz = std::min(kSlab, Lb - z0);
            const int64_t nr = (int64_t)nzz * Lb * Lb;
            fill_slab_kernel<<<grid_for(nr, sms), kMeshThreads, 0, st>>>(
                rbuf, Lb, z0, nzz, h, c.sigma, c.eps * c.eps, r1, r2, comp);
            if (cufftExecD2Z(px_f, rbuf, cbuf) != CUFFT_SUCCESS) return done(cudaErrorUnknown);
            deconvolve_axis_kernel<<<grid_for((int64_t)kSlab * Lb * nf, sms), kMeshThreads, 0, st>>>(
                cbuf, (int64_t)kSlab * Lb * nf, 1, nf, Lb);
            if (cufftExecZ2D(px_i, cbuf, rbuf) != CUFFT_SUCCESS) return done(cudaErrorUnknown);
            keep_x_kernel<<<grid_for((int64_t)nzz * Lb * L, sms), kMeshThreads, 0, st>>>(
                a1, rbuf, z0, nzz, Lb, M);
        }
        // pass 2: y lines of every z plane of a1
        for (int z = 0; z < Lb; ++z) {
            if (cufftExecD2Z(py_f, a1 + (int64_t)z * Lb * L, cbuf) != CUFFT_SUCCESS)
                return done(cudaErrorUnknown);
            deconvolve_axis_kernel<<<grid_for((int64_t)nf * L, sms), kMeshThreads, 0, st>>>(
                cbuf, (int64_t)nf * L, L, nf, Lb);
            if (cufftExecZ2D(py_i, cbuf, rbuf) != CUFFT_SUCCESS) return done(cudaErrorUnknown);
            keep_y_kernel<<<grid_for((int64_t)L * L, sms), kMeshThreads, 0, st>>>(a2, rbuf, z, Lb, M);
        }
        // pass 3: z lines of every y row of a2, into the float L box
        for (int ys = 0; ys < L; ++ys) {
            if (cufftExecD2Z(pz_f, a2 + (int64_t)ys * L, cbuf) != CUFFT_SUCCESS)
                return done(cudaErrorUnknown);
            deconvolve_axis_kernel<<<grid_for((int64_t)nf * L, sms), kMeshThreads, 0, st>>>(
                cbuf, (int64_t)nf * L, L, nf, Lb);
            if (cufftExecZ2D(pz_i, cbuf, rbuf) != CUFFT_SUCCESS) return done(cudaErrorUnknown);
            keep_z_kernel<<<grid_for((int64_t)L * L, sms), kMeshThreads, 0, st>>>(small, rbuf, ys, Lb,
                                                                                  M, scale);
        }
        if ((err = cudaGetLastError())) return done(err);
        if (cufftExecR2C(sfwd, small, m->spectra + comp * nlc) != CUFFT_SUCCESS)
            return done(cudaErrorUnknown);
    }
    if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return done(err);
    // evaluation plans on the L box
    *what = "mesh evaluation plans";
    if (m->plans) {
        cufftDestroy(m->r2c);
        cufftDestroy(m->c2r);
        m->plans = false;
    }
    if (cufftPlan3d(&m->r2c, L, L, L, CUFFT_R2C) != CUFFT_SUCCESS) return done(cudaErrorUnknown);
    if (cufftPlan3d(&m->c2r, L, L, L, CUFFT_C2R) != CUFFT_SUCCESS) {
        cufftDestroy(m->r2c);
        return done(cudaErrorUnknown);
    }
    m->plans = true;
    m->cfg = c;
    m->M = M;
    m->L = L;
    m->x0 = c.lo - g * h;
    const double span = M * h;
    m->nc = (int)std::floor(span * kCellReach / c.rc);
    if (m->nc < 1) m->nc = 1;
    if (m->nc > 512) m->nc = 512;
    m->built = true;
    *what = "";
    return done(cudaSuccess);
}

// Repulsion sums of the N packed samples into out[i] = (sum d/r, sum |d|_eps)
// over all j (directed, the self pair included as eps in the potential).
// Asynchronous: once the buffers have their size for N (the first call of a
// sample count allocates them and waits once for the length of its
// short-range work list), a call only enqueues work on `st` and can be
// captured.
// no_alloc (a call under stream capture): return cudaErrorStreamCaptureUnsupported
// instead of growing a buffer.
cudaError_t mesh_eval(MeshState *m, const float4 *pos, int64_t N, bool energy, dacc4 *out,
                      int *status, int sms, cudaStream_t st, const char **what, int *launches,
                      bool no_alloc)
{
    const MeshConfig &c = m->cfg;
    const int M = m->M, L = m->L, nc = m->nc;
    const int64_t nm = (int64_t)M * M * M, nl = (int64_t)L * L * L, nlc = (int64_t)L * L * (L / 2 + 1);
    const int nfield = energy ? 1 : 3;
    const int NV = energy ? 1 : 3;
    const int ncell = nc * nc * nc;
    const double h = (c.hi - c.lo) / c.n_cells;
    cudaError_t err;
    *what = "mesh evaluation buffers";
    size_t sort_bytes = 0, scan_bytes = 0;
    int end_bit = 1;
    while (((int64_t)1 << end_bit) < ncell) ++end_bit;
    cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, m->keys, m->keys, m->vals, m->vals,
                                    (int)N, 0, end_bit, st);
    cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, m->cellwork, m->cellwork, ncell, st);
    const size_t cub_bytes = std::max(sort_bytes, scan_bytes);
    if (no_alloc &&
        (nm * sizeof(unsigned long long) > m->Q_cap ||
         (size_t)(nfield + 1) * nl * sizeof(float) > m->box_cap ||
         nlc * sizeof(cufftComplex) > m->qhat_cap || nlc * sizeof(cufftComplex) > m->tmp_cap ||
         (size_t)2 * N * sizeof(unsigned int) > m->keys_cap ||
         (size_t)2 * N * sizeof(int) > m->vals_cap ||
         (size_t)2 * ncell * sizeof(int) > m->ranges_cap ||
         (size_t)N * sizeof(float4) > m->spos_cap ||
         (size_t)N * 3 * sizeof(unsigned long long) > m->shortr_cap ||
         (size_t)3 * ncell * sizeof(int) > m->cellwork_cap || cub_bytes + 256 > m->cub_cap ||
         !m->dsmall || !m->short_ctas[0] || m->items_n != N))
        return cudaErrorStreamCaptureUnsupported;

    if ((err = grow(m->Q, m->Q_cap, nm * sizeof(unsigned long long))) ||
        (err = grow(m->box, m->box_cap, (size_t)(nfield + 1) * nl * sizeof(float))) ||
        (err = grow(m->qhat, m->qhat_cap, nlc * sizeof(cufftComplex))) ||
        (err = grow(m->tmp, m->tmp_cap, nlc * sizeof(cufftComplex))) ||
        (err = grow(m->keys, m->keys_cap, (size_t)2 * N * sizeof(unsigned int))) ||
        (err = grow(m->vals, m->vals_cap, (size_t)2 * N * sizeof(int))) ||
        (err = grow(m->ranges, m->ranges_cap, (size_t)2 * ncell * sizeof(int))) ||
        (err = grow(m->spos, m->spos_cap, (size_t)N * sizeof(float4))) ||
        (err = grow(m->shortr, m->shortr_cap, (size_t)N * 3 * sizeof(unsigned long long))) ||
        (err = grow(m->cellwork, m->cellwork_cap, (size_t)3 * ncell * sizeof(int))) ||
        (err = grow(m->cub, m->cub_cap, cub_bytes + 256)))
        return err;
    if (!m->dsmall && (err = cudaMalloc(&m->dsmall, 2 * sizeof(unsigned long long)))) return err;
    if (!m->short_ctas[0]) {
        int a = 0, b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, short_items_kernel<false>, kShortThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, short_items_kernel<true>, kShortThreads, 0);
        m->short_ctas[0] = sms * std::max(a, 1);
        m->short_ctas[1] = sms * std::max(b, 1);
    }
    if (cufftSetStream(m->r2c, st) != CUFFT_SUCCESS || cufftSetStream(m->c2r, st) != CUFFT_SUCCESS)
        return cudaErrorUnknown;
    *what = "mesh evaluation";
    const int gN = grid_for(N, sms), gC = grid_for(ncell, sms);
    int nk = 0;
    // short-range part: samples sorted by cell, work items, pair sums
    const float cs = (float)(M * h / nc);
    cell_keys_kernel<<<gN, kMeshThreads, 0, st>>>(pos, N, (float)m->x0, 1.f / cs, nc, m->keys,
                                                  m->vals);
    if ((err = cub::DeviceRadixSort::SortPairs(m->cub, sort_bytes, m->keys, m->keys + N, m->vals,
                                               m->vals + N, (int)N, 0, end_bit, st)))
        return err;
    if ((err = cudaMemsetAsync(m->ranges, 0, (size_t)2 * ncell * sizeof(int), st))) return err;
    int *start = m->ranges, *end = m->ranges + ncell;
    cell_ranges_kernel<<<gN, kMeshThreads, 0, st>>>(m->keys + N, m->vals + N, pos, N, start, end,
                                                    m->spos);
    int *counts = m->cellwork, *slices = counts + ncell, *offsets = slices + ncell;
    count_items_kernel<<<gC, kMeshThreads, 0, st>>>(start, end, nc, counts, slices);
    if ((err = cub::DeviceScan::ExclusiveSum(m->cub, scan_bytes, counts, offsets, ncell, st)))
        return err;
    unsigned int *queue = reinterpret_cast<unsigned int *>(m->dsmall);
    long long *d_total = reinterpret_cast<long long *>(m->dsmall + 1);
    if (!no_alloc && m->items_n != N) {
        // The first evaluation of a sample count sizes the stored list: it
        // waits once for the list's length and keeps room for half as many
        // again (the list changes as the samples move; any items beyond the
        // room are decoded by the short-range kernel).  The list is not
        // reallocated while the sample count stays the same.
        fill_items_kernel<<<1, 32, 0, st>>>(counts, offsets, slices, start, end, nc, 0, nullptr,
                                            d_total);
        ++nk;
        long long total = 0;
        if ((err = cudaMemcpyAsync(&total, d_total, sizeof(long long), cudaMemcpyDeviceToHost, st)) ||
            (err = cudaStreamSynchronize(st)))
            return err;
        const size_t want = (size_t)std::max<long long>(total, 0);
        const size_t bytes = (want + want / 2 + 1024) * sizeof(int4);
        cudaFree(m->items);
        m->items = nullptr;
        m->items_cap = 0;
        m->items_n = -1;
        if ((err = cudaMalloc(&m->items, bytes))) return err;
        m->items_cap = bytes;
        m->items_n = N;
    }
    const int64_t cap = (int64_t)(m->items_cap / sizeof(int4));
    if ((err = cudaMemsetAsync(queue, 0, sizeof(unsigned int), st))) return err;
    fill_items_kernel<<<grid_for(std::max<int64_t>(cap, 1), sms), kMeshThreads, 0, st>>>(
        counts, offsets, slices, start, end, nc, cap, m->items, d_total);
    if ((err = cudaMemsetAsync(m->shortr, 0, (size_t)N * NV * sizeof(unsigned long long), st)))
        return err;
    const float rc2 = (float)(c.rc * c.rc), inv_sigma = (float)(1.0 / c.sigma);
    const float spi = (float)(c.sigma * 0.56418958354775628);
    const float eps2 = (float)(c.eps * c.eps);
    if (energy)
        short_items_kernel<true><<<m->short_ctas[1], kShortThreads, 0, st>>>(
            m->items, cap, counts, offsets, slices, start, end, nc, queue, m->spos, m->vals + N,
            rc2, inv_sigma, spi, eps2, m->shortr);
    else
        short_items_kernel<false><<<m->short_ctas[0], kShortThreads, 0, st>>>(
            m->items, cap, counts, offsets, slices, start, end, nc, queue, m->spos, m->vals + N,
            rc2, inv_sigma, spi, eps2, m->shortr);
    nk += 6;
    // long-range part
    if ((err = cudaMemsetAsync(m->Q, 0, nm * sizeof(unsigned long long), st))) return err;
    spread_kernel<<<gN, kMeshThreads, 0, st>>>(pos, N, m->Q, m->x0, 1.0 / h, M, status);
    charges_to_box_kernel<<<grid_for(nl, sms), kMeshThreads, 0, st>>>(m->Q, m->box, M, L);
    if (cufftExecR2C(m->r2c, m->box, m->qhat) != CUFFT_SUCCESS) return cudaErrorUnknown;
    for (int k = 0; k < nfield; ++k) {
        const int comp = energy ? 3 : k;
        spectrum_product_kernel<<<grid_for(nlc, sms), kMeshThreads, 0, st>>>(
            m->tmp, m->qhat, m->spectra + comp * nlc, nlc);
        if (cufftExecC2R(m->c2r, m->tmp, m->box + (1 + k) * nl) != CUFFT_SUCCESS)
            return cudaErrorUnknown;
    }
    if (energy)
        gather_kernel<true><<<gN, kMeshThreads, 0, st>>>(pos, N, m->box + nl, nl, L, m->x0,
                                                         1.0 / h, M, m->shortr, out);
    else
        gather_kernel<false><<<gN, kMeshThreads, 0, st>>>(pos, N, m->box + nl, nl, L, m->x0,
                                                          1.0 / h, M, m->shortr, out);
    nk += 3 + nfield + 1;
    *launches = nk;
    *what = "";
    return cudaGetLastError();
}

} // namespace sparkling
