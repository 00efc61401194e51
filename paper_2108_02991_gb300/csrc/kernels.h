// Internal interface between the C-ABI layer (api.cu) and the kernels
// (pairs.cu, project.cu).  Not installed; not part of the ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sparkling {

constexpr int kThreads = 256;          // threads per CTA of the pair kernels
constexpr int kTargetsPerThread = 4;   // register-blocked targets per thread
constexpr int kTile = kThreads * kTargetsPerThread;  // targets per tile
constexpr int kStages = 3;             // TMA pipeline depth
constexpr int kStageFloats = 4096;     // 16 KB per stage
constexpr int kSrcBlock = kStageFloats / 4;  // repulsion sources per stage (float4)
constexpr int kMaxNx = kStageFloats;   // longest grid row a stage can hold
constexpr float kEps2 = 1e-30f;        // added to every r^2 (zero-distance guard)

// Device status bits (OR-ed into the context's status word).
constexpr int kDevNonFinite = 1;
constexpr int kDevTimeout = 2;

// Four FP64 partial sums of one target: force (x, y, z) and energy (w).
struct __align__(32) dacc4 {
    double x, y, z, w;
};
__host__ __device__ inline dacc4 make_dacc4(double x, double y, double z, double w)
{
    dacc4 v;
    v.x = x; v.y = y; v.z = z; v.w = w;
    return v;
}

// Even split of `units` work units over `ctas` persistent CTAs, where a tile
// of targets owns `per_tile` consecutive units (grid rows or source blocks).
// CTA c processes units [begin(c), begin(c+1)); the CTAs that touch a tile
// write one partial each, in consecutive "slots".
struct Split {
    int64_t units;
    int64_t per_tile;
    int64_t ctas;
    int64_t slots;
};

__host__ __device__ inline int64_t split_begin(const Split &s, int64_t c)
{
    return s.units * c / s.ctas;
}

// The CTA whose range holds unit u (the largest c with begin(c) <= u).
__host__ __device__ inline int64_t split_cta_of(const Split &s, int64_t u)
{
    return ((u + 1) * s.ctas - 1) / s.units;
}

// Split of tiles * per_tile units over at most max_ctas CTAs.
inline Split make_split(int64_t tiles, int64_t per_tile, int64_t max_ctas)
{
    Split s;
    s.per_tile = per_tile;
    s.units = tiles * per_tile;
    s.ctas = max_ctas < s.units ? max_ctas : s.units;
    if (s.ctas < 1) s.ctas = 1;
    s.slots = (s.ctas + tiles - 1) / tiles + 1;
    return s;
}

struct AttrArgs {
    const float4 *tgt;    // packed targets (x, y, z, 0) [N]
    int64_t N;
    const float *rho;     // density rows, zero-padded to gxp: [ny*nz][gxp]
    const float *coords;  // xs[gxp], ys[ny], zs[nz] (cell centres, rounded to float)
    int gxp, ny, nz;
    int rows_per_stage;
    double x0;            // lo + h/2: x coordinate of grid column 0
    float hx;             // grid spacing along x (columns are x0 + q hx)
    Split sp;             // per_tile = ny*nz rows
    dacc4 *part;        // [tiles][slots][kTile] (x, y, z, energy)
    int *status;
};

struct RepArgs {
    const float4 *pos;    // packed samples [N] (targets and sources)
    int64_t N;
    Split sp;             // per_tile = ceil(N / kSrcBlock) source blocks
    dacc4 *part;
    int *status;
};

struct CombineArgs {
    int64_t N;
    const dacc4 *part_a;
    const dacc4 *part_r;
    Split spa, spr;
    void *G, *A, *R;      // outputs [N][3] (A, R may be null)
    double *G64;          // optional FP64 copy of G [N][3]
    double scale;         // G, A, R are multiplied by scale * (*scale_dev if set)
    const double *scale_dev;
    double2 *energy_blocks;  // energy mode: per-block (sum ea, sum er)
};

// Launchers (pairs.cu).  dtype: 0 float, 1 double.
cudaError_t launch_pack_positions(const void *K, int dtype, int64_t N, float4 *out, int *status,
                                  int sms, cudaStream_t st);
cudaError_t launch_pack_grid(const float *rho, int nx, int ny, int nz, int gxp, double lo,
                             double hi, float *rho_out, float *coords, int *status, int sms,
                             cudaStream_t st);
size_t attraction_smem_bytes(int gxp);
int attraction_ctas_per_sm(int acc, bool energy, int gxp);
cudaError_t launch_attraction(const AttrArgs &a, int acc, bool energy, cudaStream_t st);
size_t repulsion_smem_bytes();
int repulsion_ctas_per_sm(int acc, bool energy);
cudaError_t launch_repulsion(const RepArgs &a, int acc, bool energy, cudaStream_t st);
cudaError_t launch_combine(const CombineArgs &c, int out_dtype, int sms, cudaStream_t st);
int energy_blocks(int64_t N);
cudaError_t launch_combine_energy(const CombineArgs &c, double *out2, cudaStream_t st);

// Projection (project.cu).
struct ProjArgs {
    void *K;               // [Nc*Ns][3] in/out
    const double *G;       // optional gradient [Nc*Ns][3]: k = K - eta G
    double eta;
    int64_t Nc;
    int Ns;
    double alpha, beta, box, tol, margin;
    double pin[3];
    int pin_index, n_iter, check_every;
    double *gstate;        // per-CTA state in global memory (18 * Ns doubles) or null
    int *status;
    unsigned long long *viol;  // optional [4] (non-negative doubles as bits)
    int *notconv;          // optional count of shots that did not certify
};
size_t project_state_bytes(int Ns);   // 18 * Ns doubles
bool project_state_in_smem(int Ns);
int project_block(int Ns);
int project_ctas_per_sm(int dtype, int Ns);
cudaError_t launch_project(const ProjArgs &p, int dtype, int grid, cudaStream_t st);

} // namespace sparkling
