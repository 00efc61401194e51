// Internal interface between the C-ABI layer (api.cu) and the kernel files
// (pairs.cu, repulsion.cu, repulsion_sym.cu, project.cu, engine.cu,
// field.cu, mesh.cu, driver.cu).  Not installed; not part of the ABI.
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace sparkling {

constexpr int kTile = 1024;            // targets per tile (one CTA's targets)
constexpr int kThreads = 256;          // threads per CTA of the engine and the default shapes
constexpr int kStages = 3;             // TMA pipeline depth
constexpr int kStageFloats = 4096;     // 16 KB per stage
constexpr int kSrcBlock = kStageFloats / 4;  // repulsion sources per stage (float4)
constexpr int kMaxNx = kStageFloats;   // longest grid row a stage can hold
constexpr float kEps2 = 1e-30f;        // smallest eps^2 added to every r^2 (zero-distance guard)

// Device status bits (OR-ed into the context's status word).
constexpr int kDevNonFinite = 1;
constexpr int kDevTimeout = 2;
constexpr int kDevRange = 4;            // a sample outside the fast-repulsion mesh

// Default budget of a bounded device wait, in SM clock cycles (~2 s at 2 GHz).
constexpr long long kWaitCycles = 4000000000LL;

// Device control block of a context: the status word the kernels OR their
// error bits into and, behind it, the budget of their bounded waits.  Every
// `int *status` a kernel receives points at the first member of one of these.
struct DevCtl {
    int status;
    int reserved;
    long long wait_cycles;   // budget of a bounded wait (cycles); the drains after a timeout use kWaitCycles
};

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

// Upper triangle of tile pairs (I, J), 0 <= I <= J < T, numbered row by row:
// row I holds T - I pairs and starts at tri_row_start(I, T).
__host__ __device__ inline int64_t tri_row_start(int64_t I, int64_t T)
{
    return I * T - I * (I - 1) / 2;
}

__host__ __device__ inline int64_t tri_count(int64_t T) { return T * (T + 1) / 2; }

// (I, J) of pair number u (0 <= u < tri_count(T)).
__host__ __device__ inline void tri_pair(int64_t u, int64_t T, int64_t &I, int64_t &J)
{
    const double b = 2.0 * (double)T + 1.0;
    double d = b * b - 8.0 * (double)u;
    d = d > 0.0 ? d : 0.0;
    int64_t i = (int64_t)((b - sqrt(d)) * 0.5);
    if (i < 0) i = 0;
    if (i > T - 1) i = T - 1;
    while (i + 1 <= T - 1 && tri_row_start(i + 1, T) <= u) ++i;
    while (i > 0 && tri_row_start(i, T) > u) --i;
    I = i;
    J = i + (u - tri_row_start(i, T));
}

// Fixed-point scale of the symmetric repulsion's integer accumulators: a sum
// is kept as round(x * 2^32) in an int64 (exact, order-independent addition).
constexpr double kFixScale = 4294967296.0;

// One trajectory of a batched symmetric repulsion: samples [off, off + N)
// of pos / acc, its tiles and the first global unit of its triangle.
struct SymTraj {
    int64_t off, N, tiles, unit0;
};

struct SymArgs {
    const float4 *pos;          // packed samples [N] (all trajectories when traj is set)
    int64_t N;
    int64_t tiles;              // ceil(N / kTile)
    int64_t ctas;               // persistent CTAs; the units are split evenly
    unsigned long long *acc;    // [N][NV] fixed-point sums (zeroed before the launch)
    const SymTraj *traj = nullptr;   // batched: B trajectories (device), else one (N, tiles)
    int32_t B = 1;
    int64_t units = 0;          // batched: total units of all triangles
    float eps2 = kEps2;         // kernel sqrt(r^2 + eps^2): eps^2 (>= kEps2) added to every r^2
    int *status;
};

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
    float eps2 = kEps2;   // eps^2 (>= kEps2) added to every r^2
    int *status;
};

struct RepArgs {
    const float4 *pos;    // packed samples [N] (targets and sources)
    int64_t N;
    Split sp;             // per_tile = ceil(N / kSrcBlock) source blocks
    dacc4 *part;
    float eps2 = kEps2;   // eps^2 (>= kEps2) added to every r^2
    int *status;
};

struct CombineArgs {
    int64_t N;
    const dacc4 *part_a;
    const dacc4 *part_r;
    Split spa, spr;
    void *G, *A, *R;      // outputs [N][3] (A, R may be null)
    double *G64;          // optional FP64 copy of G [N][3]
    const unsigned long long *racc;   // symmetric repulsion sums [N][NV] (replaces part_r)
    const dacc4 *a_direct;            // attraction per target [N] (replaces part_a), or null
    const dacc4 *r_direct;            // repulsion sums per target [N] (replaces racc/part_r), or null
    double scale;         // G, A, R are multiplied by scale * (*scale_dev if set)
    const double *scale_dev;
    double2 *energy_blocks;  // energy mode: per-block (sum ea, sum er)
    double eps;           // regularisation: the N self pairs (|d| = eps each) leave F^r
};

// Tile shapes of the pair kernels, chosen per problem by the autotuner
// (api.cu).  Every shape keeps kTile targets per CTA; it trades threads per
// CTA against targets held in registers per thread (and, for the repulsion,
// the unroll of the source loop).
constexpr int kAttrVariants = 3;       // threads 128 / 256 / 512 (8 / 4 / 2 targets each)
constexpr int kRepVariants = 5;        // (threads, unroll) 128x2, 256x1, 256x2, 256x4, 512x2
constexpr int kAttrDefault = 1, kRepDefault = 2;
int attr_variant_threads(int v);
int rep_variant_threads(int v);
int rep_variant_unroll(int v);

// Launchers (pairs.cu, repulsion.cu).  dtype: 0 float, 1 double.
cudaError_t launch_pack_positions(const void *K, int dtype, int64_t N, float4 *out, int *status,
                                  int sms, cudaStream_t st);
cudaError_t launch_pack_grid(const float *rho, int nx, int ny, int nz, int gxp, double lo,
                             double hi, float *rho_out, float *coords, int *status, int sms,
                             cudaStream_t st);
size_t attraction_smem_bytes(int gxp);
int attraction_ctas_per_sm(int acc, bool energy, int variant);
cudaError_t launch_attraction(const AttrArgs &a, int acc, bool energy, int variant, cudaStream_t st);
size_t repulsion_smem_bytes();
int repulsion_ctas_per_sm(int acc, bool energy, int variant);
cudaError_t launch_repulsion(const RepArgs &a, int acc, bool energy, int variant, cudaStream_t st);
cudaError_t launch_combine(const CombineArgs &c, int out_dtype, int sms, cudaStream_t st);
// Symmetric repulsion (repulsion_sym.cu): every unordered pair once.
// Shapes: 256 threads (4 targets per lane) with 2 or 4 sources per lane and
// the targets paired (0, 1) or 2 sources paired (2); 128 threads (8 targets
// per lane), 2 sources paired (3).
constexpr int kSymVariants = 4;
constexpr int kSymDefault = 3;        // shape used where nothing was tuned or pinned
int sym_variant_sources(int v);
bool sym_variant_source_paired(int v);
int sym_variant_threads(int v);
size_t repulsion_sym_smem_bytes();
int repulsion_sym_ctas_per_sm(bool energy, int variant);
cudaError_t launch_repulsion_sym(const SymArgs &a, bool energy, int variant, cudaStream_t st);
int energy_blocks(int64_t N);
cudaError_t launch_combine_energy(const CombineArgs &c, double *out2, cudaStream_t st);

// Fast attraction (field.cu): node field of a density and its interpolation.
size_t field_bytes(int nx, int ny, int nz);
cudaError_t field_build(const float *rho, int nx, int ny, int nz, double lo, double hi, double eps,
                        float4 *field, int sms, cudaStream_t st, const char **what);
cudaError_t launch_interp(const float4 *pos, int64_t N, const float4 *field, int nx, int ny, int nz,
                          double lo, double hi, dacc4 *out, int sms, cudaStream_t st);

// Fast repulsion (mesh.cu): particle-particle particle-mesh summation.
struct MeshConfig {
    int n_cells;          // mesh cells across [lo, hi]
    double lo, hi;
    double sigma, rc;     // split width and short-range cut-off (absolute units)
    double eps;           // regularisation of the kernel
};
struct MeshState;
MeshState *mesh_state_create();
void mesh_state_destroy(MeshState *m);
int mesh_guard(int n_cells);
bool mesh_matches(const MeshState *m, const MeshConfig &c);
cudaError_t mesh_build(MeshState *m, const MeshConfig &c, int sms, cudaStream_t st,
                       const char **what);
// no_alloc: a call under stream capture; cudaErrorStreamCaptureUnsupported
// where a buffer would have to grow.
cudaError_t mesh_eval(MeshState *m, const float4 *pos, int64_t N, bool energy, dacc4 *out,
                      int *status, int sms, cudaStream_t st, const char **what, int *launches,
                      bool no_alloc);

// Multi-resolution driver (driver.cu).  dtype: 0 float, 1 double.
cudaError_t launch_upsample(const void *Kc, void *Kf, int dtype, int64_t Nc, int64_t d, int sms,
                            cudaStream_t st);
int bb_blocks(int64_t n, int sms);
cudaError_t launch_bb(const void *K, int dtype, double *Kp, const double *G, double *Gp, int64_t n,
                      bool dots, double2 *part, double *out, int sms, cudaStream_t st);

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
    int mixed;             // FP32 K, fixed iterations: iterate in FP32 on the displacement
    int *status;
    unsigned long long *viol;  // optional [4] (non-negative doubles as bits)
    int *notconv;          // optional count of shots that did not certify
};
size_t project_state_bytes(int Ns);   // 18 * Ns doubles
bool project_state_in_smem(int Ns);
int project_block(int Ns);
int project_ctas_per_sm(int dtype, int Ns);
cudaError_t launch_project(const ProjArgs &p, int dtype, int grid, cudaStream_t st);

// Persistent engine (engine.cu): one launch runs a work list of pair items
// (attraction or repulsion of one target tile against a run of grid rows or
// source blocks, or symmetric repulsion of one target tile against a run of
// source tiles) for any number of trajectories, followed by per-shot
// projection items that wait until their trajectory's pair items are done.
struct EngineTraj {
    int64_t off;             // first sample of the trajectory in K / pos
    int64_t N;               // samples
    int64_t part_off;        // first partial (dacc4 units) of this trajectory
    const float *rho;        // density rows padded to gxp, 16-byte aligned rows
    const float *coords;     // x[gxp], y[ny], z[nz]
    double x0;               // lo + h/2
    double eta;              // step size (G units)
    double alpha, beta, box;
    double pin[3];
    float hx;
    int32_t Nc, Ns;
    int32_t gxp, ny, nz, rows_per_stage;
    int32_t tiles, slots, a_chunks;   // slots per tile: a_chunks attraction + the rest repulsion
    int32_t n_pair_items;
    int32_t pin_index, n_iter;
};

constexpr int kItemAttraction = 0, kItemRepulsion = 1, kItemProject = 2, kItemSym = 3;
constexpr int kSmSlots = 512;         // per-SM counters of the role dispatch (%smid & 511)

struct EngineItem {
    int32_t kind, traj;
    int32_t tile, slot;      // pair items: target tile and partial slot; project: shot, -
    int64_t u0, u1;          // pair items: grid-row or source-block range; sym: source tiles
};

struct EngineArgs {
    const EngineTraj *traj;
    const EngineItem *items;
    int32_t n_items;
    int32_t proj_in_smem;    // projection state fits in the shared-memory union
    int32_t proj_mixed;      // FP32 K: the mixed-precision projection (else FP64 throughout)
    const float4 *pos;       // packed samples of all trajectories
    void *K;                 // [sum N][3], updated in place by the projection items
    dacc4 *part;
    unsigned int *queue;     // next item: [3] (see roles) (reset to 0 before every launch)
    unsigned int *done;      // [B] completed pair items per trajectory (reset to 0)
    // Role dispatch (one-launch shape): the list is attraction items
    // [0, n_attr), symmetric items [n_attr, n_attr + n_sym), then projection
    // items; queue[k] counts part k's dispensed items.  On every SM one CTA
    // in three takes symmetric items first and the others attraction items
    // first (sm_slots[kSmSlots] counts the CTAs that started on each SM);
    // projection items are taken once both pair parts are dispensed.
    int32_t roles = 0;
    int32_t n_attr = 0, n_sym = 0;
    unsigned int *sm_slots = nullptr;
    // A projection item waits for its trajectory's pair items up to
    // wait_scale times the context's wait budget (at least 4; more where the
    // largest pair item may take longer, see api.cu).
    int32_t wait_scale = 4;
    double *gstate;          // per-CTA projection state when it is not in shared memory
    unsigned long long *racc = nullptr;   // symmetric repulsion sums [sum N][3], or null
    float eps2 = kEps2;      // eps^2 (>= kEps2) added to every r^2
    int *status;
};

size_t engine_smem_bytes();
size_t engine_proj_smem_limit();     // largest 18*Ns*8 that fits the shared-memory union
constexpr int kEngineVariants = 2;    // threads 256 (repulsion unroll 4) / 512 (unroll 2)
// The one-launch shape: 128 threads (8 targets per thread, three CTAs per
// SM), whose work list also holds the symmetric repulsion (kItemSym items).
constexpr int kEngineOneLaunch = 2;
int engine_variant_threads(int v);
int engine_ctas_per_sm(int acc, int dtype, int variant);
cudaError_t launch_engine(const EngineArgs &e, int acc, int dtype, int variant, int ctas,
                          cudaStream_t st);

} // namespace sparkling
