// Internal declarations of the BSGD library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bsgd.h"

namespace bsgd {

// ---------------------------------------------------------------------------
// Error reporting

void set_error(const std::string &msg);
bsgd_status fail(bsgd_status s, const std::string &msg);
// INVALID_ARG unless the calling thread's current CUDA device holds g's tables
// (every launch runs on the current device).
bsgd_status check_device(const bsgd_geometry *g);
bsgd_status cuda_fail(cudaError_t e, const char *what);

#define BSGD_CUDA(call)                                                    \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return ::bsgd::cuda_fail(e_, #call);        \
    } while (0)

#define BSGD_TRY(call)                                                     \
    do {                                                                   \
        bsgd_status s_ = (call);                                           \
        if (s_ != BSGD_OK) return s_;                                      \
    } while (0)

// ---------------------------------------------------------------------------
// Geometry tables (built on the host in FP64, stored in FP32 on the device)

// Ray of pixel (u, v) at one view, in voxel units relative to the volume's low
// corner: start = p0 + u * pu, end = c0 + u * cu + v * cv. For divergent beams
// the start is the source (pu = 0); for parallel beams both ends move with u.
struct ViewRay {
    float p0[3];
    float pu[3];
    float c0[3];
    float cu[3];
    float cv[3];
    float pad;
};
static_assert(sizeof(ViewRay) == 64, "ViewRay is 4 x float4");

// Detector rectangle [u0, u1] x [v0, v1] (inclusive; empty when u0 > u1).
struct Band {
    int u0, u1, v0, v1;
};

constexpr int kMaxPairs = 64;  // pairs per iteration the work list can hold

struct DeviceGeom {
    const ViewRay *rays;       // n_views
    const Band *bands;         // n_views x (N + 1); entry N = whole volume
    const int *block_views;    // M x max_views (padded with -1)
    const int *block_nviews;   // M
    const int *plane_start;    // N + 1 planes along the block axis
    const int *view_block;     // n_views
    const unsigned char *view_yfast;  // n_views: 1 if the view's rays run mostly along x
    // Compact band storage of the per-block sinograms z^j and r~^j: the rows of
    // view a inside block j's band (bands[a][j]) are stored from zoff[j][a] on,
    // v-major within the band; rows outside the band hold 0 and are not stored.
    const int64_t *zoff;       // N x n_views
    int64_t zlen;              // elements of one compact array (all blocks)
    int nx, ny, nz;
    float hx, hy, hz;
    int nu, nv, n_views;
    int M, N, axis, max_views;
    int64_t n_rows, n_cols;
    int plane_stride;          // voxels per plane along the block axis
};

}  // namespace bsgd

struct bsgd_geometry {
    bsgd_geometry_desc desc;   // angles / view_block point into the vectors below
    std::vector<double> angles;
    std::vector<int32_t> view_block;
    int M = 0, N = 0;
    int axis = 2;              // block axis: 1 = y, 2 = z
    int n_planes = 0;          // planes along the block axis
    std::vector<int> plane_start;               // N + 1
    std::vector<std::vector<int>> block_views;  // M lists
    int max_views = 0;
    std::vector<bsgd::ViewRay> rays;
    std::vector<bsgd::Band> bands;              // n_views x (N + 1), traversal bands
    std::vector<int> wband;                     // M x N x 2: exact v-band of the pair
    std::vector<int64_t> zoff;                  // N x n_views: compact band offsets
    std::vector<unsigned char> view_yfast;      // host copy of dg.view_yfast
    int64_t zlen = 0;
    int device = 0;
    // device copies
    bsgd::ViewRay *d_rays = nullptr;
    bsgd::Band *d_bands = nullptr;
    int *d_block_views = nullptr;
    int *d_block_nviews = nullptr;
    int *d_plane_start = nullptr;
    int *d_view_block = nullptr;
    unsigned char *d_view_yfast = nullptr;
    int64_t *d_zoff = nullptr;
    bsgd::DeviceGeom dg{};
    // Filled on first use by a solver state and kept for the geometry's life
    // (index: number of detector cells 1, 2 or 4): exact voxel-ray update
    // counts per (J, view, cell), and the geometric cell weights of Algorithm 2.
    mutable std::mutex cache_mu;
    mutable unsigned long long *d_counts[5] = {};
    mutable double *d_cw[5] = {};
    // Largest block Lipschitz estimate max ||A^J||^2 (STRIP) or max ||A_I^J||^2
    // (BLOCK) by power_iters power-iteration steps: a property of the geometry,
    // kept so that later states on it need no power iteration (key: rule,
    // power_iters).
    mutable std::map<std::pair<int, int>, double> lambda_cache;

    int64_t n_rows() const { return (int64_t)desc.n_views * desc.nv * desc.nu; }
    int64_t n_cols() const { return (int64_t)desc.nx * desc.ny * desc.nz; }
    int64_t block_cols(int j) const {
        return (int64_t)(plane_start[j + 1] - plane_start[j]) * dg.plane_stride;
    }
};

namespace bsgd {

// ---------------------------------------------------------------------------
// Projector launches (siddon.cu)

enum TraceMode : int {
    kFpPlain = 0,   // y = (y or 0) + A x
    kBpPlain = 1,   // x += scale A^T r
    kCount = 2,     // number of positive-length segments
};

struct PlainLaunch {
    const int *row_ids;  // host list of selected row-block ids
    int n_rb;
    int j0, j1;          // column blocks [j0, j1)
    int unused;
};

// Tiles of the largest band of these views for column blocks [j0, j1) (host
// side, from the geometry tables).
int tiles_for(const bsgd_geometry *g, const std::vector<int> &views, int j0, int j1, int tile_u,
              int tile_v);

// xT (optional): y-fastest copy of x over the launch's planes, gathered by the
// views whose rays run along x; gT (optional): y-fastest FP32 accumulator that
// those views scatter into instead of x (the caller adds it back with
// plain_add_transposed).
bsgd_status launch_fp_plain(const bsgd_geometry *g, const PlainLaunch &L, const void *x,
                            bsgd_dtype xt, void *y, bsgd_dtype yt, int accumulate,
                            cudaStream_t st, const void *xT = nullptr);
bsgd_status launch_bp_plain(const bsgd_geometry *g, const PlainLaunch &L, const void *r,
                            bsgd_dtype rt, float *x, float scale, cudaStream_t st,
                            float *gT = nullptr);
// True if a y-fastest copy pays for the listed row blocks: a volume with at
// least one view whose rays run along x.
bool plain_wants_transpose(const bsgd_geometry *g, const int *row_ids, int n_rb);
// xT[z][x][y] = x[z][y][x] over the planes of column blocks [j0, j1).
bsgd_status plain_transpose(const bsgd_geometry *g, const void *x, bsgd_dtype xt, void *xT, int j0,
                            int j1, cudaStream_t st);
// x[z][y][x] += gT[z][x][y] over the planes of column blocks [j0, j1).
bsgd_status plain_add_transposed(const bsgd_geometry *g, const float *gT, float *x, int j0, int j1,
                                 cudaStream_t st);
bsgd_status launch_count(const bsgd_geometry *g, const PlainLaunch &L,
                         unsigned long long *d_count, cudaStream_t st);
// Clear the rows of every view of the listed row blocks.
bsgd_status zero_rows(const bsgd_geometry *g, const int *row_ids, int n_rb, void *y,
                      bsgd_dtype yt, cudaStream_t st);

// Tile of rays per CTA.
constexpr int kTileU3 = 32, kTileV3 = 4;   // 3D: 4 warps, each 32 u of one detector row
constexpr int kTileU2 = 128, kTileV2 = 1;  // 2D: 4 warps of 32 u rays
inline int tile_u(const bsgd_geometry *g) { return g->desc.nv > 1 ? kTileU3 : kTileU2; }
inline int tile_v(const bsgd_geometry *g) { return g->desc.nv > 1 ? kTileV3 : kTileV2; }

// ---------------------------------------------------------------------------
// Small device helpers shared by host launchers

bsgd_status upload(void **dst, const void *src, size_t bytes);
size_t dtype_size(bsgd_dtype t);
bool dtype_ok(int t);

}  // namespace bsgd

namespace bsgd {

// ---------------------------------------------------------------------------
// Solver state shared by the solver kernels

// Device work list of one iteration, written by the sampler.
struct Work {
    int n_pairs;
    int pair_i[kMaxPairs], pair_j[kMaxPairs];
    int n_cols;                 // distinct column blocks of the pairs
    int cols[kMaxPairs];
    int n_rows;                 // distinct row blocks of the pairs
    int rows[kMaxPairs];
};

struct SolveDev {
    const void *y;     // n_rows, storage type
    void *z;           // N x n_rows, z^j (last FP of column block j)
    void *rt;          // N x n_rows, residual snapshots r~^j
    void *r;           // n_rows, r = y - sum_j z^j
    float *g;          // n_cols, aggregated gradient
    double *S;         // M x nv: sum over the row block's views and u of r^2
    const Work *work;
    const int *cells;  // kMaxPairs x max_views chosen cells (-1: whole view)
    int n_cells;       // 1 (no cells), 2 or 4
    const double *mu;  // step
    // y-fastest copies used by the views whose rays run mostly along x (3D
    // only; null otherwise): adjacent rays of a warp then gather and scatter
    // adjacent addresses
    void *xT;          // image, [z][x][y], storage type
    float *gT;         // their part of the aggregated gradient, [z][x][y]
    double *eud;       // Algorithm 3: effective update direction of the window (or null)
    // owner-computes sharding: 1 for the column blocks this process owns; the
    // FP, BP and update of a pair whose block it does not own are skipped
    // (null: every block is owned)
    const unsigned char *owned;
};

// Host tables of a geometry (rays, blocks, bands, compact band offsets) without
// touching the GPU; bsgd_geometry_create adds the device copies (geometry.cu).
bsgd_status build_host_tables(const bsgd_geometry_desc *desc, int M, int N, bsgd_geometry *g);

// Device memory from the library's stream-ordered pool (solver.cu), and the
// stream-ordered release of a solver state (serving).
bsgd_status pool_alloc(void **p, size_t bytes, cudaStream_t st);
// The same for optional scratch: false (and no recorded error) when it fails.
bool pool_try_alloc(void **p, size_t bytes, cudaStream_t st);
void pool_free(void *p, cudaStream_t st);
void state_release(bsgd_state *s, cudaStream_t st);

// Workspace of one TV prox (tv.cu): the input image b (FP32), the dual p and
// its extrapolation r in two buffers (read one, write the other; one float4
// per voxel).
struct TvWork {
    float *b = nullptr;
    float4 *p = nullptr, *r = nullptr, *r2 = nullptr;
};
bsgd_status tv_work_alloc(const bsgd_geometry *g, TvWork &w);
void tv_work_free(TvWork &w);
bsgd_status tv_prox_run(const bsgd_geometry *g, void *x, bsgd_dtype xt, double kappa, int iters,
                        cudaStream_t st, void *xlo, const TvWork &w);

// Sub-detector cell rectangle (Fig. 2): halves in u for 2 cells, quadrants
// (v half * 2 + u half) for 4.
__host__ __device__ inline void cell_rect(int nu, int nv, int n_cells, int c, Band &b) {
    if (n_cells <= 1 || c < 0) return;
    const int uh = c & 1, vh = n_cells == 4 ? (c >> 1) : 0;
    const int um = nu / 2, vm = nv / 2;
    if (uh) b.u0 = max(b.u0, um); else b.u1 = min(b.u1, um - 1);
    if (n_cells == 4) {
        if (vh) b.v0 = max(b.v0, vm); else b.v1 = min(b.v1, vm - 1);
    }
}

bsgd_status launch_fp_solve(const bsgd_geometry *g, const SolveDev &S, const void *x,
                            bsgd_dtype st_t, int max_pairs, int max_tiles, bool fused,
                            cudaStream_t st);
bsgd_status launch_bp_solve(const bsgd_geometry *g, const SolveDev &S, bsgd_dtype st_t,
                            int max_pairs, int max_tiles, cudaStream_t st);
// Several column blocks per iteration (2 .. kMaxFusedCols), every drawn row
// block paired with every drawn column block: FP, residual and BP in one pass
// over the bounding box of the selected blocks' bands; grid z = row-block
// slots (max_rows), max_tiles bounds the tiles of any such box.
// Algorithm 1 from a starting image x (device, storage type): z^j = A^j x_J in
// every block's band rows and r = y - sum_j z^j; skipped on the device when x
// is zero (flag: one device int of scratch).
// flag = 1 if any voxel of x is non-zero (flag cleared first), on stream st.
bsgd_status launch_nonzero(const bsgd_geometry *g, const void *x, bsgd_dtype st_t, int *flag,
                           cudaStream_t st);
bsgd_status launch_warm_start(const bsgd_geometry *g, const SolveDev &S, const void *x,
                              bsgd_dtype st_t, int *flag, cudaStream_t st);
constexpr int kMaxFusedCols = 4;
bsgd_status launch_fpbpm_solve(const bsgd_geometry *g, const SolveDev &S, const void *x,
                               bsgd_dtype st_t, int max_rows, int max_tiles, int n_cols,
                               cudaStream_t st);
bsgd_status launch_fpbp_solve(const bsgd_geometry *g, const SolveDev &S, const void *x,
                              bsgd_dtype st_t, int max_pairs, int max_tiles, cudaStream_t st);
bsgd_status launch_count_cells(const bsgd_geometry *g, int j, int n_cells,
                               unsigned long long *d_counts, cudaStream_t st);

}  // namespace bsgd

namespace bsgd {

struct SampleArgs {
    DeviceGeom G;
    Work *work;
    int *cells;                 // kMaxPairs x max_views
    int64_t *iter;
    int64_t it;                 // the iteration, when the launcher knows it (else -1: read *iter)
    uint64_t seed;
    int pairs_mode, cells_mode, n_cells, kM, kN;
    const double *S;            // M x nv
    const int *wband;           // M x N x 2
    const double *cw;           // N x n_views x n_cells
    const int32_t *replay;      // replay_n x stride
    int64_t replay_start, replay_n;
    int32_t *trace;             // trace_cap x stride
    int64_t trace_cap;
    int stride;
    const unsigned long long *counts;  // N x n_views x n_cells
    const unsigned long long *pair_upd;  // M x N updates of whole views (null: sum per view)
    unsigned long long *updates;
};

// ---------------------------------------------------------------------------
// Serving: one entry per resident request of a server (device table)

struct ReqDesc {
    DeviceGeom G;
    SolveDev S;
    SampleArgs A;
    void *x;                 // image (storage type)
    void *xlo;               // low-order image term (16-bit storage) or null
    int dtype;               // storage type
    int max_tiles;           // detector tiles of the largest work box of one view
    int active;
    int period;              // the request advances in rounds whose index is a multiple of it
    int kN;                  // column blocks per iteration (1: one-block fused pass)
    int64_t work_begin;      // first FP / BP work item of this request in a round
    int64_t work_count;      // max_tiles * max_views * (pairs, or row blocks when kN > 1)
    int64_t max_block_cols;  // voxels of the largest column block
    int64_t target;          // iterations of the request (no draw past the last)
};

// The round's work items come in classes, each run by its own persistent
// kernel (so that each gets the registers, and the occupancy, of its own pass):
// class = 3 * (several column blocks per iteration ? 1 : 0) + storage type.
// Table entries of class c are [lo[c], hi[c]) (the table is sorted by class);
// a request's work_begin counts within its class. Only the kernels of the
// classes present are in the round's graph.
constexpr int kRoundClasses = 6;
struct RoundCtl {
    unsigned long long next[kRoundClasses];  // persistent-kernel work counters
    int n;                                   // table entries in use
    int pad;
    unsigned long long round;                // index of the round (advanced at its end)
    int lo[kRoundClasses], hi[kRoundClasses];
    int64_t total_items[kRoundClasses];      // FP / BP work items of the round, per class
};
__host__ __device__ inline int round_class(int kN, int dtype) { return 3 * (kN > 1 ? 1 : 0) + dtype; }
// Whether a request sits out round `round` (age priority: period 2 for all
// but the oldest resident request; period 1 advances every round).
__host__ __device__ inline bool round_skips(int period, unsigned long long round) {
    return period > 1 && round % (unsigned long long)period != 0;
}

// Fill a request descriptor from a live state (solver.cu).
bsgd_status state_descriptor(const bsgd_state *s, void *x, ReqDesc *out);
bsgd_status state_first_draw(bsgd_state *s, cudaStream_t st);
// Device bytes state_create allocates for this geometry and these parameters,
// and the transient set-up buffers on top (solver.cu).
size_t state_bytes(const bsgd_geometry_desc &d, int M, int N, const bsgd_solve_params &p,
                   size_t *transient);
bsgd_status validate_desc(const bsgd_geometry_desc *d, int M, int N);
bsgd_status convert(const void *in, bsgd_dtype it, void *out, bsgd_dtype ot, int64_t n,
                    cudaStream_t st);

// Round kernels of the server (enqueued once into a captured graph).
// ct: read the table from the device's constant copy (upload_round_const_table)
bsgd_status launch_round_solve(const ReqDesc *table, RoundCtl *ctl, int cls, bool ct, int grid,
                               cudaStream_t st);
constexpr int kRoundConstSlots = 64;   // entries of the constant-memory table (one server per device)
bsgd_status upload_round_const_table(const ReqDesc *h, int n, cudaStream_t st);
// the block updates with the next draws, their promotion, and the round's end
// (the round index advanced)
bsgd_status launch_round_update(const ReqDesc *table, RoundCtl *ctl, int max_slots,
                                cudaStream_t st);
int round_persistent_grid(int cls, bool ct);

}  // namespace bsgd
