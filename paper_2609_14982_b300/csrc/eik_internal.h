// Internal declarations shared by the libeik translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "eik.h"

#include <nvtx3/nvToolsExt.h>

namespace eik {

struct TravParams;
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define EIK_CHECK(call)                                                        \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return eik::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define EIK_CHECK_LAUNCH() EIK_CHECK(cudaGetLastError())

// NVTX range over a host scope (the phases of a call), for profilers that filter or
// group kernels by range (ncu --nvtx); costs nothing when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// consecutive NVTX ranges over the phases of one host function: next() closes the open
// phase and opens the named one; the last closes at scope exit
struct NvtxPhase {
    bool open = false;
    void next(const char *name)
    {
        if (open) nvtxRangePop();
        nvtxRangePushA(name);
        open = true;
    }
    ~NvtxPhase() { if (open) nvtxRangePop(); }
};

// Capacity of one work item (positions staged in shared memory); the build option
// eik_opts.chunk picks the item size actually used (default: the capacity).
constexpr int ITEM_MAX = 64;
// Largest item a tangent may be built with (eik_opts.chunk); items above ITEM_MAX run only
// in the persistent schedule (a kernel instance with this capacity), e.g. for R = 1.
constexpr int ITEM_CAP = 256;

// Most dependencies recorded per work item.
constexpr int DEP_MAX = 32;

// Device-side fault codes latched in Tangent::err (first one wins).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_SINGULAR = 2, DEV_BAD_INDEX = 3 };

struct GridDesc {
    int ndim;
    int n[3];
    double dxi[3];
    long long N;
    long long st[3];   // strides of the logical dimensions in the linear index
};

GridDesc make_grid_desc(const eik_grid *g);

// A nontrivial SCC block of one source.
struct Block {
    int src;        // source
    int p0;         // first position (canonical order) of the block
    int k;          // size
    int level;      // level of the block in the condensation
    long long lu;   // offset of the k*k FP64 factors
    long long piv;  // offset of the k pivots
    long long ws;   // offset (in rows) of the block's rows in the workspace
};

// Off-grid point sources (see eik_points.cu): per source the 2^ndim corners of its cell
// (arrays padded to 8 corners), all device [S][.] unless noted.
struct PointData {
    int S = 0, K = 0;              // sources, corners per source (0: node sources)
    double *f = nullptr;           // [S][3] fractional logical coordinates
    int *node = nullptr;           // [S][8] corner nodes (-1 padding)
    double *phi = nullptr;         // [S][8] multilinear weights
    double *phim = nullptr;        // [S][8] phi x model factor at the corner
    double *xs = nullptr;          // [S][3] source positions
    double *ss = nullptr;          // [S] source slownesses
    double *r = nullptr;           // [S][8] seed distances |x_q - x_src|
    double *z = nullptr;           // [S][N] A^-1 e (e = r on the seed rows), natural order
    double *zrec = nullptr;        // [S][n_rec] z at the on-grid receivers
    double *sigma = nullptr;       // [S][sigma_cols] sum_q phim_q p_q of the current columns
    int sigma_cols = 0;
    double *ip_rho = nullptr;      // [S][n_ip] direct receivers: |x_r - x_src|, else -1
    double *ip_zeta = nullptr;     // [S][n_ip] rho (direct) or P z
    std::vector<int> base;         // host [S][3] cell base
    std::vector<double> xs_host;   // host [S][3]
    std::vector<double> corner_xyz;  // host [S][8][3] corner positions
};

// Per-direction launch state of the traversal: the transported field's workspace, the
// block right-hand sides and the completion counters and ticket of the persistent and
// cluster schedules.  The forward direction uses the Tangent's own fields; with
// opts.split_dirs the transpose uses Tangent::lane_t, so the two may run concurrently.
struct Lane {
    void *ws_vec = nullptr;
    size_t ws_vec_bytes = 0;
    double *ws_blk = nullptr;
    size_t ws_blk_elems = 0;
    int *item_done = nullptr;     // [nitems]
    int *done = nullptr;          // [S][maxL]
    int *ticket = nullptr;        // [4]
};

struct Tangent {
    int S = 0;
    long long N = 0;
    int n_rec = 0;
    int model = 0;
    int maxL = 0;
    GridDesc grid{};
    eik_opts opts{};
    int device = 0;
    int num_sms = 0;

    std::vector<int> nlev;                 // [S]
    std::vector<long long> level_ptr;      // [S][maxL+1] host copy
    std::vector<long long> ebase;          // [S+1] forward edge base
    std::vector<long long> tbase;          // [S+1] transposed edge base
    long long *ebase_d = nullptr;          // device copies of ebase / tbase
    long long *tbase_d = nullptr;
    std::vector<Block> blocks;
    std::vector<eik_stats> stats;          // [S]

    // ---- device structure, canonical (level-permuted) order unless noted
    int *perm = nullptr;      // [S][N] node at position; ~node (<0) for block members
    int *pos = nullptr;       // [S][N] natural -> position
    int *label = nullptr;     // [S][N] natural: SCC id (smallest local node)
    int *level = nullptr;     // [S][N] natural: level of the node's component
    int *rowptr = nullptr;    // [S][N+1] local offsets into the forward edge arrays
    int *up_node = nullptr;   // [E] canonical position of upstream node j
    float *up_w32 = nullptr;
    double *up_w64 = nullptr;
    int *cptr = nullptr;      // [S][N+1] local offsets into the transposed edge arrays
    int *dn_node = nullptr;   // [E'] canonical position of downstream node i
    float *dn_w32 = nullptr;
    double *dn_w64 = nullptr;
    double *cq64 = nullptr;   // [S][N] C*M coefficient per position
    float *cq32 = nullptr;
    double *cqn64 = nullptr;  // [S][N] same, natural order (source-sum reduction)
    float *cqn32 = nullptr;
    int *rec_slot = nullptr;  // [S][N] receiver index per position, -1 if none
    int *rec_nat = nullptr;   // [S][n_rec] receiver nodes
    // natural-order rows for export
    int *nrow_cnt = nullptr;      // [S][N]
    int *nrow_node = nullptr;     // [S][N][2*ndim]
    double *nrow_w = nullptr;     // [S][N][2*ndim]
    double *cs_nat = nullptr;     // [S][N]
    // blocks
    int nblk = 0;
    int4 *blk_desc = nullptr;     // {src, p0, k, level}
    long long *blk_off = nullptr; // [nblk][3] {lu, piv, ws}
    double *lu = nullptr;         // P A_C = L U factors of every nontrivial block
    double *binv = nullptr;       // A_C^-1 of every block, row-major, same offsets as lu
    int *piv = nullptr;
    long long lu_words = 0, piv_words = 0, ws_rows = 0;
    // work items of the traversals: {src, step, p0, p1} or {src, step, ~blk, 0}
    int nitems = 0;
    int item_max = 0;             // positions per singleton item of this tangent
    int4 *items_fwd = nullptr;
    int4 *items_bwd = nullptr;
    int2 *ebeg_fwd = nullptr;     // per item: [first, last) local edge offsets of its rows
    int2 *ebeg_bwd = nullptr;
    std::vector<int> step_ptr_fwd, step_ptr_bwd;   // [maxL+1] items per step (host)
    int *item_cnt = nullptr;      // [S][maxL] items per (source, level); bwd uses reversed step
    // per-item dependencies: the items holding the upstream positions of an item's rows
    // (at most DEP_MAX, else the item waits for its whole previous step), per direction
    int *deps_fwd = nullptr, *deps_bwd = nullptr;     // [nitems][DEP_MAX]
    int *ndeps_fwd = nullptr, *ndeps_bwd = nullptr;   // [nitems], -1 = overflow
    int *item_done = nullptr;     // [nitems] 1 once the item of the current traversal finished
    int *done = nullptr;          // [S][maxL] completed items per (source, step)
    int *ticket = nullptr;        // [2]
    int *err = nullptr;           // [4] device fault latch {code, source, step, item}
    // cluster schedule: per source the first position of every level and the first block of
    // every level (blocks are ordered by (source, level)), and the sources by decreasing level
    // count (the order in which clusters take them)
    int *lvl_d = nullptr;         // [S][maxL+1]
    int *blk_lvl_d = nullptr;     // [S][maxL+1]
    int *nlev_d = nullptr;        // [S]
    int *order_d = nullptr;       // [S]
    std::map<long long, int> cluster_fit;   // cached occupancy queries of the cluster launch
    // off-grid receivers (multilinear sampling), set by tangent_set_receivers
    int n_ip = 0, ip_k = 0;       // receivers per source, corners per receiver (2^ndim)
    int *ip_node = nullptr;       // [S][n_ip][ip_k] natural node of each corner
    double *ip_w = nullptr;       // [S][n_ip][ip_k] multilinear weight
    int n_ipt = 0;                // touched nodes per source (padded to the largest source)
    int *ipt_node = nullptr;      // [S][n_ipt] touched nodes, ascending, -1 = padding
    int *ipt_ptr = nullptr;       // [S][n_ipt+1] ranges into ipt_e
    int *ipt_e = nullptr;         // [S][n_ip*ip_k] corner entries (receiver * ip_k + corner)
    void *ws_in = nullptr;        // dense input / column-chunk staging of the interpolated paths
    size_t ws_in_bytes = 0;
    // workspaces
    void *ws_vec = nullptr;       // internal dT / lam
    size_t ws_vec_bytes = 0;
    double *ws_blk = nullptr;     // block right-hand sides
    size_t ws_blk_elems = 0;
    int host_err = 0;
    std::vector<long long> holds;   // item_cnt entries raised by tangent_debug_hold
    // per-level schedule: device-resident launch parameters (forward, transpose) and the
    // captured level sequences, keyed by (direction, element size, vector width, lanes)
    struct TravParams *params_d = nullptr;
    std::map<long long, cudaGraphExec_t> level_graphs;
    cudaStream_t cap_stream = nullptr;
    bool opts_graph = true;
    // directional sweeping (the plain form): slotted weights per (direction, precision),
    // the stopping-test words and one captured cycle per (direction, precision, R, b, x)
    void *sweep_w[4] = {nullptr, nullptr, nullptr, nullptr};
    unsigned int *sweep_flags = nullptr;
    std::map<std::vector<long long>, cudaGraphExec_t> sweep_graphs;
    // off-grid point sources (tangent_build_points); pts.K == 0 for node sources
    PointData pts;
    // the transpose direction's own launch state (opts.split_dirs)
    Lane lane_t;
    // level-synchronous schedule (eik_sync.cu), per direction (forward, transpose): the unit
    // records in step order per precision (FP32, FP64) and per step its first record and
    // singleton records; the grid-barrier counters (32 words per direction)
    void *sync_rec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int *sync_base[2] = {nullptr, nullptr};
    int sync_steps[2] = {0, 0};
    unsigned *sync_bar = nullptr;
    // batched persistent launches led by this tangent: the merged ticket order and its runs
    void *batch_buf = nullptr;
    size_t batch_bytes = 0;
    std::vector<int4> batch_runs;
};

// whether the transpose direction runs on its own launch state
inline bool split_lane(const Tangent *t, bool TR) { return TR && t->opts.split_dirs && t->lane_t.ticket; }
// the transported field's workspace of a direction
inline void *lane_ws(const Tangent *t, bool TR) { return split_lane(t, TR) ? t->lane_t.ws_vec : t->ws_vec; }
// allocate the transpose's counters and ticket (once)
int enable_split(Tangent *t);
// build the level-synchronous schedule's step tables of a precision (EIK_F32, EIK_F64, or -1 for
// both) and its barrier counters (once; synchronizes)
int prepare_sync(Tangent *t, int dtype);

// src_f (host [S][ndim] fractional logical coordinates) selects point sources; then
// src_node is ignored
int build_tangent(const eik_grid *g, const double *T, const double *s, int S, const int *src_node,
                  const int *rec_node, int n_rec, const eik_opts *opts, Tangent **out,
                  cudaStream_t stream, const double *src_f = nullptr);

// point sources: corners, weights, positions and seed distances (allocates pd's device
// arrays; synchronizes); the tangent's model factors and z = A^-1 e after its build
int point_sources(const GridDesc &g, const double *xyz, const double *s, int S, const double *f_host, PointData &pd,
                  cudaStream_t st);
void free_point_data(PointData &pd);
int point_tangent_setup(Tangent *t, const double *s, cudaStream_t st);
// J: sigma of the current columns from the model input; out[a][j][r] += sigma zeta[a][j]
int seed_sigma(Tangent *t, const void *in, int shared_in, long long ld_in, int w, int dtype, cudaStream_t st);
int seed_add(Tangent *t, long long n, int w, const double *zeta, void *out, long long ld, int dtype, cudaStream_t st);
// J^T: g += M^T Phi^T (r . lam_seeds + rho . y_direct), in source order, from the workspace
int seed_scatter(Tangent *t, int w, void *g, long long ld_g, bool per_source, const void *y, long long ld_y,
                 int n_y, const double *rho, int dtype, cudaStream_t st);
int seed_interp_setup(Tangent *t, const std::vector<double> &rho_host, cudaStream_t st);
void free_tangent(Tangent *t);

enum Mode : int { MODE_J = 0, MODE_RAW = 1 };

int traverse(Tangent *t, bool transpose, int mode, const void *in, int shared_in, int R,
             void *out_full, void *out_aux, int sum_sources, int dtype, cudaStream_t stream);

// J p (TR false: in = shared model p [N_k][R_k], out = d_rec) or J^T y summed over
// sources (TR true: in = y, out = g [N_k][R_k]) of several tangents in one cluster launch
int traverse_batch(Tangent *const *ts, int ntan, bool TR, const void *const *in, const int *R, void *const *out,
                   int dtype, cudaStream_t st);

int sweep(Tangent *t, bool transpose, const void *b, int R, void *x, int dtype,
          const eik_opts *opts, int *cycles, cudaStream_t stream);

int ensure_workspace(Tangent *t, size_t vec_bytes, size_t blk_elems, bool TR = false);
// g (row stride ld_g) = sum over sources of c_a x_a for the w columns in the workspace, or
// g += that sum when accumulate
int source_sum(Tangent *t, int w, void *g, long long ld_g, int dtype, cudaStream_t st, bool accumulate = false);
// off-grid receivers (multilinear P): set from host [S][n_rec][ndim] fractional indices,
// then J p -> [S][n_rec][R] and J^T y -> [N][R] (summed over sources)
// node <- cell averaging map (to_nodes) or its transpose, vectors [.][R]
int cell_map(int ndim, const int *n, const void *in, int R, void *out, bool to_nodes, int dtype, cudaStream_t st);
int set_receivers_interp(Tangent *t, int n_rec, const double *f);
int apply_interp_entry(Tangent *t, const void *ds, int shared, int R, void *d_rec, int dtype, cudaStream_t st);
int apply_interp_T_entry(Tangent *t, const void *y, int R, void *g, int dtype, cudaStream_t st);

void launch_sample(long long N, int S, int n_rec, const int *rec, const double *field, double *out, cudaStream_t st);

}  // namespace eik
