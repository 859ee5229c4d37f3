/*
 * libeik: frozen full-metric Eikonal tangent transport on one B300 (sm_103a).
 *
 * The library applies A^-1 and A^-T of the frozen linearized transport (Sec. 3.1,
 * Eq. transport-system, A = I - W) inside the Jacobian actions J p and J^T y
 * (Sec. 4.4, Eqs. source-jacobian and source-transpose) as a block-triangular solve
 * over the SCC condensation of the upwind dependency graph (Sec. 4.1, Eq. block-form,
 * Prop. 3).  All work runs in the library's own CUDA kernels.
 *
 * Conventions
 *   Grid: logical dims 3-D (xi, eta, zeta) or 2-D (xi, zeta); zeta last, zeta = 0 is
 *     the top surface.  Node (i,j,k) has linear index (i*n1 + j)*n2 + k (2-D: i*n1 + k);
 *     N = product of n.
 *   Vectors: right-hand-side index fastest.  A per-source field is [S][N][R]; a model
 *     vector shared by all sources is [N][R]; receiver data is [S][n_rec][R].
 *   Pointers documented "device" must be device memory of the current device; "host"
 *     pointers are read before the call returns.
 *   Streams: every call is asynchronous on `stream` (a cudaStream_t) unless stated;
 *     NULL means the legacy default stream.
 *   Ownership: the caller owns every buffer it passes.  The library owns an
 *     eik_tangent (structure, weights, factors, workspaces) until tangent_free.
 *   Errors: every call returns EIK_OK (0) or a negative eik_status and never throws
 *     across the ABI; eik_last_error() gives a thread-local message.  Faults detected
 *     on the device (a singular block, a wait that timed out) are latched in the
 *     tangent and returned by tangent_status().
 */
#ifndef EIK_H
#define EIK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *eik_stream;      /* same object as cudaStream_t */

typedef enum {
    EIK_OK = 0,
    EIK_ERR_INVALID = -1,          /* bad argument (sizes, null pointers, duplicate receivers) */
    EIK_ERR_OOM = -2,              /* device allocation failed */
    EIK_ERR_SINGULAR_BLOCK = -3,   /* an SCC block had a pivot below eik_opts.lu_pivot_tol */
    EIK_ERR_NOT_CONVERGED = -4,    /* iterative solve (eik_forward, sweeping) hit its limit */
    EIK_ERR_TIMEOUT = -5,          /* a bounded device-side wait ran out */
    EIK_ERR_CUDA = -6,             /* CUDA runtime error */
    EIK_ERR_CYCLE = -7             /* internal: condensation not acyclic (never expected) */
} eik_status;

typedef enum { EIK_F64 = 0, EIK_F32 = 1 } eik_dtype;

/* Model map M (Sec. 2.3): ds = p (slowness), ds = -s^2 dv (velocity), ds = -s m
 * (relative velocity perturbation m = dv/v). */
typedef enum { EIK_MODEL_SLOWNESS = 0, EIK_MODEL_VELOCITY = 1, EIK_MODEL_RELATIVE = 2 } eik_model;

/* Traversal schedule of tangent_apply / tangent_apply_T. */
typedef enum {
    EIK_SCHED_PERSISTENT = 0,      /* one persistent launch, device level queue, bounded waits */
    EIK_SCHED_LEVELS = 1,          /* one launch per level, replayed from a CUDA graph */
    EIK_SCHED_STAGED = 2,          /* per-level launches whose vector rows are staged in shared
                                      memory by per-thread async copies (needs R x element size a
                                      multiple of 16 bytes, >= 64, items x 16-byte lanes <= 512
                                      and the two stages within 200 KB; else as LEVELS) */
    EIK_SCHED_CLUSTER = 3,         /* one launch; a thread-block cluster owns one source at a time
                                      and walks its levels with one hardware cluster barrier per
                                      level (no device-side spin waits) */
    EIK_SCHED_SYNC = 4             /* one cooperative launch (all CTAs resident); every source
                                      advances one level per global step and the steps end at a
                                      bounded grid-wide barrier; an SCC block takes two steps of
                                      its source (right-hand side, then the inverse product spread
                                      over the grid); needs block_lu_min = 0 and holds the whole
                                      GPU, so two such traversals do not overlap */
} eik_schedule;

typedef struct {
    int ndim;             /* 2 or 3 */
    int n[3];             /* nodes per logical dimension, each >= 3 */
    double dxi[3];        /* logical spacing per dimension (> 0) */
    const double *xyz;    /* device [N][ndim] physical coordinates (x[, y], z) */
} eik_grid;

typedef struct {
    int model;                 /* eik_model, used by tangent_build for the M map */
    double lu_pivot_tol;       /* |pivot| below this marks a block singular (default 1e-13) */
    int schedule;              /* eik_schedule (default persistent) */
    int threads;               /* CTA size of the traversal kernels (default 256) */
    int chunk;                 /* singleton nodes per work item (default 0 = 64; at most 256:
                                  items above 64 suit few right-hand sides, e.g. R = 1 in
                                  Krylov loops, and run in the persistent or cluster schedule) */
    int ctas_per_sm;           /* persistent grid = SMs x this (default 0 = occupancy) */
    double wait_timeout_s;     /* bound on any device-side wait (default 2 s) */
    /* eik_forward */
    double eik_tol;            /* stop when max |d tau| < eik_tol over a cycle (default 1e-12) */
    int eik_max_cycles;        /* (default 2000) */
    double eik_src_radius;     /* tau = 1 for |x - x_src| <= radius * max(dxi) (default 1.0) */
    /* sweeping baseline */
    double sweep_tol;          /* max |dx| <= sweep_tol * max |x| over one cycle (default 1e-12) */
    int sweep_max_cycles;      /* (default 10000) */
    /* traversal */
    int rhs_chunk;             /* process right-hand sides in column chunks of this many
                                  (0 = all at once); bounds the internal workspace */
    /* eik_forward precision split */
    int eik_fp32;              /* 1: nodes farther than eik_fp64_radius * max(dxi) from the
                                  source update in FP32 arithmetic (FP64 storage), the source
                                  neighbourhood stays FP64; the stop test then uses
                                  max(eik_tol, 1e-6).  0 (default): FP64 everywhere */
    double eik_fp64_radius;    /* (default 8) */
    /* persistent schedule */
    int item_deps;             /* 1 (default): a work item waits only for the items holding its
                                  upstream rows; 0: for every item of its source's previous
                                  level (the plain level barrier) */
    /* cluster schedule */
    int cluster_size;          /* CTAs per cluster, 1..16 (default 0 = the largest size that keeps
                                  every source's cluster resident at once) */
    int cluster_threads;       /* threads per CTA, a multiple of 32 in 64..256 (default 0 = 256) */
    int pass_units;            /* most right-hand-side vectors a thread of the cluster schedule
                                  carries for one position: 1, 2 or 4 (default 0 = 4); a thread
                                  carries 4 / that many positions per round.  Level-synchronous
                                  schedule: rows a thread has in flight, 0 = 1 (1024 threads per
                                  CTA), 2 (768 threads), 4 (512 threads) */
    /* SCC block solves */
    int block_lu_min;          /* blocks of at least this many nodes are solved by FP64 forward and
                                  back substitution with their partial-pivot LU factors (one warp
                                  per right-hand side), the accuracy tier for ill-conditioned
                                  blocks; other blocks multiply by the explicit inverse formed from
                                  the same factors, which has the same FP64 work (k^2 per column)
                                  and more parallelism (default 0: always the inverse) */
    /* concurrency */
    int split_dirs;            /* 1: the transpose direction keeps its own workspace, counters and
                                  ticket, so tangent_apply and tangent_apply_T on one tangent may
                                  run concurrently on two streams (give each about half the CTAs,
                                  ctas_per_sm); costs one more [S][N][R] workspace.  The other
                                  calls (interp forms, solves, sweeping) still must not overlap.
                                  0 (default): calls on one tangent must not overlap on the
                                  device */
    int item_slots;            /* persistent schedule: work items a CTA holds at once, 1 (default)
                                  or 2..4; with several, each item's structure lands in its own
                                  shared-memory slot and the CTA computes whichever held item
                                  has its upstream items done first (one right-hand-side vector
                                  per thread; items above 64 positions use two slots) */
} eik_opts;

typedef struct {
    int64_t nodes;             /* N */
    int64_t edges;             /* dependencies w_ij > 0 */
    int64_t components;        /* SCCs (singletons included) */
    int64_t nontrivial;        /* SCCs with >= 2 nodes */
    int64_t cyclic_nodes;      /* nodes in nontrivial SCCs */
    int64_t largest;           /* largest SCC */
    int64_t levels;            /* levels of the condensation DAG (longest path + 1) */
    int64_t max_level_width;   /* most nodes in one level */
    int64_t identity_rows;     /* non-seed rows without an upstream face */
    int64_t lu_doubles;        /* FP64 words held by block factors */
} eik_stats;

/* Fill opts with the defaults listed above. */
void eik_opts_default(eik_opts *opts);

/* Thread-local message of the last failing call ("" if none). */
const char *eik_last_error(void);

/* Library build string (architecture, version). */
const char *eik_version(void);

/*
 * eik_forward -- first-arrival traveltimes T_a for S point sources (Sec. 2.1,
 * Eq. eikonal with the point-source factorization T = T0 tau, and Sec. 2.2,
 * Eq. metric-eikonal).  The paper cites its state solver (FTDEE) without giving it;
 * this call solves the factored full-metric equation with first-order Lax-Friedrichs
 * sweeping to a discrete fixed point (tau = 1 near the source).
 *   g        grid (xyz device)
 *   s        device [N] slowness
 *   S        number of sources
 *   src_node host [S] node index of each source
 *   T        device [S][N] output (seconds in the grid's units times slowness units)
 *   cycles   host, optional: number of sweep cycles used
 * Returns EIK_ERR_NOT_CONVERGED when eik_max_cycles is reached (T holds the last
 * iterate).  Synchronizes the stream once per cycle to test convergence.
 */
int eik_forward(const eik_grid *g, const double *s, int S, const int *src_node,
                double *T, const eik_opts *opts, int *cycles, eik_stream stream);

/*
 * eik_forward_noalloc -- the paper has no counterpart to this call; it exists for
 * callers that cannot allocate device memory, for example code running inside a
 * framework whose caching allocator owns all device memory, or inside a region
 * where cudaMalloc and cudaFree are not allowed (they synchronize the device).
 * It computes exactly what eik_forward computes, with the same arguments, but calls no
 * allocator: its scratch is one file-scope device array of
 * eik_forward_noalloc_capacity() bytes (64 MiB), held by every GPU that loads the
 * library until the process exits.
 *   Limit: the call needs 2 N ndim^2 + S N (2 + 2 ndim) doubles + S N bytes + S x 8 KiB
 *   (the per-source convergence slots: 1024 64-bit words each) + S x 13 bytes, each
 *   piece rounded up to 256 bytes; larger requests return EIK_ERR_INVALID with the sizes
 *   in the message (about 320k 3-D nodes for one source).
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current and keeps it for the life of the
 *   process; make that first call before any stream capture, and do not use this call
 *   across a cudaDeviceReset of that device (the array moves, the kept address does not).
 *   Sharing: every call, on any stream, uses the same array and overwrites it; calls
 *   that overlap on the GPU race with each other.  Issue them one after the other.  A
 *   call that returns an error has first waited for its own queued work, so a following
 *   call does not race with it.
 */
int eik_forward_noalloc(const eik_grid *g, const double *s, int S, const int *src_node,
                        double *T, const eik_opts *opts, int *cycles, eik_stream stream);

/*
 * eik_forward_warm -- eik_forward started from a given traveltime field instead of the
 * homogeneous solution (tau = T_init / T0 at every non-fixed node; tau = 1 where T_init is
 * not positive and finite): the re-setup of an outer Gauss-Newton iteration (Alg. 1 Phase
 * I after a model update) starts from the previous iteration's state.  The sweeps, the
 * stopping rule and the result's fixed point are those of eik_forward; the state agrees
 * with a cold start to the stopping tolerance, in fewer cycles when T_init is close.
 *   T_init   device [S][N] (may be the same buffer as T)
 *   other arguments and errors as eik_forward
 */
int eik_forward_warm(const eik_grid *g, const double *s, int S, const int *src_node,
                     const double *T_init, double *T, const eik_opts *opts, int *cycles, eik_stream stream);

/*
 * eik_forward_points -- the state solve of eik_forward for point sources between grid
 * nodes (the off-grid sources of Sec. 3.1 / 4.4; the paper gives the source treatment no
 * formula).  Reading: source a sits at fractional logical coordinates f[a] (0 <= f_d <=
 * n_d - 1); its cell has corner base b_d = min(floor(f_d), n_d - 2) and the corners the
 * multilinear weights phi_q of f; the source position is x_src = sum_q phi_q x_q and its
 * slowness s_src = sum_q phi_q s_q (corner q: axis 0 the most significant bit).  The
 * factored solve uses T0 = s_src |x - x_src|; nodes within max(eik_src_radius x largest
 * spacing, largest corner distance) of x_src keep tau = 1, so every corner holds
 * T = s_src |x_q - x_src|.
 *   src_f    host [S][ndim] fractional logical coordinates of the sources
 *   T        device [S][N] output; other arguments and errors as eik_forward
 */
int eik_forward_points(const eik_grid *g, const double *s, int S, const double *src_f,
                       double *T, const eik_opts *opts, int *cycles, eik_stream stream);

/* Bytes of the fixed scratch array behind eik_forward_noalloc. */
size_t eik_forward_noalloc_capacity(void);

typedef struct eik_tangent eik_tangent;

/*
 * tangent_build -- Phase I of Algorithm 1 (Sec. 4.6, Alg. 1 steps 7-10) for S sources:
 * face-based upwind rows A_a = I - W_a (Sec. 3.1), calibration c^(s) = (A T)/s
 * (Sec. 3.2), dependency graph (Sec. 3.3), SCCs and the canonical level order of the
 * condensation DAG (Sec. 4.1), dense LU of every nontrivial SCC block (Sec. 4.3).
 *   T        device [S][N] frozen traveltimes (e.g. from eik_forward)
 *   s        device [N] slowness
 *   src_node host [S] seed node of each source (its row is the identity, q = 0)
 *   rec_node host [S][n_rec] receiver nodes per source (P_a: on-grid sampling);
 *            must be distinct within a source; n_rec may be 0
 *   out      receives the new tangent (owned by the library)
 * Canonical order (the paper fixes none): component id = its smallest node; level =
 * longest path in the condensation; components ordered by (level, smallest node),
 * nodes ascending inside a component.  Synchronizes the stream (sizes are read back).
 * Returns EIK_ERR_SINGULAR_BLOCK if a block pivot falls below lu_pivot_tol.
 */
int tangent_build(const eik_grid *g, const double *T, const double *s, int S,
                  const int *src_node, const int *rec_node, int n_rec,
                  const eik_opts *opts, eik_tangent **out, eik_stream stream);

/*
 * tangent_build_points -- tangent_build for point sources (eik_forward_points' reading):
 * the seed rows of source a are the 2^ndim corners of its cell (identities), with the
 * differentiated source treatment as their right-hand side, q_q = r_q sum_k phi_k ds_k
 * (r_q = |x_q - x_src|, ds = M p).  Every Jacobian call of the tangent includes these
 * rows; an off-grid receiver set later with tangent_set_receivers that lies in its
 * source's cell is carried by the direct term D_a of Eq. (source-jacobian):
 * d_rec = |x_r - x_src| sum_k phi_k ds_k, with a zero row of P.  The build also forms
 * z_a = A_a^-1 e_a (e_a = r on the seed rows; FP64 [S][N], one extra traversal), so J p
 * adds sigma_a z_a at the outputs (sigma_a = sum_k phi_k ds_k) and J^T y adds
 * M^T Phi^T sum_q r_q lam_q in source order.
 *   src_f    host [S][ndim] fractional logical coordinates (as eik_forward_points)
 *   T        device [S][N] states of these sources (e.g. from eik_forward_points)
 * Other arguments, ownership and errors as tangent_build.  The batched applies
 * (tangent_apply_batch, tangent_apply_T_batch) reject point-source tangents.
 */
int tangent_build_points(const eik_grid *g, const double *T, const double *s, int S,
                         const double *src_f, const int *rec_node, int n_rec,
                         const eik_opts *opts, eik_tangent **out, eik_stream stream);

/*
 * tangent_apply -- J p for all sources (Sec. 4.4, Eq. source-jacobian, D = 0;
 * Alg. 1 steps 15-16): ds = M p, q = C ds, dT = A^-1 q by the forward block traversal
 * B_a, d_rec = P dT.
 *   p            device: [N][R] if shared_model else [S][N][R]
 *   dT_full      device [S][N][R] or NULL (then an internal workspace holds dT)
 *   d_rec        device [S][n_rec][R] or NULL
 *   dtype        EIK_F64: FP64 vectors and arithmetic; EIK_F32: FP32 vectors, weights
 *                and accumulation, FP64 SCC block solves.
 * Asynchronous; device faults are latched (see tangent_status).
 */
int tangent_apply(eik_tangent *t, const void *p, int shared_model, int R,
                  void *dT_full, void *d_rec, int dtype, eik_stream stream);

/*
 * tangent_apply_T -- J^T y (Sec. 4.4, Eq. source-transpose, D = 0; Alg. 1 steps
 * 17-18): r = P^T y, lam = A^-T r by the reverse block traversal B_a^T (U^T, L^T, P^T
 * on blocks), g_a = M^T C^T lam_a, and g = sum_a g_a when sum_sources.
 *   y            device [S][n_rec][R]
 *   sum_sources  0: g_a per source; 1: g = sum_a g_a; 2: g += sum_a g_a (accumulates
 *                over calls, e.g. over source chunks of one gradient)
 *   g            device [N][R] if sum_sources else [S][N][R]
 *   lam_full     device [S][N][R] or NULL (internal workspace)
 * The source sum is a deterministic reduction in source order (EIK_F64: FP64;
 * EIK_F32: FP32 products with a compensated FP32 sum); with sum_sources = 2 the call's
 * sum is then added to g.
 */
int tangent_apply_T(eik_tangent *t, const void *y, int R, int sum_sources,
                    void *g, void *lam_full, int dtype, eik_stream stream);

/*
 * tangent_apply_batch / tangent_apply_T_batch -- J p and J^T y (as tangent_apply with a
 * shared model and tangent_apply_T with the source sum, Sec. 4.4) of up to 4 distinct
 * tangents, e.g. one per grid of a multi-grid workload, in ONE traversal launch, so
 * condensation DAGs of uneven depth and size run side by side.  By default the launch is
 * the persistent schedule over the work items of all the tangents in one merged order
 * (step s of every tangent before step s + 1 of any; max(2, item_slots of t[0]) items
 * held per CTA); if t[0]'s schedule is EIK_SCHED_CLUSTER (or a tangent was built with
 * items above 64 positions) it is the cluster schedule, whose thread-block clusters take
 * (tangent, source) units from one queue.  The source sums of J^T follow, one per
 * tangent.  Results equal the single-tangent calls bit for bit.
 *   t[k]      tangent k (same device for all)
 *   p[k]      device [N_k][R[k]] model vector block of tangent k (shared by its sources)
 *   y[k]      device [S_k][n_rec_k][R[k]] receiver data
 *   d_rec[k]  device [S_k][n_rec_k][R[k]] output;  g[k] device [N_k][R[k]] output
 *   dtype     common to all; R[k] may differ (the widest vector dividing all is used)
 * Every tangent's internal workspace is sized to all R[k] columns (no column chunks).
 */
int tangent_apply_batch(eik_tangent *const *t, int ntan, const void *const *p, const int *R, void *const *d_rec,
                        int dtype, eik_stream stream);
int tangent_apply_T_batch(eik_tangent *const *t, int ntan, const void *const *y, const int *R, void *const *g,
                          int dtype, eik_stream stream);

/*
 * tangent_solve / tangent_solve_T -- the bare transport solves dT = A^-1 q and
 * lam = A^-T r for all sources (Prop. 3, Sec. 4.3), q and r device [S][N][R],
 * outputs device [S][N][R].  Used for parity tests of the traversal alone.
 */
int tangent_solve(eik_tangent *t, const void *q, int R, void *x, int dtype, eik_stream stream);
int tangent_solve_T(eik_tangent *t, const void *r, int R, void *x, int dtype, eik_stream stream);

/*
 * tangent_sample -- receiver sampling P_a of a per-source field (Sec. 4.4, P_a):
 * out[a][k] = field[a][rec_a[k]], field device [S][N] FP64, out device [S][n_rec] FP64.
 */
int tangent_sample(const eik_tangent *t, const double *field, double *out, eik_stream stream);

/* Counts of one source's structure (Sec. 5.2, Eq. graph-fractions; Table 4 rows). Host. */
int tangent_stats(const eik_tangent *t, int source, eik_stats *out);

/* Number of sources S, nodes N and receivers per source held by the tangent. */
int tangent_dims(const eik_tangent *t, int *S, int64_t *N, int *n_rec);

/*
 * tangent_export -- one source's structure for bit-exact checks, into host buffers:
 *   label     [N]  SCC id (smallest node of the component), or NULL
 *   level     [N]  level of each node's component, or NULL
 *   perm      [N]  canonical position -> node, or NULL
 *   level_ptr [levels+1] first position of each level, or NULL
 *   row_ptr   [N+1], col [edges], w [edges]  gather-form rows A = I - W in natural
 *             node order (FP64 weights), each NULL-able
 *   cs        [N]  calibration c^(s) (0 on the seed row), or NULL
 * Synchronizes the device.
 */
int tangent_export(const eik_tangent *t, int source, int *label, int *level, int *perm,
                   int64_t *level_ptr, int64_t *row_ptr, int *col, double *w, double *cs);

/*
 * tangent_status -- waits for the tangent's work on `stream` and returns the first
 * device-side fault latched since the last call (EIK_ERR_TIMEOUT for a bounded wait
 * that ran out), then clears it.
 */
int tangent_status(eik_tangent *t, eik_stream stream);

/*
 * tangent_tune -- replace the run-time options of a built tangent: schedule, ctas_per_sm,
 * rhs_chunk, wait_timeout_s, item_deps, cluster_size, cluster_threads, pass_units,
 * block_lu_min, split_dirs and item_slots are taken from opts (structure options are
 * ignored).
 * Turning split_dirs on allocates the transpose's counters (synchronizes the device).
 * The level-synchronous schedule builds its step tables (about 48 bytes per row and
 * direction for FP32 traversals, 64 for FP64) at its first traversal of each precision,
 * which synchronizes the device and must not happen inside a stream capture: run one
 * traversal of that precision before capturing (the Krylov solvers' start calls do).
 * Used by the autotuner; affects later calls only.
 */
int tangent_tune(eik_tangent *t, const eik_opts *opts);

/*
 * tangent_debug_hold -- test hook for the bounded device-side waits of the persistent
 * schedule.  Raises by one the number of completed items the forward traversal waits
 * for before (source, step), so that wait can never be satisfied, and makes every item
 * wait for its whole previous level while a hold is in place: the next persistent
 * tangent_apply / tangent_solve ends after about wait_timeout_s and tangent_status
 * returns EIK_ERR_TIMEOUT.  In the level-synchronous schedule a hold makes CTA 0 skip its
 * arrival at global step `step` (either direction), so every CTA's barrier wait runs out
 * the same way.  source < 0 undoes every hold.  No fault is raised on the device; the
 * context stays usable.
 */
int tangent_debug_hold(eik_tangent *t, int source, int step);

/*
 * tangent_debug_poke_edge -- test hook of the checked build (build.py --checked) only:
 * overwrites upstream edge `edge` (index into source `source`'s forward rows, canonical
 * order) with the position `value`, so a test can show that the checked traversal reports
 * an out-of-range index (EIK_ERR_CUDA from tangent_status, "index out of range") instead of
 * reading it.  The normal build returns EIK_ERR_INVALID and changes nothing.
 * Synchronizes the device.
 */
int tangent_debug_poke_edge(eik_tangent *t, int source, long long edge, int value);

/* Release everything the tangent owns (waits for its streams). NULL is ignored. */
void tangent_free(eik_tangent *t);

/*
 * sweep_apply -- the plain form: directional Gauss-Seidel sweeping (Sec. 3.6) of the
 * same frozen A (or A^T when transpose != 0) over the 2^ndim logical orderings,
 * hyperplane-parallel on the device, all sources and right-hand sides at once, cycled
 * until max |dx| <= sweep_tol * max |x| over one full cycle.
 *   b, x     device [S][N][R] (x is overwritten; starts from 0)
 *   cycles   host, optional: cycles used
 * Returns EIK_ERR_NOT_CONVERGED at sweep_max_cycles.  Synchronizes once per cycle.
 */
int sweep_apply(eik_tangent *t, int transpose, const void *b, int R, void *x, int dtype,
                const eik_opts *opts, int *cycles, eik_stream stream);

/*
 * LSQR on the frozen Jacobian (Paige & Saunders 1982): the inner Krylov least-squares
 * solve of Sec. 4.5 / Alg. 1 step 20 (without the regularization rows), min |J x - b|
 * for a slowness-type model x [N] and data b [S][n_rec], using tangent_apply and
 * tangent_apply_T (sum over sources) with one right-hand side.  All vectors and
 * scalars stay on the device, so one iteration can be captured in a CUDA graph.
 *   lsqr_create   allocates the work vectors (owned by the solver) for tangent t;
 *                 dtype EIK_F64 or EIK_F32 (vectors and traversal precision)
 *   lsqr_start    device b [S][n_rec]: beta u = b, alpha v = J^T u, w = v, x = 0
 *   lsqr_iterate  runs `iters` iterations; use_graph != 0 captures one iteration into a
 *                 CUDA graph on the first call (stream must not be the legacy default
 *                 stream) and replays it
 *   lsqr_solution copies x (device [N], may be NULL) and, if scalars != NULL, the host
 *                 doubles {alpha, beta, rhobar, phibar, phi, rho, theta, c, s};
 *                 phibar is the current residual norm |b - J x|
 *   lsqr_free     releases the solver (not the tangent)
 */
typedef struct eik_lsqr eik_lsqr;
int lsqr_create(eik_tangent *t, int dtype, eik_lsqr **out);
int lsqr_start(eik_lsqr *l, const void *b, eik_stream stream);
int lsqr_iterate(eik_lsqr *l, int iters, int use_graph, eik_stream stream);
int lsqr_solution(eik_lsqr *l, void *x, double *scalars, eik_stream stream);
void lsqr_free(eik_lsqr *l);

/*
 * Off-grid receivers (Sec. 4.4: P_a samples the transported field at source a's
 * receivers; D_a = 0 for on-grid sources).  The paper gives no formula for receivers
 * between nodes; reading: multilinear interpolation in logical index space.
 *   tangent_set_receivers   f: host [S][n_rec][ndim] fractional logical indices of each
 *                           source's receivers, 0 <= f_d <= n_d - 1 (corner base
 *                           min(floor(f_d), n_d - 2)); n_rec = 0 clears them.  Independent
 *                           of the on-grid receivers given to tangent_build.  Synchronizes
 *                           the device.  EIK_ERR_INVALID for a coordinate out of range.
 *   tangent_apply_interp    J p with P = the multilinear sampling: ds device [N][R]
 *                           (shared_model != 0) or [S][N][R]; d_rec device [S][n_rec][R]
 *   tangent_apply_interp_T  J^T y = sum_a M^T C^T A_a^-T P_a^T y_a: y device
 *                           [S][n_rec][R], g device [N][R] (summed over sources)
 * Both follow rhs_chunk; they use an internal staging buffer of [S][N][chunk] (kept by
 * the tangent).  EIK_ERR_INVALID when no off-grid receivers are set.
 */
int tangent_set_receivers(eik_tangent *t, int n_rec, const double *f);
int tangent_apply_interp(eik_tangent *t, const void *ds, int shared_model, int R, void *d_rec, int dtype,
                         eik_stream stream);
int tangent_apply_interp_T(eik_tangent *t, const void *y, int R, void *g, int dtype, eik_stream stream);

/*
 * Cell-based velocity model (the inversion cells of Sec. 5.3, one per grid hexahedron,
 * indexed like nodes on the grid of extents n_d - 1).  The paper gives no formula for the
 * cell-to-node map; reading: a node's perturbation is the mean over its adjacent cells.
 * A Jacobian action on cells is then J (A p_cell) with the tangent's velocity model map,
 * and its transpose A^T (J^T y).
 *   model_cells_to_nodes  p_node[j][r] = mean over the cells c adjacent to node j of
 *                         p_cell[c][r]   (device [n_cells][R] -> device [N][R])
 *   model_nodes_to_cells  the transpose: g_cell[c][r] = sum over the corner nodes j of c
 *                         of g_node[j][r] / (number of cells adjacent to j)
 *                         (device [N][R] -> device [n_cells][R])
 * g: only ndim and n are read (each n_d >= 2); dtype EIK_F32 or EIK_F64 (sums in FP64);
 * asynchronous on stream; both are gathers (deterministic).
 */
int model_cells_to_nodes(const eik_grid *g, const void *p_cell, int R, void *p_node, int dtype, eik_stream stream);
int model_nodes_to_cells(const eik_grid *g, const void *g_node, int R, void *g_cell, int dtype, eik_stream stream);

/*
 * The augmented Gauss-Newton operator of Sec. 4.5 (Eq. augmented-ls, Eq.
 * augmented-actions) on a built tangent, one model vector:
 *   K p   = [ W_d J p ; lambda R p ; lambda S p ]              S = gamma diag(1 / v_k)
 *   K^T y = J^T W_d y_d + lambda R^T y_R + lambda S^T y_S      (Eq. relative-damping)
 * J is the tangent's Jacobian with its model map (the paper's model is the nodal
 * velocity: build the tangent with EIK_MODEL_VELOCITY).  R, which the paper leaves
 * undefined, is read as unit first differences along every logical axis:
 * (R p)_row = p[i + e_d] - p[i], rows axis by axis, within an axis in the linear order of
 * the lower node i; n_rough = sum over d of (n_d - 1) x prod of the other extents.
 * K-space vectors are [n_data + n_rough + N]: the data block [S][n_rec], then R's rows,
 * then the N damping rows.  Vectors are FP64 or FP32 per dtype; W_d, S and all scalars
 * are FP64.
 *   gn_create     wd: device FP64 [S][n_rec], the diagonal of W_d; vk: device FP64 [N],
 *                 the current model (positive).  Both are copied; the caller keeps them.
 *                 lambda >= 0, gamma >= 0.  The solver owns its work vectors; the tangent
 *                 must outlive it.  Synchronizes the device once.
 *   gn_dims       host outputs (each may be NULL): rows of K, data rows, roughness rows
 *   gn_apply      p device [N] -> out device [n_rows]  (K p)
 *   gn_apply_T    y device [n_rows] -> out device [N]  (K^T y)
 * LSMR (Fong & Saunders 2011; x0 = 0, no extra damping: the regularization is in K) on
 * min |K x - b|, with every vector and scalar on the device:
 *   gn_lsmr_start    b device [n_rows] (e.g. [-W_d r_k; 0; 0]): beta u = b, alpha v = K^T u
 *   gn_lsmr_iterate  runs `iters` iterations; use_graph != 0 captures one iteration into
 *                    a CUDA graph on the first call (not on the legacy default stream)
 *   gn_lsmr_solution copies x (device [N], may be NULL) and, if scalars != NULL, the host
 *                    doubles {|r_k| (recurrence), |K^T r_k|, |K| estimate (Frobenius of
 *                    the bidiagonal), |x_k|, |b|, iterations}; a caller stops when
 *                    |K^T r| <= atol |K| |r| (the paper uses 1e-4)
 *   gn_free          releases the solver (not the tangent)
 */
typedef struct eik_gn eik_gn;
int gn_create(eik_tangent *t, const double *wd, const double *vk, double lambda, double gamma, int dtype,
              eik_gn **out);
/* The same operator with the model on the cells (one per grid hexahedron, see
 * model_cells_to_nodes): K p = [W_d J A p; lambda R_c p; lambda S p], with A the node <-
 * cell map, R_c first differences on the cell grid (extents n_d - 1) and S = gamma
 * diag(1 / v_cells); v_cells device FP64 [n_cells].  Model vectors (p, K^T y, the LSMR
 * solution) are [n_cells]. */
int gn_create_cells(eik_tangent *t, const double *wd, const double *v_cells, double lambda, double gamma, int dtype,
                    eik_gn **out);
int gn_dims(const eik_gn *g, int64_t *n_rows, int64_t *n_data, int64_t *n_rough);
int gn_apply(eik_gn *g, const void *p, void *out, eik_stream stream);
int gn_apply_T(eik_gn *g, const void *y, void *out, eik_stream stream);
/* gn_rhs: the right-hand side b = [-W_d r; 0; 0] of Eq. (augmented-ls) for a data
 * residual r (device FP64 [S][n_rec]) into b (device [n_rows], the solver's dtype). */
int gn_rhs(eik_gn *g, const double *r, void *b, eik_stream stream);
int gn_lsmr_start(eik_gn *g, const void *b, eik_stream stream);
int gn_lsmr_iterate(eik_gn *g, int iters, int use_graph, eik_stream stream);
int gn_lsmr_solution(eik_gn *g, void *x, double *scalars, eik_stream stream);
void gn_free(eik_gn *g);

#ifdef __cplusplus
}
#endif
#endif /* EIK_H */
