// Phase I of Algorithm 1 on the device: metric, face-upwind rows and calibration,
// dependency graph, SCC condensation with canonical levels, block LU, traversal items.
//
// This translation unit is compiled with -fmad=false: the sign of every face
// coefficient a_f decides whether an edge exists, and it must come out of the same
// sequence of correctly rounded IEEE operations that the formulas below state.
#include <cub/cub.cuh>
#include <thrust/iterator/counting_iterator.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdarg>
#include <thread>
#include <cstdio>
#include <cstring>

#include "eik_internal.h"

namespace eik {

static thread_local std::string g_err;

void set_error(const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

const char *last_error() { return g_err.c_str(); }

int cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    return e == cudaErrorMemoryAllocation ? EIK_ERR_OOM : EIK_ERR_CUDA;
}

GridDesc make_grid_desc(const eik_grid *g)
{
    GridDesc d{};
    d.ndim = g->ndim;
    d.N = 1;
    for (int a = 0; a < 3; ++a) { d.n[a] = a < g->ndim ? g->n[a] : 1; d.dxi[a] = a < g->ndim ? g->dxi[a] : 1.0; }
    for (int a = 0; a < g->ndim; ++a) d.N *= g->n[a];
    if (g->ndim == 3) { d.st[2] = 1; d.st[1] = g->n[2]; d.st[0] = (long long)g->n[1] * g->n[2]; }
    else { d.st[1] = 1; d.st[0] = g->n[1]; d.st[2] = 0; }
    return d;
}

constexpr int INF = 0x7fffffff;

__device__ __forceinline__ void node_coords(const GridDesc &g, long long i, int *c)
{
    if (g.ndim == 3) { c[2] = (int)(i % g.n[2]); c[1] = (int)((i / g.n[2]) % g.n[1]); c[0] = (int)(i / g.st[0]); }
    else { c[1] = (int)(i % g.n[1]); c[0] = (int)(i / g.n[1]); c[2] = 0; }
}

// derivative along logical axis `ax` of component `comp` of an interleaved field:
// central difference inside, second-order one-sided difference on the two edges
__device__ double axis_derivative(const double *f, int ncomp, int comp, long long i, int at, int nax,
                                  long long step, double h)
{
    double num;
    if (at == 0) {
        num = (-3.0 * f[i * ncomp + comp] + 4.0 * f[(i + step) * ncomp + comp]) - f[(i + 2 * step) * ncomp + comp];
    } else if (at == nax - 1) {
        num = (3.0 * f[i * ncomp + comp] - 4.0 * f[(i - step) * ncomp + comp]) + f[(i - 2 * step) * ncomp + comp];
    } else {
        num = f[(i + step) * ncomp + comp] - f[(i - step) * ncomp + comp];
    }
    return num / (2.0 * h);
}

// ---------------------------------------------------------------------------
// Sec. 2.2, Eq. (metric-eikonal): Jm = dx/dxi (finite differences of the node
// coordinates), Kinv = Jm^-1 by the adjugate, G = Kinv Kinv^T.
// ---------------------------------------------------------------------------
__global__ void k_metric(GridDesc g, const double *__restrict__ xyz, double *__restrict__ G,
                         double *__restrict__ Jout)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    int c[3];
    node_coords(g, i, c);
    const int nd = g.ndim;
    double Jm[3][3];
    for (int a = 0; a < nd; ++a)
        for (int b = 0; b < nd; ++b) Jm[a][b] = axis_derivative(xyz, nd, a, i, c[b], g.n[b], g.st[b], g.dxi[b]);
    if (nd == 3) {
        double m00 = Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1];
        double m01 = Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2];
        double m02 = Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0];
        double m10 = Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2];
        double m11 = Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0];
        double m12 = Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1];
        double m20 = Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1];
        double m21 = Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2];
        double m22 = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
        double det = (Jm[0][0] * m00 + Jm[0][1] * m01) + Jm[0][2] * m02;
        double K[3][3] = {{m00 / det, m10 / det, m20 / det},
                          {m01 / det, m11 / det, m21 / det},
                          {m02 / det, m12 / det, m22 / det}};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                G[i * 9 + a * 3 + b] = (K[a][0] * K[b][0] + K[a][1] * K[b][1]) + K[a][2] * K[b][2];
    } else {
        double det = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
        double K[2][2] = {{Jm[1][1] / det, -Jm[0][1] / det}, {-Jm[1][0] / det, Jm[0][0] / det}};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) G[i * 4 + a * 2 + b] = K[a][0] * K[b][0] + K[a][1] * K[b][1];
    }
    if (Jout)
        for (int a = 0; a < nd; ++a)
            for (int b = 0; b < nd; ++b) Jout[i * nd * nd + a * nd + b] = Jm[a][b];
}

// nodal logical gradient of T for every source: gT [S][N][ndim]
__global__ void k_grad(GridDesc g, int S, const double *__restrict__ T, double *__restrict__ gT)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= g.N * S) return;
    long long a = v / g.N, i = v - a * g.N;
    int c[3];
    node_coords(g, i, c);
    const double *Ta = T + a * g.N;
    for (int b = 0; b < g.ndim; ++b)
        gT[v * g.ndim + b] = axis_derivative(Ta, 1, 0, i, c[b], g.n[b], g.st[b], g.dxi[b]);
}

// ---------------------------------------------------------------------------
// Sec. 3.1-3.2: face-based upwind rows and calibration, one thread per (source, node).
// Faces are visited axis ascending, lower side first.  For neighbour j across a face
// normal to axis d: the face metric row and gradient are the averages of the two
// nodes, except the normal gradient component, which is the compact difference across
// the face; a_f = sum_b Gf[d][b] gf[b]; j is upstream iff -side * a_f > 0, with
// coupling c = -side * a_f / h_d.  Row: d_i = sum c, w = c / d_i; l_i = T_i - sum w T_j,
// cs_i = l_i / s_i.  Seed rows (the source node, or the cell corners of a point source:
// seeds [S][8], -1 padded) are identities with cs = 0; a non-seed row without an upstream
// face is an identity with cs = T_i / s_i.
// upmask bit (2 d + (side > 0)) marks an upstream face.
// ---------------------------------------------------------------------------
__global__ void k_assemble(GridDesc g, int S, const double *__restrict__ G, const double *__restrict__ gT,
                           const double *__restrict__ T, const double *__restrict__ s, const int *__restrict__ seeds,
                           int *__restrict__ cnt, int *__restrict__ nnode, double *__restrict__ nw,
                           unsigned char *__restrict__ upmask, double *__restrict__ cs,
                           unsigned long long *__restrict__ n_identity)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= g.N * S) return;
    const int nd = g.ndim, nd2 = nd * nd, slots = 2 * nd;
    long long a = v / g.N, i = v - a * g.N;
    const double *Ta = T + a * g.N;
    const double *gTa = gT + a * g.N * nd;
    bool seed = false;
    for (int q = 0; q < 8; ++q) seed = seed || seeds[a * 8 + q] == i;
    if (seed) {
        cnt[v] = 0; upmask[v] = 0; cs[v] = 0.0;
        return;
    }
    int c[3];
    node_coords(g, i, c);
    int m = 0;
    unsigned char mask = 0;
    double cw[6];
    int nb[6];
    for (int d = 0; d < nd; ++d) {
        for (int side = -1; side <= 1; side += 2) {
            int at = c[d] + side;
            if (at < 0 || at >= g.n[d]) continue;
            long long j = i + side * g.st[d];
            double gf[3];
            for (int b = 0; b < nd; ++b) gf[b] = (gTa[i * nd + b] + gTa[j * nd + b]) * 0.5;
            gf[d] = side < 0 ? (Ta[i] - Ta[j]) / g.dxi[d] : (Ta[j] - Ta[i]) / g.dxi[d];
            double af = 0.0;
            for (int b = 0; b < nd; ++b) {
                double Gf = (G[i * nd2 + d * nd + b] + G[j * nd2 + d * nd + b]) * 0.5;
                af = af + Gf * gf[b];
            }
            double up = side < 0 ? af : -af;
            if (up > 0.0) {
                nb[m] = (int)j;
                cw[m] = up / g.dxi[d];
                mask |= (unsigned char)(1u << (2 * d + (side > 0)));
                ++m;
            }
        }
    }
    cnt[v] = m;
    upmask[v] = mask;
    if (m == 0) {
        cs[v] = Ta[i] / s[i];
        atomicAdd(n_identity + a, 1ull);
        return;
    }
    double dsum = 0.0;
    for (int e = 0; e < m; ++e) dsum = dsum + cw[e];
    double acc = 0.0;
    for (int e = 0; e < m; ++e) {
        double w = cw[e] / dsum;
        nnode[v * slots + e] = nb[e];
        nw[v * slots + e] = w;
        acc = acc + w * Ta[nb[e]];
    }
    cs[v] = (Ta[i] - acc) / s[i];
}

// ---------------------------------------------------------------------------
// Dependency graph helpers.  Global vertex id v = source * N + node; an edge u -> v
// exists iff bit (2 d + (side > 0)) of upmask[v] is set with u = v + side * st[d].
// ---------------------------------------------------------------------------
template <typename F>
__device__ __forceinline__ void for_preds(const GridDesc &g, long long v, unsigned char mask, F f)
{
    for (int b = 0; b < 2 * g.ndim; ++b)
        if (mask & (1u << b)) {
            int d = b >> 1, side = (b & 1) ? 1 : -1;
            f(v + side * g.st[d]);
        }
}

// successors u of v: neighbours whose upstream face points back at v
template <typename F>
__device__ __forceinline__ void for_succs(const GridDesc &g, long long v, const unsigned char *upmask, F f)
{
    int c[3];
    node_coords(g, v % g.N, c);
    for (int d = 0; d < g.ndim; ++d)
        for (int side = -1; side <= 1; side += 2) {
            int at = c[d] + side;
            if (at < 0 || at >= g.n[d]) continue;
            long long u = v + side * g.st[d];
            if (upmask[u] & (1u << (2 * d + (side < 0)))) f(u);
        }
}

// ---------------------------------------------------------------------------
// Kahn trimming with frontier queues (Sec. 3.5, Prop. 2): each round removes the
// vertices whose last remaining predecessor (successor) was removed in the previous
// round, so the total work is O(V + E) instead of one pass over all vertices per round.
// fst[v] = Kahn round of v = 1 + max over predecessors (0 without predecessor), INF for
// the downstream closure of the cycles; bst likewise from the sinks of that residual.
// The values do not depend on the order inside a frontier.
// ---------------------------------------------------------------------------
__global__ void k_trim_fwd_init(long long SN, const unsigned char *__restrict__ upmask, int *deg, int *fst, int *front,
                                int *nfront)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= SN) return;
    const int d = __popc((unsigned)upmask[v]);
    deg[v] = d;
    fst[v] = INF;
    if (d == 0) { fst[v] = 0; front[atomicAdd(nfront, 1)] = (int)v; }
}

__global__ void k_trim_fwd_step(GridDesc g, const unsigned char *__restrict__ upmask, int *deg, int *fst,
                                const int *__restrict__ cur, const int *ncur, int *next, int *nnext, int round)
{
    const int n = *ncur;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const long long v = cur[k];
        for_succs(g, v, upmask, [&](long long u) {
            if (atomicSub(&deg[u], 1) == 1) { fst[u] = round + 1; next[atomicAdd(nnext, 1)] = (int)u; }
        });
    }
}

__global__ void k_trim_bwd_init(GridDesc g, long long SN, const unsigned char *__restrict__ upmask,
                                const int *__restrict__ fst, int *deg, int *bst, int *front, int *nfront)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= SN) return;
    bst[v] = INF;
    if (fst[v] != INF) return;
    int d = 0;
    for_succs(g, v, upmask, [&](long long u) { if (fst[u] == INF) ++d; });
    deg[v] = d;
    if (d == 0) { bst[v] = 0; front[atomicAdd(nfront, 1)] = (int)v; }
}

__global__ void k_trim_bwd_step(GridDesc g, const unsigned char *__restrict__ upmask, const int *__restrict__ fst,
                                int *deg, int *bst, const int *__restrict__ cur, const int *ncur, int *next, int *nnext,
                                int round)
{
    const int n = *ncur;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const long long v = cur[k];
        for_preds(g, v, upmask[v], [&](long long u) {
            if (fst[u] == INF && atomicSub(&deg[u], 1) == 1) { bst[u] = round + 1; next[atomicAdd(nnext, 1)] = (int)u; }
        });
    }
}

// residual flag (in both closures: downstream and upstream of a cycle) and labels of
// every vertex outside it (singleton components: the vertex itself)
__global__ void k_residual_flags(long long SN, const int *__restrict__ fst, const int *__restrict__ bst,
                                 unsigned char *flag, int *label)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= SN) return;
    const bool r = fst[v] == INF && bst[v] == INF;
    flag[v] = r;
    label[v] = (int)v;
}

__global__ void k_gather_masks(const int *__restrict__ list, int n, const unsigned char *__restrict__ upmask,
                               unsigned char *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = upmask[list[k]];
}

__global__ void k_scatter_labels(const int *__restrict__ list, const int *__restrict__ lab_res, int n, int *label)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) label[list[k]] = lab_res[k];
}

__global__ void k_comp_size(long long SN, const int *__restrict__ label, int *csize)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= SN) return;
    atomicAdd(&csize[label[v]], 1);
}

// ---------------------------------------------------------------------------
// Canonical levels (longest path in the condensation DAG): a component's level is 1 +
// the largest level among its external predecessor components (0 without one).  The
// per-component values live at the component's root vertex.
// ---------------------------------------------------------------------------
__global__ void k_lvl_init(long long SN, const int *__restrict__ fst, const int *__restrict__ label, int *lvl, int *asg,
                           int *cmax, int *blk, int *list, int *count)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= SN) return;
    // vertices removed by forward Kahn are singletons with all ancestors removed too:
    // their Kahn round is their longest-path level
    if (fst[v] != INF) { lvl[v] = fst[v]; asg[v] = -1; }
    else {
        if (label[v] == v) { asg[v] = INF; cmax[v] = -1; blk[v] = 0; }
        int k = atomicAdd(count, 1);
        list[k] = (int)v;
    }
}

__global__ void k_node_level(long long SN, long long N, const int *__restrict__ label, const int *__restrict__ lvl,
                             int *level, int *lmax)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= SN) return;
    int L = lvl[label[v]];
    level[v] = L;
    long long a = v / N;
    atomicMax(&lmax[a], L);
}

// sort key: (source, level) segment | component id (local smallest node) | node, the last
// two in nb bits each (nb = bits of N - 1), the segment above them
__global__ void k_keys(long long SN, long long N, int maxL, int nb, const int *__restrict__ label,
                       const int *__restrict__ level, unsigned long long *keys)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= SN) return;
    long long a = v / N;
    unsigned long long seg = (unsigned long long)(a * maxL + level[v]);
    unsigned long long comp = (unsigned long long)(label[v] - a * N);
    unsigned long long node = (unsigned long long)(v - a * N);
    keys[v] = (seg << (2 * nb)) | (comp << nb) | node;
}

__global__ void k_perm(long long SN, long long N, int maxL, int nb, const unsigned long long *__restrict__ skeys,
                       const int *__restrict__ label, const int *__restrict__ csize, int *perm, int *pos, int *lcount,
                       int *head)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= SN) return;
    unsigned long long key = skeys[p];
    long long a = p / N, pl = p - a * N;
    const unsigned long long mask = (1ull << nb) - 1;
    int node = (int)(key & mask);
    int seg = (int)(key >> (2 * nb));
    long long v = a * N + node;
    bool member = csize[label[v]] > 1;
    perm[p] = member ? ~node : node;
    pos[v] = (int)pl;
    atomicAdd(&lcount[seg], 1);
    int is_head = 0;
    if (member) {
        if (pl == 0) is_head = 1;
        else {
            int prev = (int)(skeys[p - 1] & mask);
            is_head = label[a * N + prev] != label[v];
        }
    }
    head[p] = is_head;
}

// per position: forward edge count (external only for block members) and transposed count
__global__ void k_counts(GridDesc g, long long SN, const int *__restrict__ perm, const int *__restrict__ label,
                         const int *__restrict__ cnt, const int *__restrict__ nnode, const unsigned char *__restrict__ upmask,
                         int *fcnt, int *tcnt)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= SN) return;
    long long a = p / g.N;
    int pn = perm[p];
    bool member = pn < 0;
    long long v = a * g.N + (member ? ~pn : pn);
    const int slots = 2 * g.ndim;
    int f = 0;
    for (int e = 0; e < cnt[v]; ++e) {
        long long u = a * g.N + nnode[v * slots + e];
        if (!member || label[u] != label[v]) ++f;
    }
    int tc = 0;
    for_succs(g, v, upmask, [&](long long u) { if (!member || label[u] != label[v]) ++tc; });
    fcnt[p] = f;
    tcnt[p] = tc;
}

__global__ void k_fill(GridDesc g, long long SN, const int *__restrict__ perm, const int *__restrict__ pos, const int *__restrict__ label,
                       const int *__restrict__ cnt, const int *__restrict__ nnode, const double *__restrict__ nw,
                       const unsigned char *__restrict__ upmask, const long long *__restrict__ fscan,
                       const long long *__restrict__ tscan, const long long *__restrict__ fbase,
                       const long long *__restrict__ tbase, int *rowptr, int *cptr, int *up_node, float *up_w32,
                       double *up_w64, int *dn_node, float *dn_w32, double *dn_w64)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= SN) return;
    long long a = p / g.N, pl = p - a * g.N;
    int pn = perm[p];
    bool member = pn < 0;
    long long v = a * g.N + (member ? ~pn : pn);
    const int slots = 2 * g.ndim;
    long long fo = fscan[p], to = tscan[p];
    rowptr[a * (g.N + 1) + pl] = (int)(fo - fbase[a]);
    cptr[a * (g.N + 1) + pl] = (int)(to - tbase[a]);
    if (pl == g.N - 1) {
        rowptr[a * (g.N + 1) + g.N] = (int)(fbase[a + 1] - fbase[a]);
        cptr[a * (g.N + 1) + g.N] = (int)(tbase[a + 1] - tbase[a]);
    }
    for (int e = 0; e < cnt[v]; ++e) {
        int j = nnode[v * slots + e];
        long long u = a * g.N + j;
        if (member && label[u] == label[v]) continue;
        double w = nw[v * slots + e];
        up_node[fo] = pos[u];            // the traversal's workspace is in canonical order
        up_w64[fo] = w;
        up_w32[fo] = (float)w;
        ++fo;
    }
    const int self = (int)(v - a * g.N);
    for_succs(g, v, upmask, [&](long long u) {
        if (member && label[u] == label[v]) return;
        double w = 0.0;
        for (int e = 0; e < cnt[u]; ++e)
            if (nnode[u * slots + e] == self) w = nw[u * slots + e];
        dn_node[to] = pos[u];
        dn_w64[to] = w;
        dn_w32[to] = (float)w;
        ++to;
    });
}

// calibration times model map, per position and per node (Sec. 3.2 and Sec. 2.3)
__global__ void k_cq(long long SN, long long N, int model, const int *__restrict__ perm, const double *__restrict__ cs,
                     const double *__restrict__ s, double *cq64, float *cq32, double *cqn64, float *cqn32)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= SN) return;
    long long a = p / N, pl = p - a * N;
    // natural-order entry for node pl
    {
        double si = s[pl];
        double m = model == EIK_MODEL_SLOWNESS ? 1.0 : (model == EIK_MODEL_VELOCITY ? -(si * si) : -si);
        double c = cs[p] * m;
        cqn64[p] = c;
        cqn32[p] = (float)c;
    }
    int pn = perm[p];
    long long i = pn < 0 ? ~pn : pn;
    double si = s[i];
    double m = model == EIK_MODEL_SLOWNESS ? 1.0 : (model == EIK_MODEL_VELOCITY ? -(si * si) : -si);
    double c = cs[a * N + i] * m;
    cq64[p] = c;
    cq32[p] = (float)c;
}

__global__ void k_rec_mark(int S, long long N, int n_rec, const int *__restrict__ rec, int *recpos, int *bad)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= (long long)S * n_rec) return;
    long long a = k / n_rec;
    int r = (int)(k - a * n_rec);
    int node = rec[k];
    if (node < 0 || node >= N) { atomicExch(bad, 1); return; }
    if (atomicCAS(&recpos[a * N + node], -1, r) != -1) atomicExch(bad, 2);
}

__global__ void k_rec_slot(long long SN, long long N, const int *__restrict__ perm, const int *__restrict__ recpos,
                           int *rec_slot)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= SN) return;
    long long a = p / N;
    int pn = perm[p];
    rec_slot[p] = recpos[a * N + (pn < 0 ? ~pn : pn)];
}

// dense A_C = I - W_CC of every nontrivial block (nodes ascending = positions p0..p0+k-1)
__global__ void k_block_fill(GridDesc g, const int4 *__restrict__ desc, const long long *__restrict__ off,
                             const int *__restrict__ perm, const int *__restrict__ pos, const int *__restrict__ label,
                             const int *__restrict__ cnt, const int *__restrict__ nnode, const double *__restrict__ nw,
                             double *lu)
{
    int b = blockIdx.x;
    int4 d = desc[b];
    int a = d.x, p0 = d.y, k = d.z;
    double *A = lu + off[3 * b + 0];
    for (long long e = threadIdx.x; e < (long long)k * k; e += blockDim.x) A[e] = (e / k == e % k) ? 1.0 : 0.0;
    __syncthreads();
    const int slots = 2 * g.ndim;
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        long long v = a * g.N + ~perm[a * g.N + p0 + r];
        for (int e = 0; e < cnt[v]; ++e) {
            long long u = a * g.N + nnode[v * slots + e];
            if (label[u] != label[v]) continue;
            int c = pos[u] - p0;
            A[(long long)r * k + c] -= nw[v * slots + e];
        }
    }
}

// Sec. 4.3: P_C A_C = L_C U_C with partial pivoting (first largest |a| on ties)
__global__ void k_block_lu(const int4 *__restrict__ desc, const long long *__restrict__ off, double *lu, int *piv,
                           double tol, int *err)
{
    int b = blockIdx.x;
    int k = desc[b].z;
    double *A = lu + off[3 * b + 0];
    int *P = piv + off[3 * b + 1];
    __shared__ double s_val[256];
    __shared__ int s_idx[256];
    __shared__ int s_p;
    for (int r = 0; r < k; ++r) {
        double best = -1.0;
        int bi = k;
        for (int t = r + threadIdx.x; t < k; t += blockDim.x) {
            double x = fabs(A[(long long)t * k + r]);
            if (x > best) { best = x; bi = t; }
        }
        s_val[threadIdx.x] = best;
        s_idx[threadIdx.x] = bi;
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) {
                double o = s_val[threadIdx.x + h];
                int oi = s_idx[threadIdx.x + h];
                if (o > s_val[threadIdx.x] || (o == s_val[threadIdx.x] && oi < s_idx[threadIdx.x])) {
                    s_val[threadIdx.x] = o;
                    s_idx[threadIdx.x] = oi;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s_p = s_idx[0];
            P[r] = s_p;
            if (!(s_val[0] >= tol)) atomicCAS(err, 0, DEV_SINGULAR);
        }
        __syncthreads();
        int p = s_p;
        if (p != r)
            for (int c = threadIdx.x; c < k; c += blockDim.x) {
                double x = A[(long long)r * k + c];
                A[(long long)r * k + c] = A[(long long)p * k + c];
                A[(long long)p * k + c] = x;
            }
        __syncthreads();
        double pv = A[(long long)r * k + r];
        for (int t = r + 1 + threadIdx.x; t < k; t += blockDim.x) A[(long long)t * k + r] /= pv;
        __syncthreads();
        long long rem = (long long)(k - r - 1) * (k - r - 1);
        for (long long e = threadIdx.x; e < rem; e += blockDim.x) {
            int t = r + 1 + (int)(e / (k - r - 1)), c = r + 1 + (int)(e % (k - r - 1));
            A[(long long)t * k + c] -= A[(long long)t * k + r] * A[(long long)r * k + c];
        }
        __syncthreads();
    }
}

// Longest-path levels of the components downstream of the cycles by component-level
// Kahn with frontier queues: pend[c] counts the edges into component c from other
// components of the level list, cmax[c] is the largest level among c's predecessors;
// a component enters the frontier when its last such edge is resolved, takes level
// cmax + 1, and resolves the edges leaving its members.  Values live at the root.
__global__ void k_lvl_count(GridDesc g, const int *__restrict__ list, int n, const unsigned char *__restrict__ upmask,
                            const int *__restrict__ fst, const int *__restrict__ label, int *pend, int *cmax)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long v = list[k];
    const int c = label[v];
    for_preds(g, v, upmask[v], [&](long long u) {
        const int cu = label[u];
        if (cu == c) return;
        if (fst[u] != INF) atomicMax(&cmax[c], fst[u]);   // a trimmed singleton: its level is its Kahn round
        else atomicAdd(&pend[c], 1);
    });
}

__global__ void k_lvl_front0(const int *__restrict__ list, int n, const int *__restrict__ label,
                             const int *__restrict__ pend, int *front, int *nfront)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int v = list[k];
    if (label[v] == v && pend[v] == 0) front[atomicAdd(nfront, 1)] = v;
}

// list vertices that belong to a nontrivial component, and their roots
__global__ void k_nontrivial_flags(const int *__restrict__ list, int n, const int *__restrict__ label,
                                   const int *__restrict__ csize, unsigned char *flag, int *root)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int c = label[list[k]];
    flag[k] = csize[c] > 1;
    root[k] = c;
}

// members of the nontrivial components, grouped by root: moff[root] = first position
__global__ void k_member_offsets(const int *__restrict__ roots, int n, int *moff)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (i == 0 || roots[i] != roots[i - 1])) moff[roots[i]] = i;
}

__global__ void k_lvl_step(GridDesc g, const unsigned char *__restrict__ upmask, const int *__restrict__ label,
                           const int *__restrict__ csize, const int *__restrict__ moff, const int *__restrict__ members,
                           int *lvl, int *asg, int *cmax, int *pend, const int *__restrict__ cur, const int *ncur, int *next,
                           int *nnext, int round)
{
    const int n = *ncur;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int c = cur[k];
        const int L = cmax[c] + 1;
        lvl[c] = L;
        asg[c] = round;
        const int sz = csize[c];
        for (int m = 0; m < sz; ++m) {
            const long long v = sz == 1 ? c : members[moff[c] + m];
            for_succs(g, v, upmask, [&](long long u) {
                const int cu = label[u];
                if (cu == c) return;
                atomicMax(&cmax[cu], L);
                if (atomicSub(&pend[cu], 1) == 1) next[atomicAdd(nnext, 1)] = cu;
            });
        }
    }
}

__global__ void k_check_assigned(long long SN, const int *label, const int *asg, int *bad)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= SN) return;
    if (label[v] == v && asg[v] == INF) atomicAdd(bad, 1);
}

// per-source sums of a per-vertex count: the lanes of a warp that belong to the same
// source (almost always all of them) are summed first, one atomic per source and warp
__device__ __forceinline__ void add_per_source(long long v, long long SN, long long N, unsigned long long x,
                                               unsigned long long *sum)
{
    const long long a = v < SN ? v / N : -1;
    const unsigned full = 0xffffffffu;
    const long long a0 = __shfl_sync(full, a, 0);
    if (__all_sync(full, a == a0)) {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(full, x, o);
        if ((threadIdx.x & 31) == 0 && a0 >= 0 && x) atomicAdd(&sum[a0], x);
    } else if (a >= 0 && x) {
        atomicAdd(&sum[a], x);
    }
}

__global__ void k_count_roots(long long SN, long long N, const int *label, unsigned long long *nroots)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    add_per_source(v, SN, N, (v < SN && label[v] == v) ? 1ull : 0ull, nroots);
}

__global__ void k_count_edges(long long SN, long long N, const int *cnt, unsigned long long *ne)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    add_per_source(v, SN, N, v < SN ? (unsigned long long)cnt[v] : 0ull, ne);
}

__global__ void k_local_labels(long long SN, long long N, int *label)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= SN) return;
    label[v] -= (int)((v / N) * N);
}


__global__ void k_item_edges(int n, long long N, const int4 *items, const int *rowptr, int2 *eb)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 it = items[i];
    if (it.z < 0) { eb[i] = make_int2(0, 0); return; }
    const int *rp = rowptr + (long long)it.x * (N + 1);
    eb[i] = make_int2(rp[it.z], rp[it.w]);
}

// A_C^-1 from the factors P A_C = L U: column c of the inverse solves A_C x = e_c
// (row swaps, then L, then U), one column per thread, written in place into column c of
// the row-major k x k result.
__global__ void k_block_inverse(const int4 *__restrict__ desc, const long long *__restrict__ off,
                                const double *__restrict__ lu, const int *__restrict__ piv, double *inv)
{
    int b = blockIdx.x;
    int k = desc[b].z;
    const double *LU = lu + off[3 * b + 0];
    const int *P = piv + off[3 * b + 1];
    double *X = inv + off[3 * b + 0];
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        for (int m = 0; m < k; ++m) X[(long long)m * k + c] = m == c ? 1.0 : 0.0;
        for (int m = 0; m < k; ++m) {
            int q = P[m];
            if (q != m) {
                double t = X[(long long)m * k + c];
                X[(long long)m * k + c] = X[(long long)q * k + c];
                X[(long long)q * k + c] = t;
            }
        }
        for (int m = 0; m < k; ++m) {
            double acc = X[(long long)m * k + c];
            for (int j = 0; j < m; ++j) acc -= LU[(long long)m * k + j] * X[(long long)j * k + c];
            X[(long long)m * k + c] = acc;
        }
        for (int m = k - 1; m >= 0; --m) {
            double acc = X[(long long)m * k + c];
            for (int j = m + 1; j < k; ++j) acc -= LU[(long long)m * k + j] * X[(long long)j * k + c];
            X[(long long)m * k + c] = acc / LU[(long long)m * k + m];
        }
    }
}

// Item index of every canonical position, one direction's item list.  A singleton
// item's range also spans the members of the level's nontrivial blocks (perm < 0),
// which belong to their block items instead.
__global__ void k_item_of_pos(int n, long long N, const int4 *__restrict__ items, const int4 *__restrict__ blk_desc,
                              const int *__restrict__ perm, int *iop)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 it = items[i];
    const bool blk = it.z < 0;
    int p0, p1;
    if (!blk) { p0 = it.z; p1 = it.w; }
    else { int4 d = blk_desc[~it.z]; p0 = d.y; p1 = d.y + d.z; }
    const long long o = (long long)it.x * N;
    for (int p = p0; p < p1; ++p)
        if (blk || perm[o + p] >= 0) iop[o + p] = i;
}

// The distinct items holding the upstream positions of the rows item i computes (all
// at lower steps, hence lower tickets); -1 when there are more than DEP_MAX.
__global__ void k_item_deps(int n, long long N, const int4 *__restrict__ items, const int4 *__restrict__ blk_desc,
                            const int *__restrict__ perm, const int *__restrict__ rowptr, const int *__restrict__ enode,
                            const long long *__restrict__ ebase, const int *__restrict__ iop, int *deps, int *ndeps)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 it = items[i];
    const bool blk = it.z < 0;
    int p0, p1;
    if (!blk) { p0 = it.z; p1 = it.w; }
    else { int4 d = blk_desc[~it.z]; p0 = d.y; p1 = d.y + d.z; }
    const long long o = (long long)it.x * N;
    const int *rp = rowptr + (long long)it.x * (N + 1);
    const int *en = enode + ebase[it.x];
    const int *io = iop + o;
    int m = 0;
    int *out = deps + (long long)i * DEP_MAX;
    for (int p = p0; p < p1 && m >= 0; ++p) {
        if (!blk && perm[o + p] < 0) continue;
        for (int e = rp[p]; e < rp[p + 1]; ++e) {
            int d = io[en[e]];
            if (d == i) continue;
            bool seen = false;
            for (int q = 0; q < m; ++q) if (out[q] == d) { seen = true; break; }
            if (seen) continue;
            if (m == DEP_MAX) { m = -1; break; }
            out[m++] = d;
        }
    }
    ndeps[i] = m;
}

__global__ void k_compact_heads(long long SN, const int *head, const int *scan, int *hpos)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p < SN && head[p]) hpos[scan[p]] = (int)p;
}

__global__ void k_block_info(int nb, long long N, const int *hpos, const int *perm, const int *label, const int *level,
                             const int *csize, int4 *info)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    long long p = hpos[b];
    long long a = p / N;
    long long v = a * N + ~perm[p];
    info[b] = make_int4((int)a, (int)(p - a * N), csize[label[v]], level[v]);
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
namespace {

struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch() { for (void *p : ptrs) cudaFree(p); }
    template <typename T>
    cudaError_t get(T **p, size_t n)
    {
        cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

// Tangent arrays carry 64 bytes of tail padding: the traversal stages slices of them with
// 16-byte-granular bulk copies whose last granule may extend past the final element.
template <typename T>
cudaError_t dalloc(T **p, size_t n) { return cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T) + 64); }

inline unsigned blocks_for(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Tarjan's algorithm (Sec. 4.1 [ref50]), iterative, on the residual vertices of one
// source: `nodes` ascending (global indices), `masks` their upwind-face bits; the edges
// are the upwind faces whose neighbour is also residual.  Writes for every vertex the
// smallest global index of its strongly connected component (the canonical label).
void tarjan_residual(const GridDesc &g, const int *nodes, const unsigned char *masks, int n, int *out,
                     std::vector<int> &where)
{
    // where[local node] = position in `nodes` (a reusable [N] map, -1 outside the residual)
    const long long base = (long long)nodes[0] / g.N * g.N;
    for (int k = 0; k < n; ++k) where[nodes[k] - base] = k;
    std::vector<int> index(n, -1), low(n), stk;
    std::vector<char> on(n, 0);
    struct Frame { int v; int b; };
    std::vector<Frame> cs;
    int counter = 0;
    auto find = [&](long long u) -> int { return where[u - base]; };
    for (int r = 0; r < n; ++r) {
        if (index[r] >= 0) continue;
        index[r] = low[r] = counter++;
        stk.push_back(r);
        on[r] = 1;
        cs.push_back({r, 0});
        while (!cs.empty()) {
            const int v = cs.back().v;
            int w = -1;
            while (cs.back().b < 2 * g.ndim) {
                const int b = cs.back().b++;
                if (!(masks[v] & (1u << b))) continue;
                const int d = b >> 1, side = (b & 1) ? 1 : -1;
                const int u = find((long long)nodes[v] + side * g.st[d]);
                if (u < 0) continue;
                if (index[u] < 0) { w = u; break; }
                if (on[u]) low[v] = std::min(low[v], index[u]);
            }
            if (w >= 0) {   // descend
                index[w] = low[w] = counter++;
                stk.push_back(w);
                on[w] = 1;
                cs.push_back({w, 0});
                continue;
            }
            if (low[v] == index[v]) {   // v roots a component: pop it
                int m = nodes[v];
                for (size_t k = stk.size(); k-- > 0;) {
                    m = std::min(m, nodes[stk[k]]);
                    if (stk[k] == v) break;
                }
                for (;;) {
                    const int x = stk.back();
                    stk.pop_back();
                    on[x] = 0;
                    out[x] = m;
                    if (x == v) break;
                }
            }
            cs.pop_back();
            if (!cs.empty()) { const int p = cs.back().v; low[p] = std::min(low[p], low[v]); }
        }
    }
    for (int k = 0; k < n; ++k) where[nodes[k] - base] = -1;
}

}  // namespace

void free_tangent(Tangent *t)
{
    if (!t) return;
    void *ptrs[] = {t->perm, t->pos, t->label, t->level, t->rowptr, t->up_node, t->up_w32, t->up_w64, t->cptr,
                    t->dn_node, t->dn_w32, t->dn_w64, t->cq64, t->cq32, t->cqn64, t->cqn32, t->rec_slot,
                    t->rec_nat, t->nrow_cnt, t->nrow_node, t->nrow_w, t->cs_nat, t->blk_desc, t->blk_off, t->lu,
                    t->binv, t->piv, t->items_fwd, t->items_bwd, t->ebeg_fwd, t->ebeg_bwd, t->deps_fwd, t->deps_bwd,
                    t->ndeps_fwd, t->ndeps_bwd, t->item_done, t->item_cnt, t->done, t->ticket, t->err, t->ws_vec,
                    t->ws_blk, t->ebase_d, t->tbase_d, t->ip_node, t->ip_w, t->ipt_node, t->ipt_ptr, t->ipt_e,
                    t->ws_in, t->lvl_d, t->blk_lvl_d, t->nlev_d, t->order_d};
    for (void *p : ptrs) if (p) cudaFree(p);
    free_point_data(t->pts);
    void *lane[] = {t->lane_t.ws_vec, t->lane_t.ws_blk, t->lane_t.item_done, t->lane_t.done, t->lane_t.ticket};
    for (void *p : lane) if (p) cudaFree(p);
    void *sync[] = {t->sync_rec[0][0], t->sync_rec[0][1], t->sync_rec[1][0], t->sync_rec[1][1], t->sync_base[0],
                     t->sync_base[1], t->sync_bar, t->batch_buf};
    for (void *p : sync) if (p) cudaFree(p);
    if (t->params_d) cudaFree((void *)t->params_d);
    for (void *p : t->sweep_w) if (p) cudaFree(p);
    if (t->sweep_flags) cudaFree(t->sweep_flags);
    for (auto &kv : t->sweep_graphs) if (kv.second) cudaGraphExecDestroy(kv.second);
    for (auto &kv : t->level_graphs) if (kv.second) cudaGraphExecDestroy(kv.second);
    if (t->cap_stream) cudaStreamDestroy(t->cap_stream);
    delete t;
}

int build_tangent(const eik_grid *gin, const double *T, const double *s, int S, const int *src_node,
                  const int *rec_node, int n_rec, const eik_opts *opts, Tangent **out, cudaStream_t st,
                  const double *src_f)
{
    NvtxRange range(src_f ? "tangent_build_points" : "tangent_build");
    NvtxPhase phase;
    *out = nullptr;
    GridDesc g = make_grid_desc(gin);
    const long long N = g.N, SN = N * (long long)S;
    const int nd = g.ndim, slots = 2 * nd;
    if (SN >= (1ll << 31)) { set_error("sources x nodes = %lld; at most 2^31 - 1 supported", SN); return EIK_ERR_INVALID; }
    if (!src_f)
        for (int a = 0; a < S; ++a)
            if (src_node[a] < 0 || src_node[a] >= N) { set_error("source %d node %d out of range", a, src_node[a]); return EIK_ERR_INVALID; }

    Tangent *t = new Tangent();
    t->S = S; t->N = N; t->n_rec = n_rec; t->grid = g; t->opts = *opts; t->model = opts->model;
    cudaGetDevice(&t->device);
    cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, t->device);
    auto fail = [&](int code) { free_tangent(t); return code; };
#define TRY(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return fail(cuda_fail(e_, #call, __FILE__, __LINE__)); } while (0)

    Scratch sc;
    double *G, *gT;
    int *cnt, *fst, *bst, *flags, *src_d, *lab, *act, *color, *list, *csize, *lvl, *asg, *cmax, *blk, *lmax;
    unsigned char *upmask;
    unsigned long long *nid;
    TRY(sc.get(&G, N * nd * nd));
    TRY(sc.get(&gT, SN * nd));
    TRY(sc.get(&upmask, SN));
    TRY(sc.get(&fst, SN));
    TRY(sc.get(&bst, SN));
    TRY(sc.get(&flags, 8));
    TRY(sc.get(&src_d, (size_t)S * 8));
    TRY(sc.get(&nid, S));
    TRY(dalloc(&t->nrow_cnt, SN));
    TRY(dalloc(&t->nrow_node, SN * slots));
    TRY(dalloc(&t->nrow_w, SN * slots));
    TRY(dalloc(&t->cs_nat, SN));
    TRY(dalloc(&t->label, SN));
    TRY(dalloc(&t->level, SN));
    cnt = t->nrow_cnt;
    lab = t->label;
    if (src_f) {
        // point sources: the seed rows are the corners of each source's cell
        int rc = point_sources(g, gin->xyz, s, S, src_f, t->pts, st);
        if (rc) return fail(rc);
        TRY(cudaMemcpyAsync(src_d, t->pts.node, (size_t)S * 8 * sizeof(int), cudaMemcpyDeviceToDevice, st));
    } else {
        std::vector<int> seeds((size_t)S * 8, -1);
        for (int a = 0; a < S; ++a) seeds[(size_t)a * 8] = src_node[a];
        TRY(cudaMemcpyAsync(src_d, seeds.data(), seeds.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        TRY(cudaStreamSynchronize(st));   // the host table goes out of scope
    }
    TRY(cudaMemsetAsync(nid, 0, S * sizeof(unsigned long long), st));

    phase.next("rows");
    // ---- metric, gradient, rows (Sec. 2.2, 3.1, 3.2)
    k_metric<<<blocks_for(N), 256, 0, st>>>(g, gin->xyz, G, nullptr);
    k_grad<<<blocks_for(SN), 256, 0, st>>>(g, S, T, gT);
    k_assemble<<<blocks_for(SN), 256, 0, st>>>(g, S, G, gT, T, s, src_d, cnt, t->nrow_node, t->nrow_w, upmask,
                                               t->cs_nat, nid);
    TRY(cudaGetLastError());

    phase.next("trimming");
    // ---- forward and backward trimming (Sec. 3.5, Prop. 2), frontier by frontier
    TRY(sc.get(&act, SN));        // in-degree counters
    TRY(sc.get(&list, SN));       // two frontier queues
    TRY(sc.get(&color, SN));
    {
        const unsigned gs = (unsigned)std::max(1, t->num_sms * 8);
        int *q[2] = {list, color};
        int *nq = flags;          // flags[0], flags[1]: frontier sizes
        auto rounds = [&](auto step) -> int {
            for (int r = 0;; ++r) {
                const int c = r & 1;
                TRY(cudaMemsetAsync(nq + (c ^ 1), 0, sizeof(int), st));
                step(q[c], nq + c, q[c ^ 1], nq + (c ^ 1), r);
                if ((r & 31) == 31) {
                    int h = 0;
                    TRY(cudaMemcpyAsync(&h, nq + (c ^ 1), sizeof(int), cudaMemcpyDeviceToHost, st));
                    TRY(cudaStreamSynchronize(st));
                    if (h == 0) return EIK_OK;
                }
                if (r > (1 << 28)) { set_error("trimming did not terminate"); return fail(EIK_ERR_CYCLE); }
            }
        };
        TRY(cudaMemsetAsync(flags, 0, 8 * sizeof(int), st));
        k_trim_fwd_init<<<blocks_for(SN), 256, 0, st>>>(SN, upmask, act, fst, q[0], nq);
        TRY(cudaGetLastError());
        int rc = rounds([&](int *cur, int *ncur, int *next, int *nnext, int r) {
            k_trim_fwd_step<<<gs, 256, 0, st>>>(g, upmask, act, fst, cur, ncur, next, nnext, r);
        });
        if (rc) return rc;
        TRY(cudaGetLastError());
        TRY(cudaMemsetAsync(flags, 0, 8 * sizeof(int), st));
        k_trim_bwd_init<<<blocks_for(SN), 256, 0, st>>>(g, SN, upmask, fst, act, bst, q[0], nq);
        TRY(cudaGetLastError());
        rc = rounds([&](int *cur, int *ncur, int *next, int *nnext, int r) {
            k_trim_bwd_step<<<gs, 256, 0, st>>>(g, upmask, fst, act, bst, cur, ncur, next, nnext, r);
        });
        if (rc) return rc;
        TRY(cudaGetLastError());
    }

    phase.next("SCC of the residual");
    // ---- SCCs of the residual (both closures) by Tarjan's algorithm (Sec. 4.1 [ref50]),
    // one host thread per group of sources: the residual is a few percent of the vertices
    {
        unsigned char *rflag;
        TRY(sc.get(&rflag, SN));
        k_residual_flags<<<blocks_for(SN), 256, 0, st>>>(SN, fst, bst, rflag, lab);
        TRY(cudaGetLastError());
        size_t tb = 0;
        thrust::counting_iterator<int> iota(0);
        TRY(cub::DeviceSelect::Flagged(nullptr, tb, iota, rflag, list, flags + 2, (int)SN, st));
        void *tmp;
        TRY(sc.get((unsigned char **)&tmp, tb));
        TRY(cub::DeviceSelect::Flagged(tmp, tb, iota, rflag, list, flags + 2, (int)SN, st));
        int nres = 0;
        TRY(cudaMemcpyAsync(&nres, flags + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        if (nres > 0) {
            unsigned char *dmask;
            TRY(sc.get(&dmask, nres));
            k_gather_masks<<<blocks_for(nres), 256, 0, st>>>(list, nres, upmask, dmask);
            std::vector<int> hnodes(nres), hlab(nres);
            std::vector<unsigned char> hmask(nres);
            TRY(cudaMemcpyAsync(hnodes.data(), list, (size_t)nres * sizeof(int), cudaMemcpyDeviceToHost, st));
            TRY(cudaMemcpyAsync(hmask.data(), dmask, (size_t)nres, cudaMemcpyDeviceToHost, st));
            TRY(cudaStreamSynchronize(st));
            // per source: its residual vertices are one contiguous range of the ascending list
            std::vector<int> rs(S + 1);
            for (int a = 0; a <= S; ++a)
                rs[a] = (int)(std::lower_bound(hnodes.begin(), hnodes.end(), (long long)a * N < INF ? (int)(a * N) : INF) -
                              hnodes.begin());
            rs[S] = nres;
            const int nth = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
            std::vector<std::thread> pool;
            std::atomic<int> next{0};
            for (int w = 0; w < nth; ++w)
                pool.emplace_back([&]() {
                    std::vector<int> where;
                    for (int a; (a = next.fetch_add(1)) < S;)
                        if (rs[a + 1] > rs[a]) {
                            if (where.empty()) where.assign((size_t)N, -1);
                            tarjan_residual(g, hnodes.data() + rs[a], hmask.data() + rs[a], rs[a + 1] - rs[a],
                                            hlab.data() + rs[a], where);
                        }
                });
            for (auto &th : pool) th.join();
            int *dlab;
            TRY(sc.get(&dlab, nres));
            TRY(cudaMemcpyAsync(dlab, hlab.data(), (size_t)nres * sizeof(int), cudaMemcpyHostToDevice, st));
            k_scatter_labels<<<blocks_for(nres), 256, 0, st>>>(list, dlab, nres, lab);
            TRY(cudaGetLastError());
            TRY(cudaStreamSynchronize(st));   // the host vectors go out of scope
        }
    }
    TRY(sc.get(&csize, SN));
    TRY(cudaMemsetAsync(csize, 0, SN * sizeof(int), st));
    k_comp_size<<<blocks_for(SN), 256, 0, st>>>(SN, lab, csize);

    phase.next("levels");
    // ---- canonical levels (longest path on the condensation)
    TRY(sc.get(&lvl, SN));
    TRY(sc.get(&asg, SN));
    TRY(sc.get(&cmax, SN));
    TRY(sc.get(&blk, SN));
    TRY(sc.get(&lmax, S));
    TRY(cudaMemsetAsync(flags, 0, 8 * sizeof(int), st));
    k_lvl_init<<<blocks_for(SN), 256, 0, st>>>(SN, fst, lab, lvl, asg, cmax, blk, list, flags + 1);
    int nlst = 0;
    TRY(cudaMemcpyAsync(&nlst, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    if (nlst > 0) {
        // pend (in blk) and cmax of the components of the level list
        k_lvl_count<<<blocks_for(nlst), 256, 0, st>>>(g, list, nlst, upmask, fst, lab, blk, cmax);
        // members of the nontrivial components of the list, grouped by root
        int *mroot, *members, *mroot_s, *members_s, *moff;
        unsigned char *mflag;
        TRY(sc.get(&mflag, nlst));
        TRY(sc.get(&mroot, nlst));
        k_nontrivial_flags<<<blocks_for(nlst), 256, 0, st>>>(list, nlst, lab, csize, mflag, mroot);
        TRY(cudaGetLastError());
        TRY(sc.get(&members, nlst));
        TRY(sc.get(&members_s, nlst));
        TRY(sc.get(&mroot_s, nlst));
        size_t tb = 0;
        TRY(cub::DeviceSelect::Flagged(nullptr, tb, list, mflag, members, flags + 5, nlst, st));
        void *tmp;
        TRY(sc.get((unsigned char **)&tmp, tb));
        TRY(cub::DeviceSelect::Flagged(tmp, tb, list, mflag, members, flags + 5, nlst, st));
        size_t tb2 = 0;
        TRY(cub::DeviceSelect::Flagged(nullptr, tb2, mroot, mflag, mroot_s, flags + 6, nlst, st));
        void *tmp2;
        TRY(sc.get((unsigned char **)&tmp2, tb2));
        TRY(cub::DeviceSelect::Flagged(tmp2, tb2, mroot, mflag, mroot_s, flags + 6, nlst, st));
        int nmem = 0;
        TRY(cudaMemcpyAsync(&nmem, flags + 5, sizeof(int), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        TRY(sc.get(&moff, SN));
        if (nmem > 0) {
            // group by root: stable sort of (root, node) pairs by root
            size_t tb3 = 0;
            TRY(cub::DeviceRadixSort::SortPairs(nullptr, tb3, mroot_s, mroot, members, members_s, nmem, 0, 32, st));
            void *tmp3;
            TRY(sc.get((unsigned char **)&tmp3, tb3));
            TRY(cub::DeviceRadixSort::SortPairs(tmp3, tb3, mroot_s, mroot, members, members_s, nmem, 0, 32, st));
            k_member_offsets<<<blocks_for(nmem), 256, 0, st>>>(mroot, nmem, moff);
            TRY(cudaGetLastError());
        }
        // frontier rounds
        const unsigned gs = (unsigned)std::max(1, t->num_sms * 8);
        int *q[2] = {color, act};
        int *nq = flags;
        TRY(cudaMemsetAsync(flags, 0, 2 * sizeof(int), st));
        k_lvl_front0<<<blocks_for(nlst), 256, 0, st>>>(list, nlst, lab, blk, q[0], nq);
        TRY(cudaGetLastError());
        for (int r = 0;; ++r) {
            const int c = r & 1;
            TRY(cudaMemsetAsync(nq + (c ^ 1), 0, sizeof(int), st));
            k_lvl_step<<<gs, 256, 0, st>>>(g, upmask, lab, csize, moff, members_s, lvl, asg, cmax, blk, q[c], nq + c,
                                           q[c ^ 1], nq + (c ^ 1), r);
            if ((r & 31) == 31) {
                int h = 0;
                TRY(cudaMemcpyAsync(&h, nq + (c ^ 1), sizeof(int), cudaMemcpyDeviceToHost, st));
                TRY(cudaStreamSynchronize(st));
                if (h == 0) break;
            }
            if (r > (1 << 28)) { set_error("level rounds did not terminate"); return fail(EIK_ERR_CYCLE); }
        }
        TRY(cudaGetLastError());
    }
    // check every component assigned
    TRY(cudaMemsetAsync(flags + 4, 0, sizeof(int), st));
    k_check_assigned<<<blocks_for(SN), 256, 0, st>>>(SN, lab, asg, flags + 4);
    TRY(cudaMemsetAsync(lmax, 0, S * sizeof(int), st));
    k_node_level<<<blocks_for(SN), 256, 0, st>>>(SN, N, lab, lvl, t->level, lmax);
    int unassigned = 0;
    std::vector<int> hlmax(S);
    TRY(cudaMemcpyAsync(&unassigned, flags + 4, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(hlmax.data(), lmax, S * sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    if (unassigned) { set_error("condensation has a cycle (%d components unassigned)", unassigned); return fail(EIK_ERR_CYCLE); }
    t->nlev.resize(S);
    int maxL = 0;
    for (int a = 0; a < S; ++a) { t->nlev[a] = hlmax[a] + 1; maxL = std::max(maxL, t->nlev[a]); }
    t->maxL = maxL;
    int segbits = 1;
    while ((1ll << segbits) < (long long)S * maxL) ++segbits;
    int nb = 1;                  // bits of a local node index
    while ((1ll << nb) < N) ++nb;
    if (2 * nb + segbits > 64) {
        set_error("%lld nodes and %lld (source, level) segments do not fit one 64-bit sort key; build fewer sources "
                  "per tangent", N, (long long)S * maxL);
        return fail(EIK_ERR_INVALID);
    }

    phase.next("canonical order");
    // ---- canonical order: sort by (source, level, component, node)
    unsigned long long *keys, *skeys;
    int *lcount, *head;
    TRY(sc.get(&keys, SN));
    TRY(sc.get(&skeys, SN));
    TRY(sc.get(&lcount, (size_t)S * maxL));
    TRY(sc.get(&head, SN));
    TRY(dalloc(&t->perm, SN));
    TRY(dalloc(&t->pos, SN));
    k_keys<<<blocks_for(SN), 256, 0, st>>>(SN, N, maxL, nb, lab, t->level, keys);
    {
        size_t tb = 0;
        TRY(cub::DeviceRadixSort::SortKeys(nullptr, tb, keys, skeys, (int64_t)SN, 0, 2 * nb + segbits, st));
        void *tmp;
        TRY(sc.get((char **)&tmp, tb));
        TRY(cub::DeviceRadixSort::SortKeys(tmp, tb, keys, skeys, (int64_t)SN, 0, 2 * nb + segbits, st));
    }
    TRY(cudaMemsetAsync(lcount, 0, (size_t)S * maxL * sizeof(int), st));
    k_perm<<<blocks_for(SN), 256, 0, st>>>(SN, N, maxL, nb, skeys, lab, csize, t->perm, t->pos, lcount, head);
    TRY(cudaGetLastError());
    std::vector<int> hl((size_t)S * maxL);
    TRY(cudaMemcpyAsync(hl.data(), lcount, hl.size() * sizeof(int), cudaMemcpyDeviceToHost, st));

    phase.next("canonical rows");
    // ---- rows in canonical order (gather form) and transposed rows
    int *fcnt, *tcnt;
    long long *fscan, *tscan;
    TRY(sc.get(&fcnt, SN));
    TRY(sc.get(&tcnt, SN));
    TRY(sc.get(&fscan, SN + 1));
    TRY(sc.get(&tscan, SN + 1));
    k_counts<<<blocks_for(SN), 256, 0, st>>>(g, SN, t->perm, lab, cnt, t->nrow_node, upmask, fcnt, tcnt);
    {
        size_t tb = 0, tb2 = 0;
        TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, fcnt, fscan, (int64_t)SN + 1, st));
        TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb2, tcnt, tscan, (int64_t)SN + 1, st));
        tb = std::max(tb, tb2);
        void *tmp;
        TRY(sc.get((char **)&tmp, tb));
        // counts arrays are SN long; the (SN+1)-th input must be 0: use SN items, total appended below
        TRY(cub::DeviceScan::ExclusiveSum(tmp, tb, fcnt, fscan, (int64_t)SN, st));
        TRY(cub::DeviceScan::ExclusiveSum(tmp, tb, tcnt, tscan, (int64_t)SN, st));
    }
    // per-source bases (host)
    std::vector<long long> hf(S + 1), ht(S + 1);
    {
        for (int a = 0; a < S; ++a) {
            TRY(cudaMemcpyAsync(&hf[a], fscan + (long long)a * N, sizeof(long long), cudaMemcpyDeviceToHost, st));
            TRY(cudaMemcpyAsync(&ht[a], tscan + (long long)a * N, sizeof(long long), cudaMemcpyDeviceToHost, st));
        }
        long long lf = 0, lt = 0;
        int cf = 0, ct = 0;
        TRY(cudaMemcpyAsync(&lf, fscan + SN - 1, sizeof(long long), cudaMemcpyDeviceToHost, st));
        TRY(cudaMemcpyAsync(&lt, tscan + SN - 1, sizeof(long long), cudaMemcpyDeviceToHost, st));
        TRY(cudaMemcpyAsync(&cf, fcnt + SN - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        TRY(cudaMemcpyAsync(&ct, tcnt + SN - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        hf[S] = lf + cf;
        ht[S] = lt + ct;
    }
    for (int a = 0; a < S; ++a)
        if (hf[a + 1] - hf[a] >= (1ll << 31) || ht[a + 1] - ht[a] >= (1ll << 31)) {
            set_error("too many edges per source"); return fail(EIK_ERR_INVALID);
        }
    t->ebase = hf;
    t->tbase = ht;
    TRY(dalloc(&t->ebase_d, S + 1));
    TRY(dalloc(&t->tbase_d, S + 1));
    long long *fbase_d = t->ebase_d, *tbase_d = t->tbase_d;
    TRY(cudaMemcpyAsync(fbase_d, hf.data(), (S + 1) * sizeof(long long), cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(tbase_d, ht.data(), (S + 1) * sizeof(long long), cudaMemcpyHostToDevice, st));
    TRY(dalloc(&t->rowptr, (size_t)S * (N + 1)));
    TRY(dalloc(&t->cptr, (size_t)S * (N + 1)));
    TRY(dalloc(&t->up_node, hf[S]));
    TRY(dalloc(&t->up_w32, hf[S]));
    TRY(dalloc(&t->up_w64, hf[S]));
    TRY(dalloc(&t->dn_node, ht[S]));
    TRY(dalloc(&t->dn_w32, ht[S]));
    TRY(dalloc(&t->dn_w64, ht[S]));
    k_fill<<<blocks_for(SN), 256, 0, st>>>(g, SN, t->perm, t->pos, lab, cnt, t->nrow_node, t->nrow_w, upmask, fscan, tscan,
                                           fbase_d, tbase_d, t->rowptr, t->cptr, t->up_node, t->up_w32, t->up_w64,
                                           t->dn_node, t->dn_w32, t->dn_w64);
    TRY(cudaGetLastError());

    phase.next("coefficients");
    // ---- C*M coefficients, receivers
    TRY(dalloc(&t->cq64, SN));
    TRY(dalloc(&t->cq32, SN));
    TRY(dalloc(&t->cqn64, SN));
    TRY(dalloc(&t->cqn32, SN));
    k_cq<<<blocks_for(SN), 256, 0, st>>>(SN, N, t->model, t->perm, t->cs_nat, s, t->cq64, t->cq32, t->cqn64, t->cqn32);
    int *recpos;
    TRY(sc.get(&recpos, SN));
    TRY(cudaMemsetAsync(recpos, 0xff, SN * sizeof(int), st));
    TRY(dalloc(&t->rec_slot, SN));
    TRY(dalloc(&t->rec_nat, (size_t)S * std::max(n_rec, 1)));
    if (n_rec > 0) {
        TRY(cudaMemcpyAsync(t->rec_nat, rec_node, (size_t)S * n_rec * sizeof(int), cudaMemcpyHostToDevice, st));
        TRY(cudaMemsetAsync(flags + 5, 0, sizeof(int), st));
        k_rec_mark<<<blocks_for((long long)S * n_rec), 256, 0, st>>>(S, N, n_rec, t->rec_nat, recpos, flags + 5);
        int bad = 0;
        TRY(cudaMemcpyAsync(&bad, flags + 5, sizeof(int), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        if (bad) {
            set_error(bad == 1 ? "receiver node out of range" : "duplicate receiver node within a source");
            return fail(EIK_ERR_INVALID);
        }
    }
    k_rec_slot<<<blocks_for(SN), 256, 0, st>>>(SN, N, t->perm, recpos, t->rec_slot);

    phase.next("blocks");
    // ---- level pointers (host) and blocks
    t->level_ptr.assign((size_t)S * (maxL + 1), 0);
    for (int a = 0; a < S; ++a) {
        long long acc = 0;
        for (int L = 0; L <= maxL; ++L) {
            t->level_ptr[(size_t)a * (maxL + 1) + L] = acc;
            if (L < maxL) acc += hl[(size_t)a * maxL + L];
        }
    }
    {
        int *hpos, *hscan;
        TRY(sc.get(&hpos, SN));
        TRY(sc.get(&hscan, SN));
        size_t tb = 0;
        TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, head, hscan, (int64_t)SN, st));
        void *tmp;
        TRY(sc.get((char **)&tmp, tb));
        TRY(cub::DeviceScan::ExclusiveSum(tmp, tb, head, hscan, (int64_t)SN, st));
        k_compact_heads<<<blocks_for(SN), 256, 0, st>>>(SN, head, hscan, hpos);
        int nb = 0, lastflag = 0;
        TRY(cudaMemcpyAsync(&nb, hscan + SN - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        TRY(cudaMemcpyAsync(&lastflag, head + SN - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        nb += lastflag;
        int4 *binfo;
        TRY(sc.get(&binfo, std::max(nb, 1)));
        if (nb > 0) k_block_info<<<blocks_for(nb), 256, 0, st>>>(nb, N, hpos, t->perm, lab, t->level, csize, binfo);
        std::vector<int4> hb(std::max(nb, 1));
        TRY(cudaMemcpyAsync(hb.data(), binfo, std::max(nb, 1) * sizeof(int4), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        t->nblk = nb;
        long long lo = 0, po = 0, wo = 0;
        std::vector<int4> hd(std::max(nb, 1));
        std::vector<long long> ho(3 * std::max(nb, 1));
        for (int b = 0; b < nb; ++b) {
            Block B;
            B.src = hb[b].x;
            B.p0 = hb[b].y;
            B.k = hb[b].z;
            B.level = hb[b].w;
            B.lu = lo; B.piv = po; B.ws = wo;
            lo += (long long)B.k * B.k; po += B.k; wo += B.k;
            t->blocks.push_back(B);
            hd[b] = make_int4(B.src, B.p0, B.k, B.level);
            ho[3 * b] = B.lu; ho[3 * b + 1] = B.piv; ho[3 * b + 2] = B.ws;
        }
        t->lu_words = lo; t->piv_words = po; t->ws_rows = wo;
        TRY(dalloc(&t->blk_desc, std::max(nb, 1)));
        TRY(dalloc(&t->blk_off, 3 * std::max(nb, 1)));
        TRY(dalloc(&t->lu, std::max(lo, 1ll)));
        TRY(dalloc(&t->binv, std::max(lo, 1ll)));
        TRY(dalloc(&t->piv, std::max(po, 1ll)));
        TRY(dalloc(&t->err, 4));
        TRY(cudaMemsetAsync(t->err, 0, 4 * sizeof(int), st));
        if (nb > 0) {
            TRY(cudaMemcpyAsync(t->blk_desc, hd.data(), nb * sizeof(int4), cudaMemcpyHostToDevice, st));
            TRY(cudaMemcpyAsync(t->blk_off, ho.data(), 3 * nb * sizeof(long long), cudaMemcpyHostToDevice, st));
            k_block_fill<<<nb, 256, 0, st>>>(g, t->blk_desc, t->blk_off, t->perm, t->pos, lab, cnt, t->nrow_node,
                                             t->nrow_w, t->lu);
            k_block_lu<<<nb, 256, 0, st>>>(t->blk_desc, t->blk_off, t->lu, t->piv, opts->lu_pivot_tol, t->err);
            k_block_inverse<<<nb, 128, 0, st>>>(t->blk_desc, t->blk_off, t->lu, t->piv, t->binv);
            TRY(cudaGetLastError());
            int e = 0;
            TRY(cudaMemcpyAsync(&e, t->err, sizeof(int), cudaMemcpyDeviceToHost, st));
            TRY(cudaStreamSynchronize(st));
            if (e == DEV_SINGULAR) { set_error("an SCC block is singular (pivot below %g)", opts->lu_pivot_tol); return fail(EIK_ERR_SINGULAR_BLOCK); }
        }
    }

    phase.next("items");
    // ---- traversal work items: level-major over sources
    {
        int chunk = opts->chunk > 0 ? std::min(opts->chunk, ITEM_CAP) : ITEM_MAX;
        t->item_max = chunk;
        std::vector<std::vector<int4>> per((size_t)S * maxL);
        std::vector<int> blk_ptr(S + 1, 0);
        // blocks are ordered by (source, position), hence by (source, level)
        size_t bi = 0;
        for (int a = 0; a < S; ++a) {
            for (int L = 0; L < t->nlev[a]; ++L) {
                long long p0 = t->level_ptr[(size_t)a * (maxL + 1) + L], p1 = t->level_ptr[(size_t)a * (maxL + 1) + L + 1];
                auto &vec = per[(size_t)a * maxL + L];
                for (long long p = p0; p < p1; p += chunk)
                    vec.push_back(make_int4(a, L, (int)p, (int)std::min(p1, p + chunk)));
                while (bi < t->blocks.size() && t->blocks[bi].src == a && t->blocks[bi].level == L) {
                    vec.push_back(make_int4(a, L, ~(int)bi, 0));
                    ++bi;
                }
            }
        }
        std::vector<int4> fw, bw;
        std::vector<int> icnt(2 * (size_t)S * maxL, 0);
        t->step_ptr_fwd.assign(maxL + 1, 0);
        t->step_ptr_bwd.assign(maxL + 1, 0);
        for (int stp = 0; stp < maxL; ++stp) {
            t->step_ptr_fwd[stp] = (int)fw.size();
            t->step_ptr_bwd[stp] = (int)bw.size();
            for (int a = 0; a < S; ++a) {
                if (stp >= t->nlev[a]) continue;
                for (int4 it : per[(size_t)a * maxL + stp]) { it.y = stp; fw.push_back(it); }
                icnt[(size_t)a * maxL + stp] = (int)per[(size_t)a * maxL + stp].size();
                int L = t->nlev[a] - 1 - stp;
                for (int4 it : per[(size_t)a * maxL + L]) { it.y = stp; bw.push_back(it); }
                icnt[(size_t)S * maxL + (size_t)a * maxL + stp] = (int)per[(size_t)a * maxL + L].size();
            }
        }
        t->step_ptr_fwd[maxL] = (int)fw.size();
        t->step_ptr_bwd[maxL] = (int)bw.size();
        t->nitems = (int)fw.size();
        TRY(dalloc(&t->items_fwd, fw.size()));
        TRY(dalloc(&t->items_bwd, bw.size()));
        TRY(dalloc(&t->item_cnt, icnt.size()));
        TRY(dalloc(&t->done, icnt.size()));
        TRY(dalloc(&t->ticket, 4));
        TRY(cudaMemcpyAsync(t->items_fwd, fw.data(), fw.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
        TRY(cudaMemcpyAsync(t->items_bwd, bw.data(), bw.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
        TRY(cudaMemcpyAsync(t->item_cnt, icnt.data(), icnt.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        TRY(dalloc(&t->ebeg_fwd, fw.size()));
        TRY(dalloc(&t->ebeg_bwd, bw.size()));
        k_item_edges<<<blocks_for((long long)fw.size()), 256, 0, st>>>((int)fw.size(), N, t->items_fwd, t->rowptr, t->ebeg_fwd);
        k_item_edges<<<blocks_for((long long)bw.size()), 256, 0, st>>>((int)bw.size(), N, t->items_bwd, t->cptr, t->ebeg_bwd);
        TRY(cudaGetLastError());
        // per-item dependencies of both directions
        int *iop;
        TRY(sc.get(&iop, SN));
        const int ni = (int)fw.size();
        TRY(dalloc(&t->deps_fwd, (size_t)ni * DEP_MAX));
        TRY(dalloc(&t->deps_bwd, (size_t)ni * DEP_MAX));
        TRY(dalloc(&t->ndeps_fwd, ni));
        TRY(dalloc(&t->ndeps_bwd, ni));
        TRY(dalloc(&t->item_done, ni));
        k_item_of_pos<<<blocks_for(ni), 256, 0, st>>>(ni, N, t->items_fwd, t->blk_desc, t->perm, iop);
        k_item_deps<<<blocks_for(ni), 256, 0, st>>>(ni, N, t->items_fwd, t->blk_desc, t->perm, t->rowptr, t->up_node,
                                                    t->ebase_d, iop, t->deps_fwd, t->ndeps_fwd);
        k_item_of_pos<<<blocks_for(ni), 256, 0, st>>>(ni, N, t->items_bwd, t->blk_desc, t->perm, iop);
        k_item_deps<<<blocks_for(ni), 256, 0, st>>>(ni, N, t->items_bwd, t->blk_desc, t->perm, t->cptr, t->dn_node,
                                                    t->tbase_d, iop, t->deps_bwd, t->ndeps_bwd);
        TRY(cudaGetLastError());
        // cluster schedule tables
        std::vector<int> hl_pos((size_t)S * (maxL + 1), 0), hb_lvl((size_t)S * (maxL + 1), 0), hn(S), ord(S);
        size_t bj = 0;
        for (int a = 0; a < S; ++a) {
            hn[a] = t->nlev[a];
            for (int L = 0; L <= maxL; ++L) {
                const int Lc = std::min(L, t->nlev[a]);
                hl_pos[(size_t)a * (maxL + 1) + L] = (int)t->level_ptr[(size_t)a * (maxL + 1) + Lc];
                while (bj < t->blocks.size() && (t->blocks[bj].src < a || (t->blocks[bj].src == a && t->blocks[bj].level < L)))
                    ++bj;
                hb_lvl[(size_t)a * (maxL + 1) + L] = (int)bj;
            }
        }
        for (int a = 0; a < S; ++a) ord[a] = a;
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return t->nlev[x] > t->nlev[y]; });
        TRY(dalloc(&t->lvl_d, hl_pos.size()));
        TRY(dalloc(&t->blk_lvl_d, hb_lvl.size()));
        TRY(dalloc(&t->nlev_d, S));
        TRY(dalloc(&t->order_d, S));
        TRY(cudaMemcpyAsync(t->lvl_d, hl_pos.data(), hl_pos.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        TRY(cudaMemcpyAsync(t->blk_lvl_d, hb_lvl.data(), hb_lvl.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        TRY(cudaMemcpyAsync(t->nlev_d, hn.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
        TRY(cudaMemcpyAsync(t->order_d, ord.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
        TRY(cudaStreamSynchronize(st));   // the host vectors above go out of scope
    }

    phase.next("statistics");
    // ---- statistics
    {
        std::vector<unsigned long long> hid(S);
        TRY(cudaMemcpyAsync(hid.data(), nid, S * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        unsigned long long *nroots;
        TRY(sc.get(&nroots, S));
        TRY(cudaMemsetAsync(nroots, 0, S * sizeof(unsigned long long), st));
        k_count_roots<<<blocks_for(SN), 256, 0, st>>>(SN, N, lab, nroots);
        std::vector<unsigned long long> hr(S);
        TRY(cudaMemcpyAsync(hr.data(), nroots, S * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        t->stats.assign(S, eik_stats{});
        for (int a = 0; a < S; ++a) {
            eik_stats &x = t->stats[a];
            x.nodes = N;
            x.components = (int64_t)hr[a];
            x.levels = t->nlev[a];
            long long w = 0;
            for (int L = 0; L < t->nlev[a]; ++L) w = std::max(w, (long long)hl[(size_t)a * maxL + L]);
            x.max_level_width = w;
            x.identity_rows = (int64_t)hid[a];
        }
        for (const Block &B : t->blocks) {
            eik_stats &x = t->stats[B.src];
            x.nontrivial += 1;
            x.cyclic_nodes += B.k;
            x.largest = std::max<int64_t>(x.largest, B.k);
            x.lu_doubles += (int64_t)B.k * B.k;
        }
        // edges: full rows (natural)
        unsigned long long *ne;
        TRY(sc.get(&ne, S));
        TRY(cudaMemsetAsync(ne, 0, S * sizeof(unsigned long long), st));
        k_count_edges<<<blocks_for(SN), 256, 0, st>>>(SN, N, cnt, ne);
        std::vector<unsigned long long> hne(S);
        TRY(cudaMemcpyAsync(hne.data(), ne, S * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        for (int a = 0; a < S; ++a) t->stats[a].edges = (int64_t)hne[a];
    }
    // convert labels to local ids for export
    k_local_labels<<<blocks_for(SN), 256, 0, st>>>(SN, N, lab);
    TRY(cudaGetLastError());
    TRY(cudaStreamSynchronize(st));
#undef TRY
    if (opts->split_dirs) {
        int rc = enable_split(t);
        if (rc) return fail(rc);
    }
    if (src_f) {
        // point sources: model factors at the corners and z = A^-1 e (a traversal of the
        // finished tangent)
        int rc = point_tangent_setup(t, s, st);
        if (rc) return fail(rc);
    }
    *out = t;
    return EIK_OK;
}

}  // namespace eik
