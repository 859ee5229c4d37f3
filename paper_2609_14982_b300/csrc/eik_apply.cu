// Phase III of Algorithm 1: the stored block traversals B_a (forward, A^-1) and B_a^T
// (reverse, A^-T) for all sources and right-hand sides (Prop. 3, Sec. 4.3-4.4).
//
// Data layout (right-hand-side index fastest):
//   the caller's vectors are [S][N][R] (or [N][R]) in natural node order; the
//   transported field itself (dT or lam) lives in a workspace [S][N][R] in each source's
//   canonical level order, and rows reference upstream nodes by canonical position.  A
//   level's results are then one contiguous run of rows, and its gathers read the
//   contiguous, recently written rows of earlier levels.  The structure (rows, weights,
//   C*M, receiver slots) is in the same order, so one level is a contiguous slice of
//   every array.  A natural-order copy of the field is written only when requested.
// Work: a work item is (source, step, position range) of singleton components of one
//   level, or one nontrivial SCC block.  Items are ordered step-major across sources.
//   Persistent schedule: CTAs take items by ticket; an item waits (bounded) only for
//   the items that hold its upstream positions (recorded at build time; an item with
//   too many waits for every item of its source's previous step instead).  Every such
//   item has a lower ticket, and tickets are handed out in order, so every item waited
//   on is held by a running CTA or done: no deadlock.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "eik_internal.h"

namespace eik {

// ------------------------------------------------------------------ small helpers
template <typename T, int V> struct VecT;
template <> struct VecT<float, 1> { using type = float; };
template <> struct VecT<float, 2> { using type = float2; };
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<double, 1> { using type = double; };
template <> struct VecT<double, 2> { using type = double2; };

template <typename T, int V> struct Pack { T v[V]; };

template <typename T, int V>
__device__ __forceinline__ Pack<T, V> load_ro(const T *p)
{
    using VT = typename VecT<T, V>::type;
    VT x = __ldg(reinterpret_cast<const VT *>(p));
    Pack<T, V> r;
    memcpy(&r, &x, sizeof(VT));
    return r;
}

// loads of values produced earlier in the same launch go through L2 only (L1 is not
// coherent with other SMs' writes)
template <typename T, int V>
__device__ __forceinline__ Pack<T, V> load_l2(const T *p)
{
    using VT = typename VecT<T, V>::type;
    VT x = __ldcg(reinterpret_cast<const VT *>(p));
    Pack<T, V> r;
    memcpy(&r, &x, sizeof(VT));
    return r;
}

template <typename T, int V>
__device__ __forceinline__ void store(T *p, const Pack<T, V> &v)
{
    using VT = typename VecT<T, V>::type;
    VT x;
    memcpy(&x, &v, sizeof(VT));
    *reinterpret_cast<VT *>(p) = x;
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct TravParams {
    int S, R, n_rec, maxL, nitems;   // R: right-hand sides of this launch (a column chunk)
    int item_max;                    // positions per singleton item
    long long ld_in, ld_x, ld_aux;   // row strides (elements) of in, x and aux
    long long N;
    int mode;          // MODE_J or MODE_RAW
    int shared_in;     // forward MODE_J: p is [N][R]
    int sum;           // transpose MODE_J: g is summed over sources (written by a later kernel)
    const int *perm;
    const int *rowptr;     // forward: rowptr, transpose: cptr
    const int *enode;
    const void *ew;        // float* or double* weights (matching T)
    const double *ew64;    // FP64 weights (block right-hand sides)
    const long long *ebase;
    const void *cq;        // C*M per position (T)
    const double *cq64;
    const int *rec_slot;
    const void *in;        // forward: p / q ; transpose: y / r
    void *x;               // dT or lam workspace [S][N][R], canonical order
    void *out;             // optional natural-order copy of x [S][N][R]
    long long ld_out;
    void *aux;             // forward: d_rec [S][n_rec][R]; transpose (no sum): g [S][N][R]
    const int4 *items;
    const int2 *ebeg;      // per item: staged edge range
    const int *item_cnt;   // [S][maxL] items per (source, step) of this direction
    int *done;             // [S][maxL]
    const int *deps;       // [nitems][DEP_MAX] items holding this item's upstream positions
    const int *ndeps;      // [nitems], -1: too many, wait for the whole previous step
    int *item_done;        // [nitems]
    int *ticket;
    int *err;              // {code, source, step, item}
    const int4 *blk_desc;
    const long long *blk_off;
    const double *binv;    // block inverses
    double *ws;
    unsigned long long timeout_ns;
};

// ---------------------------------------------------------------- singleton items
// The structure of one item (at most ITEM_MAX positions of one level of one source and
// their rows) is staged into shared memory by all threads in one round of independent
// loads; afterwards a node costs only its own vector loads (input, upstream values),
// all issued before they are summed.
constexpr int MAX_ROW = 6;   // at most 2 * ndim faces per row

template <typename T> struct Stage {
    int perm[ITEM_MAX];
    int rec[ITEM_MAX];
    int rp[ITEM_MAX + 1];
    T cq[ITEM_MAX];
    int en[MAX_ROW * ITEM_MAX];
    T ew[MAX_ROW * ITEM_MAX];
};

template <typename T>
__device__ __forceinline__ void stage_item(const TravParams &P, Stage<T> &sm, int a, int p0, int p1, int2 eb)
{
    const long long N = P.N;
    const int np = p1 - p0, ne = eb.y - eb.x;
    const int *perm = P.perm + a * N + p0;
    const int *rp = P.rowptr + a * (N + 1) + p0;
    const T *cq = reinterpret_cast<const T *>(P.cq) + a * N + p0;
    const int *rs = P.rec_slot + a * N + p0;
    const long long eb0 = P.ebase[a] + eb.x;
    const int *en = P.enode + eb0;
    const T *ew = reinterpret_cast<const T *>(P.ew) + eb0;
    for (int k = threadIdx.x; k <= np; k += blockDim.x) {
        sm.rp[k] = __ldg(rp + k) - eb.x;
        if (k < np) {
            sm.perm[k] = __ldg(perm + k);
            sm.rec[k] = __ldg(rs + k);
            sm.cq[k] = __ldg(cq + k);
        }
    }
    for (int k = threadIdx.x; k < ne; k += blockDim.x) {
        sm.en[k] = __ldg(en + k);
        sm.ew[k] = __ldg(ew + k);
    }
}

// Each group of G lanes owns up to NPS (1 or 2) nodes of the item (slot, slot + nslot);
// lane l handles right-hand sides l*V .. l*V+V-1, then strides by G*V.  All loads of
// the group's nodes (input and up to MAX_ROW upstream values each) are issued before
// any sum.
template <typename T, int V, bool TR>
__device__ __forceinline__ Pack<T, V> node_input(const TravParams &P, int a, int v, int rec, T c, int r)
{
    const long long N = P.N;
    const T *in = reinterpret_cast<const T *>(P.in);
    Pack<T, V> acc;
    if (!TR) {
        if (P.mode == MODE_J) {
            Pack<T, V> q = load_ro<T, V>(in + ((P.shared_in ? 0 : (long long)a * N) + v) * P.ld_in + r);
#pragma unroll
            for (int u = 0; u < V; ++u) acc.v[u] = c * q.v[u];
        } else {
            acc = load_ro<T, V>(in + ((long long)a * N + v) * P.ld_in + r);
        }
    } else {
        if (P.mode == MODE_J) {
            if (rec >= 0) acc = load_ro<T, V>(in + ((long long)a * P.n_rec + rec) * P.ld_in + r);
            else {
#pragma unroll
                for (int u = 0; u < V; ++u) acc.v[u] = T(0);
            }
        } else {
            acc = load_ro<T, V>(in + ((long long)a * N + v) * P.ld_in + r);
        }
    }
    return acc;
}

template <typename T, int V, bool TR>
__device__ __forceinline__ void node_output(const TravParams &P, int a, int v, int pos, int rec, T c, int r, T *x,
                                            const Pack<T, V> &acc)
{
    const long long N = P.N;
    T *aux = reinterpret_cast<T *>(P.aux);
    store<T, V>(x + (long long)pos * P.ld_x + r, acc);
    if (P.out) store<T, V>(reinterpret_cast<T *>(P.out) + ((long long)a * N + v) * P.ld_out + r, acc);
    if (P.mode == MODE_J && aux) {
        if (!TR) {
            if (rec >= 0) store<T, V>(aux + ((long long)a * P.n_rec + rec) * P.ld_aux + r, acc);
        } else if (!P.sum) {
            Pack<T, V> gv;
#pragma unroll
            for (int u = 0; u < V; ++u) gv.v[u] = c * acc.v[u];
            store<T, V>(aux + ((long long)a * N + v) * P.ld_aux + r, gv);
        }
    }
}

template <typename T, int V, bool TR, int NPS>
__device__ __forceinline__ void run_singletons(const TravParams &P, const Stage<T> &sm, int a, int p0, int np, int G)
{
    const int lane = threadIdx.x % G, slot = threadIdx.x / G, nslot = blockDim.x / G;
    const long long N = P.N;
    const int R = P.R;
    T *x = reinterpret_cast<T *>(P.x) + a * N * P.ld_x;
    for (int k0 = slot; k0 < np; k0 += NPS * nslot) {
        const int k1 = k0 + nslot;
        const bool has1 = NPS == 2 && k1 < np;
        const int v0 = sm.perm[k0], v1 = has1 ? sm.perm[k1] : -1;
        const bool on0 = v0 >= 0, on1 = v1 >= 0;  // members of nontrivial blocks are skipped
        const int e00 = sm.rp[k0], c0 = on0 ? sm.rp[k0 + 1] - e00 : 0;
        const int e01 = has1 ? sm.rp[k1] : 0, c1 = on1 ? sm.rp[k1 + 1] - e01 : 0;
        const int rec0 = sm.rec[k0], rec1 = has1 ? sm.rec[k1] : -1;
        const T cq0 = sm.cq[k0], cq1 = has1 ? sm.cq[k1] : T(0);
        for (int r = lane * V; r < R; r += G * V) {
            Pack<T, V> a0, a1, x0[MAX_ROW], x1[MAX_ROW];
            if (on0) a0 = node_input<T, V, TR>(P, a, v0, rec0, cq0, r);
            if (on1) a1 = node_input<T, V, TR>(P, a, v1, rec1, cq1, r);
#pragma unroll
            for (int e = 0; e < MAX_ROW; ++e) {
                if (e < c0) x0[e] = load_l2<T, V>(x + (long long)sm.en[e00 + e] * P.ld_x + r);
                if (e < c1) x1[e] = load_l2<T, V>(x + (long long)sm.en[e01 + e] * P.ld_x + r);
            }
#pragma unroll
            for (int e = 0; e < MAX_ROW; ++e) {
                if (e < c0) {
                    const T w = sm.ew[e00 + e];
#pragma unroll
                    for (int u = 0; u < V; ++u) a0.v[u] += w * x0[e].v[u];
                }
                if (e < c1) {
                    const T w = sm.ew[e01 + e];
#pragma unroll
                    for (int u = 0; u < V; ++u) a1.v[u] += w * x1[e].v[u];
                }
            }
            if (on0) node_output<T, V, TR>(P, a, v0, p0 + k0, rec0, cq0, r, x, a0);
            if (on1) node_output<T, V, TR>(P, a, v1, p0 + k1, rec1, cq1, r, x, a1);
        }
    }
}

// ---------------------------------------------------------------- block items
// FP64 solve of one nontrivial SCC block for all right-hand sides (Sec. 4.3).  The
// right-hand side gathers the block's external rows: forward b = q_C + W_ext x_ext,
// transpose b = r_C + W_ext^T lam_ext.  The solve multiplies by A_C^-1, formed once at
// build time from the partial-pivot factors P A_C = L U (the transpose reads the same
// matrix transposed, A_C^-T = (A_C^-1)^T), so each (row, right-hand side) is one
// independent dot product instead of a k-step triangular sweep.
struct CtaSync { __device__ void operator()() const { __syncthreads(); } };

// the solve runs on threads tid = 0 .. nthr-1 of the CTA, which sync() synchronises
template <typename T, bool TR, typename Sync = CtaSync>
__device__ void run_block(const TravParams &P, int a, int b, int tid = threadIdx.x, int nthr = blockDim.x,
                          Sync sync = Sync())
{
    const int4 d = P.blk_desc[b];
    const int p0 = d.y, k = d.z;
    const long long luo = P.blk_off[3 * b], wso = P.blk_off[3 * b + 2];
    const int R = P.R;
    const long long N = P.N;
    const int *perm = P.perm + a * N;
    const int *rp = P.rowptr + a * (N + 1);
    const long long eb = P.ebase[a];
    const int *en = P.enode + eb;
    const double *ew = P.ew64 + eb;
    const T *in = reinterpret_cast<const T *>(P.in);
    T *x = reinterpret_cast<T *>(P.x) + a * N * P.ld_x;
    T *aux = reinterpret_cast<T *>(P.aux);
    double *W = P.ws + wso * R;
    const double *Ainv = P.binv + luo;
    for (long long idx = tid; idx < (long long)k * R; idx += nthr) {
        const int m = (int)(idx / R), r = (int)(idx % R);
        const int p = p0 + m;
        const int v = ~__ldg(perm + p);
        double acc;
        const int rec = P.rec_slot[a * N + p];
        if (!TR) {
            if (P.mode == MODE_J)
                acc = P.cq64[a * N + p] * (double)in[((P.shared_in ? 0 : (long long)a * N) + v) * P.ld_in + r];
            else
                acc = (double)in[((long long)a * N + v) * P.ld_in + r];
        } else {
            if (P.mode == MODE_J) acc = rec >= 0 ? (double)in[((long long)a * P.n_rec + rec) * P.ld_in + r] : 0.0;
            else acc = (double)in[((long long)a * N + v) * P.ld_in + r];
        }
        for (int e = rp[p]; e < rp[p + 1]; ++e) acc += ew[e] * (double)__ldcg(x + (long long)en[e] * P.ld_x + r);
        W[(long long)m * R + r] = acc;
    }
    sync();
    for (long long idx = tid; idx < (long long)k * R; idx += nthr) {
        const int m = (int)(idx / R), r = (int)(idx % R);
        double val = 0.0;
        if (!TR) {
            const double *row = Ainv + (long long)m * k;
            for (int c = 0; c < k; ++c) val += row[c] * W[(long long)c * R + r];
        } else {
            for (int c = 0; c < k; ++c) val += Ainv[(long long)c * k + m] * W[(long long)c * R + r];
        }
        const int p = p0 + m;
        const int v = ~perm[p];
        x[(long long)p * P.ld_x + r] = (T)val;
        if (P.out) reinterpret_cast<T *>(P.out)[((long long)a * N + v) * P.ld_out + r] = (T)val;
        if (P.mode == MODE_J && aux) {
            const int rec = P.rec_slot[a * N + p];
            if (!TR) {
                if (rec >= 0) aux[((long long)a * P.n_rec + rec) * P.ld_aux + r] = (T)val;
            } else if (!P.sum) {
                aux[((long long)a * N + v) * P.ld_aux + r] = (T)(P.cq64[a * N + p] * val);
            }
        }
    }
}

template <typename T, int V, bool TR>
__device__ __forceinline__ void run_item(const TravParams &P, Stage<T> &sm, int4 it, int2 eb, int G)
{
    if (it.z >= 0) {
        stage_item<T>(P, sm, it.x, it.z, it.w, eb);
        __syncthreads();
        run_singletons<T, V, TR, 2>(P, sm, it.x, it.z, it.w - it.z, G);
    } else {
        run_block<T, TR>(P, it.x, ~it.z);
    }
}

__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------- per-level schedule
// One launch per step: every CTA runs one item, with no ticket, wait or counter.  The
// launches are chained with programmatic dependent launch: a CTA stages its item's
// structure (never written by the traversal) before griddepcontrol.wait, so staging
// overlaps the tail of the previous level; after the wait every value of earlier levels
// is complete and visible.  Parameters are read from device memory, so a captured
// sequence of these launches does not depend on the caller's buffers.
template <typename T, int V, bool TR, int NPS>
__global__ void __launch_bounds__(256, 4) k_traverse_level(const TravParams *__restrict__ Pd, int G, int first)
{
    __shared__ Stage<T> sm;
    const TravParams &P = *Pd;
    const int i = first + blockIdx.x;
    const int4 it = P.items[i];
    grid_dependents_launch();
    if (it.z >= 0) {
        stage_item<T>(P, sm, it.x, it.z, it.w, P.ebeg[i]);
        grid_dependency_wait();
        __syncthreads();
        run_singletons<T, V, TR, NPS>(P, sm, it.x, it.z, it.w - it.z, G);
    } else {
        grid_dependency_wait();
        run_block<T, TR>(P, it.x, ~it.z);
    }
}

__global__ void k_set_params(TravParams *Pd, TravParams P) { *Pd = P; }

// ---------------------------------------------------------------- staged (async-copy) schedule
// One launch per step; each CTA walks the step's items with two pipeline stages.  A CTA
// has item_max x G threads: thread (k, lane) owns position k of the item and the lane's
// 16-byte column chunk.  For an item it copies, with cp.async, its chunk of the
// position's input row and of every upstream row into shared memory; it later reads
// back only what it copied itself, so the copies need no barrier, hold no registers
// while in flight, and two items per CTA are in flight at once.  While one item
// computes, the next item's structure is staged and its copies are issued.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

struct StagedMeta {
    int a, kind, np, ne, block, p0;   // source; 1 singleton range / 0 block; positions; edges; block; first position
};

template <typename T>
__device__ __forceinline__ void staged_structure(const TravParams &P, Stage<T> &sm, StagedMeta &meta, int i)
{
    const int4 it = P.items[i];
    if (it.z < 0) {
        if (threadIdx.x == 0) { meta.a = it.x; meta.kind = 0; meta.np = 0; meta.ne = 0; meta.block = ~it.z; }
        return;
    }
    const int2 eb = P.ebeg[i];
    stage_item<T>(P, sm, it.x, it.z, it.w, eb);
    if (threadIdx.x == 0) { meta.a = it.x; meta.kind = 1; meta.np = it.w - it.z; meta.ne = eb.y - eb.x; meta.block = -1; meta.p0 = it.z; }
}

// rows of a stage, each ROWB bytes: position k's input row at k, edge e's upstream row
// at item_max + e; this thread copies its 16-byte chunks (column r) of its own position
template <typename T, bool TR>
__device__ __forceinline__ void staged_issue(const TravParams &P, const Stage<T> &sm, const StagedMeta &meta,
                                             unsigned char *rows, int G)
{
    const int k = threadIdx.x / G, lane = threadIdx.x % G;
    if (!meta.kind || k >= meta.np) return;
    const int v = sm.perm[k];
    if (v < 0) return;
    constexpr int V = 16 / sizeof(T);
    const int R = P.R;
    const size_t rowb = (size_t)R * sizeof(T);
    const long long a = meta.a;
    const T *in = reinterpret_cast<const T *>(P.in);
    const T *x = reinterpret_cast<const T *>(P.x) + a * P.N * P.ld_x;
    const T *src_in = nullptr;
    if (!TR) src_in = in + ((P.mode == MODE_J && P.shared_in ? 0 : a * P.N) + v) * P.ld_in;
    else if (P.mode == MODE_J) src_in = sm.rec[k] >= 0 ? in + (a * P.n_rec + sm.rec[k]) * P.ld_in : nullptr;
    else src_in = in + (a * P.N + v) * P.ld_in;
    const int e0 = sm.rp[k], cnt = sm.rp[k + 1] - e0;
    for (int r = lane * V; r < R; r += G * V) {
        if (src_in) cp_async16(rows + (size_t)k * rowb + r * sizeof(T), src_in + r);
        for (int e = 0; e < cnt; ++e)
            cp_async16(rows + (size_t)(P.item_max + e0 + e) * rowb + r * sizeof(T), x + (long long)sm.en[e0 + e] * P.ld_x + r);
    }
}

template <typename T, bool TR>
__device__ __forceinline__ void staged_compute(const TravParams &P, const Stage<T> &sm, const StagedMeta &meta,
                                               const unsigned char *rows, int G)
{
    const int k = threadIdx.x / G, lane = threadIdx.x % G;
    if (k >= meta.np) return;
    const int v = sm.perm[k];
    if (v < 0) return;
    constexpr int V = 16 / sizeof(T);
    const int R = P.R;
    const size_t rowb = (size_t)R * sizeof(T);
    T *x = reinterpret_cast<T *>(P.x) + meta.a * P.N * P.ld_x;
    const int e0 = sm.rp[k], cnt = sm.rp[k + 1] - e0;
    const int rec = sm.rec[k];
    const T c = sm.cq[k];
    const bool has_in = !(TR && P.mode == MODE_J && rec < 0);
    const T scale = (!TR && P.mode == MODE_J) ? c : T(1);
    for (int r = lane * V; r < R; r += G * V) {
        Pack<T, V> acc;
        if (has_in) {
            Pack<T, V> q = *reinterpret_cast<const Pack<T, V> *>(rows + (size_t)k * rowb + r * sizeof(T));
#pragma unroll
            for (int u = 0; u < V; ++u) acc.v[u] = scale * q.v[u];
        } else {
#pragma unroll
            for (int u = 0; u < V; ++u) acc.v[u] = T(0);
        }
        for (int e = 0; e < cnt; ++e) {
            const T w = sm.ew[e0 + e];
            Pack<T, V> xv = *reinterpret_cast<const Pack<T, V> *>(rows + (size_t)(P.item_max + e0 + e) * rowb + r * sizeof(T));
#pragma unroll
            for (int u = 0; u < V; ++u) acc.v[u] += w * xv.v[u];
        }
        node_output<T, V, TR>(P, meta.a, v, meta.p0 + k, rec, c, r, x, acc);
    }
}

template <typename T, bool TR>
__global__ void __launch_bounds__(512) k_traverse_staged(const TravParams *__restrict__ Pd, int G, int first, int n)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ Stage<T> sm[2];
    __shared__ StagedMeta meta[2];
    const TravParams &P = *Pd;
    const size_t stage_bytes = (size_t)P.item_max * (1 + MAX_ROW) * P.R * sizeof(T);
    grid_dependents_launch();
    int idx = blockIdx.x;
    if (idx >= n) return;
    staged_structure<T>(P, sm[0], meta[0], first + idx);
    grid_dependency_wait();          // rows of earlier levels are complete and visible
    __syncthreads();
    staged_issue<T, TR>(P, sm[0], meta[0], dyn, G);
    cp_async_commit();
    for (int j = 0;; ++j) {
        const int buf = j & 1;
        const int nxt = idx + gridDim.x;
        if (nxt < n) {
            staged_structure<T>(P, sm[buf ^ 1], meta[buf ^ 1], first + nxt);
            __syncthreads();
            staged_issue<T, TR>(P, sm[buf ^ 1], meta[buf ^ 1], dyn + (buf ^ 1) * stage_bytes, G);
        }
        cp_async_commit();           // (possibly empty) group of the next item
        cp_async_wait<1>();          // this thread's copies of the current item have landed
        if (meta[buf].kind) staged_compute<T, TR>(P, sm[buf], meta[buf], dyn + buf * stage_bytes, G);
        else run_block<T, TR>(P, meta[buf].a, meta[buf].block);
        __syncthreads();             // structure of this stage is reused two items later
        if (nxt >= n) break;
        idx = nxt;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------- shared-memory item stages
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
template <typename T> __device__ __forceinline__ void cp_async_t(T *dst, const T *src)
{
    if (sizeof(T) == 8) cp_async8(dst, src);
    else cp_async4(dst, src);
}

template <typename T> struct ItemStage {
    T cq[ITEM_MAX];
    T ew[MAX_ROW * ITEM_MAX];
    int perm[ITEM_MAX];
    int rec[ITEM_MAX];
    int rp[ITEM_MAX + 1];        // raw local edge offsets (subtract ebx)
    int en[MAX_ROW * ITEM_MAX];
    int deps[DEP_MAX];           // items holding the upstream rows (persistent schedule)
    int nd;                      // their number; -1: wait for the whole previous level
    int4 it;                     // item descriptor
    int idx;                     // ticket; >= nitems ends the compute warps
    int ebx, eby;                // the item's local edge range
};

// row of the traversal's input for a position of source a, or nullptr (zero input)
template <typename T, bool TR>
__device__ __forceinline__ const T *input_row(const TravParams &P, long long a, int v, int rec)
{
    const T *in = reinterpret_cast<const T *>(P.in);
    if (!TR) return in + ((P.mode == MODE_J && P.shared_in ? 0 : a * P.N) + v) * P.ld_in;
    if (P.mode == MODE_J) return rec >= 0 ? in + (a * P.n_rec + rec) * P.ld_in : nullptr;
    return in + (a * P.N + v) * P.ld_in;
}

template <typename T, int V, bool TR>
__device__ __forceinline__ void run_stage_singletons(const TravParams &P, const ItemStage<T> &S, const unsigned char *tile,
                                                int G)
{
    const int lane = threadIdx.x % G, slot = threadIdx.x / G, nslot = blockDim.x / G;
    const long long a = S.it.x;
    const int p0 = S.it.z, np = S.it.w - S.it.z;
    const int R = P.R;
    const size_t rowb = (size_t)R * sizeof(T);
    T *x = reinterpret_cast<T *>(P.x) + a * P.N * P.ld_x;
    for (int k = slot; k < np; k += nslot) {
        const int v = S.perm[k];
        if (v < 0) continue;      // member of a nontrivial block
        const int e0 = S.rp[k] - S.ebx, cnt = S.rp[k + 1] - S.rp[k];
        const int rec = S.rec[k];
        const T c = S.cq[k];
        const bool has_in = !(TR && P.mode == MODE_J && rec < 0);
        const T scale = (!TR && P.mode == MODE_J) ? c : T(1);
        for (int r = lane * V; r < R; r += G * V) {
            Pack<T, V> xv[MAX_ROW];
#pragma unroll
            for (int e = 0; e < MAX_ROW; ++e)
                if (e < cnt) xv[e] = load_l2<T, V>(x + (long long)S.en[e0 + e] * P.ld_x + r);
            Pack<T, V> acc;
            if (tile) {
                if (has_in) {
                    const Pack<T, V> q = *reinterpret_cast<const Pack<T, V> *>(tile + (size_t)k * rowb + r * sizeof(T));
#pragma unroll
                    for (int u = 0; u < V; ++u) acc.v[u] = scale * q.v[u];
                } else {
#pragma unroll
                    for (int u = 0; u < V; ++u) acc.v[u] = T(0);
                }
            } else {
                acc = node_input<T, V, TR>(P, (int)a, v, rec, c, r);
            }
#pragma unroll
            for (int e = 0; e < MAX_ROW; ++e)
                if (e < cnt) {
                    const T w = S.ew[e0 + e];
#pragma unroll
                    for (int u = 0; u < V; ++u) acc.v[u] += w * xv[e].v[u];
                }
            node_output<T, V, TR>(P, (int)a, v, p0 + k, rec, c, r, x, acc);
        }
    }
}

// ---------------------------------------------------------------- persistent schedule
// One launch; CTAs take items by ticket, each CTA in increasing ticket order, and an
// item waits (bounded) only for lower tickets -- the items holding its upstream rows,
// or every item of its source's previous level -- so every item waited on is held by a
// running CTA or done: no deadlock.  Per CTA the work of neighbouring items overlaps:
//   while item c computes, the structure (and dependency list) of the next item n is
//   copied into the other shared-memory stage with cp.async and the ticket after n is
//   taken; after c, n's input rows are copied into shared memory with cp.async while
//   warp 0 waits for n's dependencies.
// So between two dependent levels only the wait, the upstream gathers (L2) and the
// release (one fence) remain.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void st_relaxed(int *p, int v)
{
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// structure of item S.idx (descriptor already in S) into S, by all threads of the CTA
template <typename T>
__device__ __forceinline__ void issue_structure(const TravParams &P, ItemStage<T> &S)
{
    const int i = S.idx;
    const int4 it = S.it;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (P.ndeps && it.y > 0) {
        if (tid < DEP_MAX) cp_async4(&S.deps[tid], P.deps + (long long)i * DEP_MAX + tid);
        else if (tid == DEP_MAX) cp_async4(&S.nd, P.ndeps + i);
    }
    if (it.z < 0) return;
    const long long N = P.N, a = it.x;
    const int p0 = it.z, np = it.w - it.z, ne = S.eby - S.ebx;
    const int *rp = P.rowptr + a * (N + 1) + p0;
    const long long o = a * N + p0;
    const T *cq = reinterpret_cast<const T *>(P.cq) + o;
    for (int k = tid; k <= np; k += nt) {
        cp_async4(&S.rp[k], rp + k);
        if (k < np) {
            cp_async4(&S.perm[k], P.perm + o + k);
            cp_async4(&S.rec[k], P.rec_slot + o + k);
            cp_async_t<T>(&S.cq[k], cq + k);
        }
    }
    const long long e0 = P.ebase[a] + S.ebx;
    const T *ew = reinterpret_cast<const T *>(P.ew) + e0;
    for (int k = tid; k < ne; k += nt) {
        cp_async4(&S.en[k], P.enode + e0 + k);
        cp_async_t<T>(&S.ew[k], ew + k);
    }
}

// input rows of item S (structure visible) into the tile, 16 bytes per copy
template <typename T, bool TR>
__device__ __forceinline__ void issue_input(const TravParams &P, const ItemStage<T> &S, unsigned char *tile)
{
    if (S.it.z < 0) return;
    const long long a = S.it.x;
    const int np = S.it.w - S.it.z;
    const size_t rowb = (size_t)P.R * sizeof(T);
    const int chunks = (int)(rowb / 16);
    for (int q = threadIdx.x; q < np * chunks; q += blockDim.x) {
        const int k = q / chunks, c = q - k * chunks;
        const int v = S.perm[k];
        if (v < 0) continue;
        const T *src = input_row<T, TR>(P, a, v, S.rec[k]);
        if (src) cp_async16(tile + (size_t)k * rowb + (size_t)c * 16, reinterpret_cast<const unsigned char *>(src) + (size_t)c * 16);
    }
}

// descriptor of ticket i into S (one thread)
template <typename T>
__device__ __forceinline__ void load_desc(const TravParams &P, ItemStage<T> &S, int i)
{
    S.idx = i;
    if (i < P.nitems) {
        S.it = P.items[i];
        const int2 eb = P.ebeg[i];
        S.ebx = eb.x;
        S.eby = eb.y;
    }
    S.nd = -1;
}

template <typename T, int V, bool TR>
__global__ void __launch_bounds__(256, 4) k_traverse_persistent(TravParams P, int G, int tile_bytes)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ ItemStage<T> stg[2];
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    const int nitems = P.nitems;
    const unsigned FULL = 0xffffffffu;
    if (tid == 0) {
        load_desc(P, stg[0], atomicAdd(P.ticket, 1));
        stg[1].idx = atomicAdd(P.ticket, 1);
    }
    __syncthreads();
    if (stg[0].idx >= nitems) return;
    issue_structure<T>(P, stg[0]);
    cp_async_commit();
    if (tid == 0) load_desc(P, stg[1], stg[1].idx);
    cp_async_wait<0>();
    __syncthreads();
    if (tile_bytes) issue_input<T, TR>(P, stg[0], dyn);
    cp_async_commit();
    for (int b = 0;; b ^= 1) {
        ItemStage<T> &C = stg[b];
        ItemStage<T> &Nx = stg[b ^ 1];
        const int4 it = C.it;
        const int i = C.idx;
        // ---- wait (warp 0) for the items holding the upstream rows
        if (tid < 32) {
            int ok = 1;
            if (it.y > 0) {
                const int nd = C.nd;
                const int *flag = nullptr;
                int need = 1;
                if (nd < 0) {
                    if (tid == 0) {
                        flag = P.done + (long long)it.x * P.maxL + it.y - 1;
                        need = P.item_cnt[(long long)it.x * P.maxL + it.y - 1];
                    }
                } else if (tid < nd) {
                    flag = P.item_done + C.deps[tid];
                }
                bool mine = flag == nullptr || ld_acquire(flag) >= need;
                if (!__all_sync(FULL, mine)) {
                    const unsigned long long t0 = global_ns();
                    for (;;) {
                        __nanosleep(32);
                        if (!mine) mine = ld_acquire(flag) >= need;
                        if (__all_sync(FULL, mine)) break;
                        int stop = 0;
                        if (tid == 0) {
                            if (*(volatile int *)P.err != 0) stop = 1;
                            else if (global_ns() - t0 > P.timeout_ns) {
                                if (atomicCAS(P.err, 0, DEV_TIMEOUT) == 0) { P.err[1] = it.x; P.err[2] = it.y; P.err[3] = i; }
                                stop = 1;
                            }
                        }
                        if (__shfl_sync(FULL, stop, 0)) { ok = 0; break; }
                    }
                }
            }
            if (tid == 0) s_ok = ok;
        }
        cp_async_wait<0>();          // this thread's copies of C's input rows have landed
        __syncthreads();             // (A) dependencies done, C's inputs visible
        if (!s_ok) break;
        const bool has_next = Nx.idx < nitems;
        if (has_next) issue_structure<T>(P, Nx);
        cp_async_commit();
        int t2 = 0;
        if (tid == 1 && has_next) t2 = atomicAdd(P.ticket, 1);   // its value is first needed after (B)
        // ---- compute C
        if (it.z >= 0) run_stage_singletons<T, V, TR>(P, C, tile_bytes ? dyn + b * (size_t)tile_bytes : nullptr, G);
        else run_block<T, TR>(P, it.x, ~it.z);
        __syncthreads();             // (B) every row of C written
        if (tid == 32) {
            // release pattern: one fence, then the (relaxed) completion marks
            fence_acq_rel_gpu();
            atomicAdd(P.done + (long long)it.x * P.maxL + it.y, 1);
            st_relaxed(P.item_done + i, 1);
        }
        if (tid == 1) {
            if (has_next) load_desc(P, C, t2);
            else C.idx = nitems;
        }
        cp_async_wait<0>();          // this thread's copies of Nx's structure have landed
        __syncthreads();             // (C) Nx's structure and the following descriptor visible
        if (!has_next) break;
        if (tile_bytes) issue_input<T, TR>(P, Nx, dyn + (b ^ 1) * (size_t)tile_bytes);
        cp_async_commit();
    }
    cp_async_wait<0>();
}

// g[j][r] = sum_a cq_a[j] lam_a[j][r] in source order.  FP64 path: FP64 products and
// sum.  FP32 path: FP32 products with a compensated (Kahan) FP32 sum, so the rounding
// error does not grow with the number of sources (B300's FP64 rate would make an FP64
// accumulation the bottleneck of this pass).  Loads are issued SUMB at a time.
constexpr int SUMB = 8;

template <typename T>
__global__ void k_source_sum(long long N, int S, int R, const T *__restrict__ cqn, const int *__restrict__ pos,
                             const T *__restrict__ lam, long long ld_lam, T *__restrict__ g, long long ld_g)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= N * R) return;
    long long j = t / R;
    int r = (int)(t - j * R);
    T acc = 0, comp = 0;
    for (int a0 = 0; a0 < S; a0 += SUMB) {
        T vals[SUMB];
#pragma unroll
        for (int b = 0; b < SUMB; ++b)
            vals[b] = a0 + b < S ? __ldg(cqn + (long long)(a0 + b) * N + j) *
                                       __ldcs(lam + ((long long)(a0 + b) * N + __ldg(pos + (long long)(a0 + b) * N + j)) * ld_lam + r)
                                 : T(0);
#pragma unroll
        for (int b = 0; b < SUMB; ++b) {
            if (sizeof(T) == 8) {
                acc += vals[b];
            } else {
                T y = vals[b] - comp;
                T t = acc + y;
                comp = (t - acc) - y;
                acc = t;
            }
        }
    }
    g[j * ld_g + r] = acc;
}

// Vector form of the same sum (same operations per element, in the same source order):
// a CTA takes a tile of rows j, stages pos_a[j] and cq_a[j] of up to SUM_STAGE sources in
// shared memory, and each thread (one row, one V-wide column chunk) then issues the
// row loads of SUM_GRP sources at once.  The loads of lam stream (evict-first).
constexpr int SUM_STAGE = 32;
constexpr int SUM_GRP = 12;
constexpr int SUM_ROWS = 64;

template <typename T, int V>
__global__ void __launch_bounds__(256) k_source_sum_vec(long long N, int S, int R, int rows,
                                                        const T *__restrict__ cqn, const int *__restrict__ pos,
                                                        const T *__restrict__ lam, long long ld_lam, T *__restrict__ g,
                                                        long long ld_g)
{
    using VT = typename VecT<T, V>::type;
    __shared__ int s_pos[SUM_STAGE * SUM_ROWS];
    __shared__ T s_c[SUM_STAGE * SUM_ROWS];
    const int L = R / V;
    const int t = threadIdx.x, row = t / L, c = t - row * L;
    const long long j0 = (long long)blockIdx.x * rows, j = j0 + row;
    const int r = c * V;
    Pack<T, V> acc, comp;
#pragma unroll
    for (int u = 0; u < V; ++u) { acc.v[u] = T(0); comp.v[u] = T(0); }
    for (int s0 = 0; s0 < S; s0 += SUM_STAGE) {
        const int ns = min(SUM_STAGE, S - s0);
        __syncthreads();
        for (int q = t; q < ns * rows; q += blockDim.x) {
            const int a = q / rows, rr = q - a * rows;
            const long long jj = j0 + rr;
            if (jj < N) {
                s_pos[a * rows + rr] = __ldg(pos + (long long)(s0 + a) * N + jj);
                s_c[a * rows + rr] = __ldg(cqn + (long long)(s0 + a) * N + jj);
            }
        }
        __syncthreads();
        if (j >= N) continue;
        for (int a0 = 0; a0 < ns; a0 += SUM_GRP) {
            Pack<T, V> vals[SUM_GRP];
#pragma unroll
            for (int b = 0; b < SUM_GRP; ++b)
                if (a0 + b < ns) {
                    const int a = a0 + b;
                    const VT x = __ldcs(reinterpret_cast<const VT *>(
                        lam + ((long long)(s0 + a) * N + s_pos[a * rows + row]) * ld_lam + r));
                    memcpy(&vals[b], &x, sizeof(VT));
                }
#pragma unroll
            for (int b = 0; b < SUM_GRP; ++b)
                if (a0 + b < ns) {
                    const T cc = s_c[(a0 + b) * rows + row];
#pragma unroll
                    for (int u = 0; u < V; ++u) {
                        const T prod = cc * vals[b].v[u];
                        if (sizeof(T) == 8) {
                            acc.v[u] += prod;
                        } else {
                            const T y = prod - comp.v[u];
                            const T tt = acc.v[u] + y;
                            comp.v[u] = (tt - acc.v[u]) - y;
                            acc.v[u] = tt;
                        }
                    }
                }
        }
    }
    if (j < N) store<T, V>(g + j * ld_g + r, acc);
}

// receiver sampling P: out[a][k] = field[a][rec[a][k]]
__global__ void k_sample(long long N, int S, int n_rec, const int *__restrict__ rec, const double *__restrict__ field,
                         double *__restrict__ out)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)S * n_rec) return;
    long long a = i / n_rec;
    out[i] = field[a * N + rec[i]];
}

void launch_sample(long long N, int S, int n_rec, const int *rec, const double *field, double *out, cudaStream_t st)
{
    long long n = (long long)S * n_rec;
    k_sample<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(N, S, n_rec, rec, field, out);
}

// ---------------------------------------------------------------- host side
int ensure_workspace(Tangent *t, size_t vec_bytes, size_t blk_elems)
{
    if (vec_bytes > t->ws_vec_bytes) {
        if (t->ws_vec) cudaFree(t->ws_vec);
        t->ws_vec = nullptr;
        t->ws_vec_bytes = 0;
        EIK_CHECK(cudaMalloc(&t->ws_vec, vec_bytes));
        t->ws_vec_bytes = vec_bytes;
    }
    if (blk_elems > t->ws_blk_elems) {
        if (t->ws_blk) cudaFree(t->ws_blk);
        t->ws_blk = nullptr;
        t->ws_blk_elems = 0;
        EIK_CHECK(cudaMalloc(&t->ws_blk, blk_elems * sizeof(double)));
        t->ws_blk_elems = blk_elems;
    }
    return EIK_OK;
}

template <typename T, int V, bool TR, int NPS>
static int launch_levels(Tangent *t, int G, int threads, int first_step, TravParams *Pd, cudaStream_t st)
{
    const std::vector<int> &sp = TR ? t->step_ptr_bwd : t->step_ptr_fwd;
    for (int s = first_step; s < t->maxL; ++s) {
        int n = sp[s + 1] - sp[s];
        if (n <= 0) continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)n);
        cfg.blockDim = dim3((unsigned)threads);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        // the first level follows the parameter upload: launch it fully ordered
        cfg.attrs = attr;
        cfg.numAttrs = s == first_step ? 0 : 1;
        EIK_CHECK(cudaLaunchKernelEx(&cfg, k_traverse_level<T, V, TR, NPS>, (const TravParams *)Pd, G, sp[s]));
    }
    return EIK_OK;
}

template <typename T, int V, bool TR>
static int launch_staged(Tangent *t, int G, int threads, size_t dyn, int per_sm, TravParams *Pd, cudaStream_t st)
{
    const std::vector<int> &sp = TR ? t->step_ptr_bwd : t->step_ptr_fwd;
    const int cap = t->num_sms * per_sm;
    for (int s = 0; s < t->maxL; ++s) {
        int n = sp[s + 1] - sp[s];
        if (n <= 0) continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)std::min(n, cap));
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = dyn;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = s == 0 ? 0 : 1;
        EIK_CHECK(cudaLaunchKernelEx(&cfg, k_traverse_staged<T, TR>, (const TravParams *)Pd, G, sp[s], n));
    }
    return EIK_OK;
}

template <typename T, int V, bool TR>
static int launch_traverse(Tangent *t, TravParams &P, int G, cudaStream_t st)
{
    const size_t rowb = (size_t)P.R * sizeof(T);
    const bool staged_ok = rowb % 16 == 0 && rowb >= 64 && (P.ld_in * sizeof(T)) % 16 == 0 &&
                           (P.ld_x * sizeof(T)) % 16 == 0 && V * sizeof(T) == 16;
    const size_t staged_dyn = 2 * (size_t)t->item_max * (1 + MAX_ROW) * rowb;
    if (t->opts.schedule == EIK_SCHED_STAGED && staged_ok && t->item_max * G <= 512 && staged_dyn <= 200 * 1024) {
        // one thread per (position, 16-byte lane); rows wider than 32 lanes loop over columns
        const int threads = std::max(32, t->item_max * G);
        const size_t dyn = staged_dyn;
        EIK_CHECK(cudaFuncSetAttribute(k_traverse_staged<T, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        int per_sm = 0;
        EIK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traverse_staged<T, TR>, threads, dyn));
        per_sm = std::max(per_sm, 1);
        if (!t->params_d) EIK_CHECK(cudaMalloc(&t->params_d, 2 * sizeof(TravParams)));
        TravParams *Pd = t->params_d + (TR ? 1 : 0);
        k_set_params<<<1, 1, 0, st>>>(Pd, P);
        EIK_CHECK_LAUNCH();
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        EIK_CHECK(cudaStreamIsCapturing(st, &cs));
        if (cs != cudaStreamCaptureStatusNone || !t->opts_graph)
            return launch_staged<T, V, TR>(t, G, threads, dyn, per_sm, Pd, st);
        const long long key = (1ll << 50) | ((long long)TR << 40) | ((long long)sizeof(T) << 32) | ((long long)P.R << 8) | G;
        cudaGraphExec_t &exec = t->level_graphs[key];
        if (!exec) {
            if (!t->cap_stream) EIK_CHECK(cudaStreamCreateWithFlags(&t->cap_stream, cudaStreamNonBlocking));
            EIK_CHECK(cudaStreamBeginCapture(t->cap_stream, cudaStreamCaptureModeThreadLocal));
            int rc = launch_staged<T, V, TR>(t, G, threads, dyn, per_sm, Pd, t->cap_stream);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(t->cap_stream, &g);
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
            e = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { exec = nullptr; return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__); }
        }
        EIK_CHECK(cudaGraphLaunch(exec, st));
        return EIK_OK;
    }
    if (t->opts.schedule == EIK_SCHED_LEVELS || t->opts.schedule == EIK_SCHED_STAGED) {
        // one item per CTA; slots of G lanes, one node in flight per slot
        const bool two = false;
        const int threads = std::min(256, std::max(32, t->item_max * G));
        if (!t->params_d) EIK_CHECK(cudaMalloc(&t->params_d, 2 * sizeof(TravParams)));
        TravParams *Pd = t->params_d + (TR ? 1 : 0);
        k_set_params<<<1, 1, 0, st>>>(Pd, P);
        EIK_CHECK_LAUNCH();
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        EIK_CHECK(cudaStreamIsCapturing(st, &cs));
        if (cs != cudaStreamCaptureStatusNone || !t->opts_graph) {
            // the caller is capturing (or graphs are off): launch directly into its stream
            return two ? launch_levels<T, V, TR, 2>(t, G, threads, 0, Pd, st)
                       : launch_levels<T, V, TR, 1>(t, G, threads, 0, Pd, st);
        }
        const long long key = ((long long)TR << 40) | ((long long)sizeof(T) << 32) | ((long long)V << 16) | G;
        cudaGraphExec_t &exec = t->level_graphs[key];
        if (!exec) {
            if (!t->cap_stream) EIK_CHECK(cudaStreamCreateWithFlags(&t->cap_stream, cudaStreamNonBlocking));
            EIK_CHECK(cudaStreamBeginCapture(t->cap_stream, cudaStreamCaptureModeThreadLocal));
            int rc = two ? launch_levels<T, V, TR, 2>(t, G, threads, 0, Pd, t->cap_stream)
                         : launch_levels<T, V, TR, 1>(t, G, threads, 0, Pd, t->cap_stream);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(t->cap_stream, &g);
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
            e = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { exec = nullptr; return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__); }
        }
        EIK_CHECK(cudaGraphLaunch(exec, st));
        return EIK_OK;
    }
    // persistent: one thread per (position, lane) of an item, between 64 (two warps: the
    // waiting warp and the releasing thread 32) and 256; input rows staged in shared
    // memory when they are whole 16-byte chunks and an item's rows fit 32 KB
    const int threads = std::min(256, std::max(64, (t->item_max * G + 31) / 32 * 32));
    const bool tile = V * sizeof(T) == 16 && rowb % 16 == 0 && (P.ld_in * sizeof(T)) % 16 == 0 &&
                      ((uintptr_t)P.in & 15) == 0 && (size_t)t->item_max * rowb <= 32768;
    const int tile_bytes = tile ? (int)(t->item_max * rowb) : 0;
    const size_t dyn = 2 * (size_t)tile_bytes;
    EIK_CHECK(cudaFuncSetAttribute(k_traverse_persistent<T, V, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int per_sm = t->opts.ctas_per_sm;
    if (per_sm <= 0) {
        EIK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traverse_persistent<T, V, TR>, threads, dyn));
        per_sm = std::max(per_sm, 1);
    }
    long long grid = std::min<long long>((long long)t->num_sms * per_sm, P.nitems);
    grid = std::max<long long>(grid, 1);
    EIK_CHECK(cudaMemsetAsync(P.done, 0, (size_t)t->S * t->maxL * sizeof(int), st));
    EIK_CHECK(cudaMemsetAsync(P.ticket, 0, sizeof(int), st));
    EIK_CHECK(cudaMemsetAsync(P.item_done, 0, (size_t)std::max(P.nitems, 1) * sizeof(int), st));
    k_traverse_persistent<T, V, TR><<<(unsigned)grid, threads, dyn, st>>>(P, G, tile_bytes);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

template <typename T, bool TR>
static int dispatch_v(Tangent *t, TravParams &P, cudaStream_t st)
{
    // widest vector that divides R and keeps every row 16-byte aligned when possible
    const int R = P.R;
    auto fits = [&](int v) {
        return R % v == 0 && P.ld_in % v == 0 && P.ld_x % v == 0 && P.ld_aux % v == 0 && P.ld_out % v == 0;
    };
    int V = 1;
    if (sizeof(T) == 4 && fits(4)) V = 4;
    else if (fits(2)) V = 2;
    int lanes = (R + V - 1) / V;
    int G = 1;
    while (G < lanes && G < 32) G <<= 1;
    if (sizeof(T) == 4) {
        if (V == 4) return launch_traverse<float, 4, TR>(t, P, G, st);
        if (V == 2) return launch_traverse<float, 2, TR>(t, P, G, st);
        return launch_traverse<float, 1, TR>(t, P, G, st);
    }
    if (V == 2) return launch_traverse<double, 2, TR>(t, P, G, st);
    return launch_traverse<double, 1, TR>(t, P, G, st);
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

// g[j][r] (row stride ld_g) = sum over sources of c_a[j] * x_a[j][r] for the w columns the
// workspace holds (the reverse field of the last traversal, canonical order)
int source_sum(Tangent *t, int w, void *g, long long ld_g, int dtype, cudaStream_t st)
{
    const void *xp = t->ws_vec;
    const int V = dtype == EIK_F32 ? 4 : 2;
    const int L = w / V;
    if (w % V == 0 && ld_g % V == 0 && aligned16(xp) && aligned16(g) && L <= 256) {
        const int rows = std::min(SUM_ROWS, std::max(1, 256 / L));
        const unsigned blocks = (unsigned)((t->N + rows - 1) / rows);
        if (dtype == EIK_F32)
            k_source_sum_vec<float, 4><<<blocks, rows * L, 0, st>>>(t->N, t->S, w, rows, t->cqn32, t->pos,
                                                                    (const float *)xp, (long long)w, (float *)g, ld_g);
        else
            k_source_sum_vec<double, 2><<<blocks, rows * L, 0, st>>>(t->N, t->S, w, rows, t->cqn64, t->pos,
                                                                     (const double *)xp, (long long)w, (double *)g, ld_g);
    } else {
        const long long n = t->N * w;
        const unsigned blocks = (unsigned)((n + 255) / 256);
        if (dtype == EIK_F32)
            k_source_sum<float><<<blocks, 256, 0, st>>>(t->N, t->S, w, t->cqn32, t->pos, (const float *)xp, (long long)w,
                                                        (float *)g, ld_g);
        else
            k_source_sum<double><<<blocks, 256, 0, st>>>(t->N, t->S, w, t->cqn64, t->pos, (const double *)xp, (long long)w,
                                                         (double *)g, ld_g);
    }
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

int traverse(Tangent *t, bool TR, int mode, const void *in, int shared_in, int R, void *out_full, void *out_aux,
             int sum_sources, int dtype, cudaStream_t st)
{
    if (R <= 0) { set_error("R must be positive"); return EIK_ERR_INVALID; }
    if (!in) { set_error("input pointer is NULL"); return EIK_ERR_INVALID; }
    if (dtype != EIK_F32 && dtype != EIK_F64) { set_error("bad dtype"); return EIK_ERR_INVALID; }
    const size_t esz = dtype == EIK_F32 ? 4 : 8;
    const void *ptrs[3] = {in, out_full, out_aux};
    for (const void *p : ptrs)
        if (p && !aligned16(p)) { set_error("device buffers must be 16-byte aligned"); return EIK_ERR_INVALID; }
    // right-hand sides are processed in column chunks of Rc (all of R by default); a chunk
    // is a column slice of the caller's [.][R] buffers, so only the workspace shrinks
    int Rc = R;
    if (t->opts.rhs_chunk > 0 && t->opts.rhs_chunk < R) {
        Rc = t->opts.rhs_chunk;
        const int unit = dtype == EIK_F32 ? 4 : 2;
        if (R % unit == 0) Rc = std::max(unit, Rc / unit * unit);
    }
    // the transported field always lives in the canonical-order workspace
    size_t need_vec = (size_t)t->S * t->N * Rc * esz;
    int rc = ensure_workspace(t, need_vec, (size_t)t->ws_rows * Rc);
    if (rc) return rc;
    for (int r0 = 0; r0 < R; r0 += Rc) {
        const int w = std::min(Rc, R - r0);
        const char *inp = static_cast<const char *>(in) + r0 * esz;
        char *xp = static_cast<char *>(t->ws_vec);
        char *outp = out_full ? static_cast<char *>(out_full) + r0 * esz : nullptr;
        char *auxp = out_aux ? static_cast<char *>(out_aux) + r0 * esz : nullptr;
        TravParams P{};
        P.S = t->S; P.R = w; P.n_rec = t->n_rec; P.maxL = t->maxL; P.nitems = t->nitems; P.N = t->N;
        P.item_max = t->item_max;
        P.ld_in = R; P.ld_x = w; P.ld_aux = R; P.ld_out = R;
        P.out = outp;
        P.mode = mode; P.shared_in = shared_in; P.sum = sum_sources;
        P.perm = t->perm;
        P.rowptr = TR ? t->cptr : t->rowptr;
        P.enode = TR ? t->dn_node : t->up_node;
        P.ew = dtype == EIK_F32 ? (const void *)(TR ? t->dn_w32 : t->up_w32) : (const void *)(TR ? t->dn_w64 : t->up_w64);
        P.ew64 = TR ? t->dn_w64 : t->up_w64;
        P.ebase = TR ? t->tbase_d : t->ebase_d;
        P.cq = dtype == EIK_F32 ? (const void *)t->cq32 : (const void *)t->cq64;
        P.cq64 = t->cq64;
        P.rec_slot = t->rec_slot;
        P.in = inp; P.x = xp; P.aux = auxp;
        P.items = TR ? t->items_bwd : t->items_fwd;
        P.ebeg = TR ? t->ebeg_bwd : t->ebeg_fwd;
        P.item_cnt = t->item_cnt + (TR ? (size_t)t->S * t->maxL : 0);
        P.done = t->done; P.ticket = t->ticket; P.err = t->err;
        P.deps = TR ? t->deps_bwd : t->deps_fwd;
        // while a test hold is in place every item takes the level wait it targets
        P.ndeps = t->opts.item_deps && t->holds.empty() ? (TR ? t->ndeps_bwd : t->ndeps_fwd) : nullptr;
        P.item_done = t->item_done;
        P.blk_desc = t->blk_desc; P.blk_off = t->blk_off; P.binv = t->binv; P.ws = t->ws_blk;
        P.timeout_ns = (unsigned long long)(t->opts.wait_timeout_s * 1e9);
        if (dtype == EIK_F32) rc = TR ? dispatch_v<float, true>(t, P, st) : dispatch_v<float, false>(t, P, st);
        else rc = TR ? dispatch_v<double, true>(t, P, st) : dispatch_v<double, false>(t, P, st);
        if (rc) return rc;
        if (TR && mode == MODE_J && sum_sources && out_aux) {
            rc = source_sum(t, w, auxp, (long long)R, dtype, st);
            if (rc) return rc;
        }
    }
    return EIK_OK;
}

}  // namespace eik
