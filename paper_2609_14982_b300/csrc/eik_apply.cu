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
#include "eik_trav.h"
#include "eik_vec.cuh"

namespace eik {

// ---------------------------------------------------------------- singleton items
// The structure of one item (at most ITEM_MAX positions of one level of one source and
// their rows) is staged into shared memory by all threads in one round of independent
// loads; afterwards a node costs only its own vector loads (input, upstream values),
// all issued before they are summed.
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

// FP64 substitution with a block's partial-pivot factors P A_C = L U (large blocks), one
// warp per right-hand-side column, the dot products split over the lanes:
//   A_C x = b:    apply the row swaps to b, L y = P b (unit lower), U x = y;
//   A_C^T x = b:  U^T z = b, L^T w = z, then undo the row swaps (x = P^T w).
// W holds b on entry and x on exit, [k][R] row-major.
__device__ __forceinline__ double warp_sum_d(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ void block_lu_solve(const double *__restrict__ LU, const int *__restrict__ piv, int k, double *W, int R,
                               bool tr, int tid, int nthr)
{
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    for (int r = warp; r < R; r += nwarp) {
        double *x = W + r;
        if (!tr) {
            if (lane == 0)
                for (int m = 0; m < k; ++m) {
                    const int q = piv[m];
                    if (q != m) { const double t = x[(long long)m * R]; x[(long long)m * R] = x[(long long)q * R]; x[(long long)q * R] = t; }
                }
            __syncwarp();
            for (int m = 1; m < k; ++m) {
                double acc = 0.0;
                for (int j = lane; j < m; j += 32) acc += LU[(long long)m * k + j] * x[(long long)j * R];
                acc = warp_sum_d(acc);
                if (lane == 0) x[(long long)m * R] -= acc;
                __syncwarp();
            }
            for (int m = k - 1; m >= 0; --m) {
                double acc = 0.0;
                for (int j = m + 1 + lane; j < k; j += 32) acc += LU[(long long)m * k + j] * x[(long long)j * R];
                acc = warp_sum_d(acc);
                if (lane == 0) x[(long long)m * R] = (x[(long long)m * R] - acc) / LU[(long long)m * k + m];
                __syncwarp();
            }
        } else {
            for (int m = 0; m < k; ++m) {
                double acc = 0.0;
                for (int j = lane; j < m; j += 32) acc += LU[(long long)j * k + m] * x[(long long)j * R];
                acc = warp_sum_d(acc);
                if (lane == 0) x[(long long)m * R] = (x[(long long)m * R] - acc) / LU[(long long)m * k + m];
                __syncwarp();
            }
            for (int m = k - 2; m >= 0; --m) {
                double acc = 0.0;
                for (int j = m + 1 + lane; j < k; j += 32) acc += LU[(long long)j * k + m] * x[(long long)j * R];
                acc = warp_sum_d(acc);
                if (lane == 0) x[(long long)m * R] -= acc;
                __syncwarp();
            }
            if (lane == 0)
                for (int m = k - 1; m >= 0; --m) {
                    const int q = piv[m];
                    if (q != m) { const double t = x[(long long)m * R]; x[(long long)m * R] = x[(long long)q * R]; x[(long long)q * R] = t; }
                }
            __syncwarp();
        }
    }
}

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
        if (!EIK_POSITION_OK(P, a, p, v, rp[p], rp[p + 1] - rp[p], -1, en, rec)) continue;
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
    const bool by_lu = P.blk_lu_min > 0 && k >= P.blk_lu_min;
    if (by_lu) {
        block_lu_solve(P.lu + luo, P.piv + P.blk_off[3 * b + 1], k, W, R, TR, tid, nthr);
        sync();
    }
    for (long long idx = tid; idx < (long long)k * R; idx += nthr) {
        const int m = (int)(idx / R), r = (int)(idx % R);
        double val = 0.0;
        if (by_lu) {
            val = W[(long long)m * R + r];
        } else if (!TR) {
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

template <typename T, int IM = ITEM_MAX> struct ItemStage {
    T cq[IM];
    T ew[MAX_ROW * IM];
    int perm[IM];
    int rec[IM];
    int rp[IM + 1];              // raw local edge offsets (subtract ebx)
    int en[MAX_ROW * IM];
    int deps[DEP_MAX];           // items holding the upstream rows (persistent schedule)
    int nd;                      // their number; -1: wait for the whole previous level
    int4 it;                     // item descriptor
    int idx;                     // ticket; >= nitems ends the compute warps
    int ebx, eby;                // the item's local edge range
    int tan, tkt;                // multi-slot schedule: tangent of the item (idx is its item), ticket
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

template <typename T, int V, bool TR, int IM>
__device__ __forceinline__ void run_stage_singletons(const TravParams &P, const ItemStage<T, IM> &S, const unsigned char *tile,
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
        if (!EIK_POSITION_OK(P, a, p0 + k, v, e0, cnt, S.eby - S.ebx, S.en, rec)) continue;
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

// Lane-group form of the same item: a position's lanes (V-element vectors of right-hand
// sides) are split over G = lanes / W threads; thread (k0, g) takes lanes g, g + G, ...,
// g + (W-1) G of positions k0 + q * nslot, q < U, decodes each row once for its W lanes
// and issues all its upstream loads before any sum.  Same arithmetic, in the same order,
// as run_stage_singletons.
template <typename T, int V, int W, int U, bool TR, int IM>
__device__ __forceinline__ void run_stage_lanes(const TravParams &P, const ItemStage<T, IM> &S, const unsigned char *tile,
                                                int lanes)
{
    const int G = lanes / W;
    const int nslot = blockDim.x / G;
    const int k0 = threadIdx.x / G, g = threadIdx.x - k0 * G;
    if (k0 >= nslot) return;
    const long long a = S.it.x;
    const int p0 = S.it.z, np = S.it.w - S.it.z;
    const size_t rowb = (size_t)P.R * sizeof(T);
    const int lo = g * V, ls = G * V;
    T *x = reinterpret_cast<T *>(P.x) + a * P.N * P.ld_x;
    const bool J = P.mode == MODE_J;
    for (int kb = k0; kb < np; kb += U * nslot) {
        Pack<T, V> xv[U][3][W];
        int node[U], e0[U], cnt[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int k = kb + q * nslot;
            node[q] = k < np ? S.perm[k] : -1;
            cnt[q] = 0;
            e0[q] = 0;
            if (node[q] < 0) continue;
            e0[q] = S.rp[k] - S.ebx;
            cnt[q] = S.rp[k + 1] - S.rp[k];
            if (!EIK_POSITION_OK(P, a, p0 + k, node[q], e0[q], cnt[q], S.eby - S.ebx, S.en, S.rec[k])) {
                node[q] = -1;
                cnt[q] = 0;
                continue;
            }
#pragma unroll
            for (int e = 0; e < 3; ++e)
                if (e < cnt[q]) {
                    const T *src = x + (long long)S.en[e0[q] + e] * P.ld_x + lo;
#pragma unroll
                    for (int w = 0; w < W; ++w) xv[q][e][w] = load_l2<T, V>(src + w * ls);
                }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            if (node[q] < 0) continue;
            const int k = kb + q * nslot;
            const int rec = S.rec[k];
            const T c = S.cq[k];
            const bool has_in = !(TR && J && rec < 0);
            const T scale = (!TR && J) ? c : T(1);
            Pack<T, V> acc[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const int r = lo + w * ls;
                if (tile) {
                    if (has_in) {
                        const Pack<T, V> qv = *reinterpret_cast<const Pack<T, V> *>(tile + (size_t)k * rowb + r * sizeof(T));
#pragma unroll
                        for (int i = 0; i < V; ++i) acc[w].v[i] = scale * qv.v[i];
                    } else {
#pragma unroll
                        for (int i = 0; i < V; ++i) acc[w].v[i] = T(0);
                    }
                } else {
                    acc[w] = node_input<T, V, TR>(P, (int)a, node[q], rec, c, r);
                }
            }
#pragma unroll
            for (int e = 0; e < 3; ++e)
                if (e < cnt[q]) {
                    const T wt = S.ew[e0[q] + e];
#pragma unroll
                    for (int w = 0; w < W; ++w)
#pragma unroll
                        for (int i = 0; i < V; ++i) acc[w].v[i] += wt * xv[q][e][w].v[i];
                }
            for (int e = 3; e < cnt[q]; ++e) {
                const T wt = S.ew[e0[q] + e];
                const T *src = x + (long long)S.en[e0[q] + e] * P.ld_x + lo;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const Pack<T, V> t = load_l2<T, V>(src + w * ls);
#pragma unroll
                    for (int i = 0; i < V; ++i) acc[w].v[i] += wt * t.v[i];
                }
            }
#pragma unroll
            for (int w = 0; w < W; ++w) node_output<T, V, TR>(P, (int)a, node[q], p0 + k, rec, c, lo + w * ls, x, acc[w]);
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
template <typename T, int IM>
__device__ __forceinline__ void issue_structure(const TravParams &P, ItemStage<T, IM> &S)
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
template <typename T, bool TR, int IM>
__device__ __forceinline__ void issue_input(const TravParams &P, const ItemStage<T, IM> &S, unsigned char *tile)
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
template <typename T, int IM>
__device__ __forceinline__ void load_desc(const TravParams &P, ItemStage<T, IM> &S, int i)
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

template <typename T, int V, bool TR, int W = 0, int U = 1, int IM = ITEM_MAX>
__global__ void __launch_bounds__(256, (W * U >= 4) ? 2 : 4) k_traverse_persistent(TravParams P, int G, int tile_bytes)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ ItemStage<T, IM> stg[2];
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
        ItemStage<T, IM> &C = stg[b];
        ItemStage<T, IM> &Nx = stg[b ^ 1];
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
        if (it.z >= 0) {
            if (W > 0) run_stage_lanes<T, V, (W > 0 ? W : 1), U, TR>(P, C, tile_bytes ? dyn + b * (size_t)tile_bytes : nullptr, P.R / V);
            else run_stage_singletons<T, V, TR>(P, C, tile_bytes ? dyn + b * (size_t)tile_bytes : nullptr, G);
        }
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

// ---------------------------------------------------------------- cluster schedule
// One thread-block cluster of C CTAs owns one (tangent, source) unit at a time and walks
// its levels in order (reverse order for A^-T).  CTA r of the cluster takes the r-th of C
// contiguous slices of every level's positions (and every C-th SCC block of the level);
// after a level every CTA of the cluster meets at one hardware cluster barrier
// (barrier.cluster arrive.release / wait.acquire), which makes the level's stores visible
// to the whole cluster before the next level gathers them.  There is no flag and no
// ticket between levels, and clusters never wait for one another (each unit is a
// different source), so nothing can deadlock whether or not all clusters are resident.
// Per CTA the slices are cut into tiles of at most `tp` positions that run through a
// six-slot pipeline driven by one thread with 1-D bulk copies (cp.async.bulk, completion
// on an mbarrier per slot and stage):
//   iteration j issues the row offsets of tile j+5 and, once those have landed, the
//   structure of tile j+3 (nodes, receiver slots, C*M, upstream positions and weights);
//   every thread prefetches the input rows of tile j+1 into L2 and computes tile j.
// Each thread owns one (position, right-hand-side lane) pair per round and U positions
// per tile, and issues all loads of its U units (input row, up to three upstream rows)
// before any sum.  The structure and the inputs are never written by the traversal, so
// they are staged across level barriers; only the upstream rows wait for the barrier.
constexpr int CL_SLOTS = 6;
constexpr int CL_EDGE = 6;      // edge capacity per position in a slot (2 x ndim)
constexpr int CL_MAXTAN = 4;    // tangents per launch
constexpr int CL_PAD = 8;       // alignment slack (elements) around each staged array

struct ClusterBatch {
    TravParams P[CL_MAXTAN];
    int unit_ptr[CL_MAXTAN + 1];   // units of tangent k: [unit_ptr[k], unit_ptr[k+1])
    int ntan;
    int tp;                        // tile capacity (positions)
    int lanes[CL_MAXTAN];          // right-hand-side lanes (R / V) per tangent
    int tab;                       // capacity of the per-unit level tables (levels + 1)
    int *ticket;
};

// slot header; o_* are the element offsets of the first wanted element in each staged
// array (bulk copies start at the 16-byte granule below it)
struct ClHdr {
    int s, q0, np, ne;             // step (>= levels: empty), first position, positions, edges
    int o_rp, o_pos, o_cq, o_en, o_ew;
    int pad[3];
    unsigned long long barA;       // row offsets landed
    unsigned long long barB;       // structure landed
};

__device__ __forceinline__ unsigned cl_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cl_ncta()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_sync() { cl_arrive(); cl_wait(); }
// an int in the shared memory of CTA `rank` of this cluster
__device__ __forceinline__ int cl_load_remote(const int *p, unsigned rank)
{
    uint32_t a = smem_u32(p), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    int v;
    asm volatile("ld.shared::cluster.b32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
    return v;
}
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long *b)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
    return ok != 0;
}
// bounded wait for the phase with the given parity; on time-out the fault is latched and
// the caller carries on (the copy it waited for can only be late, not lost)
__device__ __forceinline__ void mbar_wait(unsigned long long *b, unsigned parity, const TravParams &P)
{
    if (mbar_try_wait(b, parity)) return;
    if (*(volatile int *)P.err != 0) return;    // an earlier wait already gave up
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(b, parity)) {
        if (global_ns() - t0 > P.timeout_ns) {
            if (atomicCAS(P.err, 0, DEV_TIMEOUT) == 0) { P.err[1] = -1; P.err[2] = -1; P.err[3] = -1; }
            return;
        }
    }
}
// 1-D bulk copy global -> this CTA's shared memory, completing on mbarrier b
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *b)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(b)) : "memory");
}

// Copy elements [i0, i1) of a global array into dst (16-byte aligned) starting at the
// granule that holds i0; returns the offset of element i0 in dst and adds the bytes.
template <typename E>
__device__ __forceinline__ int stage_range(E *dst, const E *src, long long i0, long long i1, unsigned long long *bar)
{
    constexpr int G = 16 / sizeof(E);
    const long long a0 = i0 / G * G, a1 = (i1 + G - 1) / G * G;
    if (a1 > a0) bulk_g2s(dst, src + a0, (unsigned)((a1 - a0) * sizeof(E)), bar);
    return (int)(i0 - a0);
}
template <typename E>
__device__ __forceinline__ unsigned range_bytes(long long i0, long long i1)
{
    constexpr int G = 16 / sizeof(E);
    return (unsigned)(((i1 + G - 1) / G * G - i0 / G * G) * sizeof(E));
}

// layout of one pipeline slot (tp positions, CL_EDGE * tp edges, CL_PAD slack per array)
template <typename T> struct ClSlot {
    ClHdr *h;
    int *rp, *perm, *rec, *en;
    T *cq, *ew;
};
__host__ __device__ __forceinline__ size_t cl_al16(size_t b) { return (b + 15) / 16 * 16; }
template <typename T>
__host__ __device__ __forceinline__ size_t cl_slot_bytes(int tp)
{
    size_t b = sizeof(ClHdr);
    b += cl_al16(sizeof(int) * (size_t)(tp + 1 + 2 * CL_PAD));    // rp
    b += 2 * cl_al16(sizeof(int) * (size_t)(tp + 2 * CL_PAD));    // perm, rec
    b += cl_al16(sizeof(int) * (size_t)(CL_EDGE * tp + 2 * CL_PAD));   // en
    b += cl_al16(sizeof(T) * (size_t)(tp + 2 * CL_PAD));          // cq
    b += cl_al16(sizeof(T) * (size_t)(CL_EDGE * tp + 2 * CL_PAD));     // ew
    return b;
}
template <typename T>
__device__ __forceinline__ ClSlot<T> cl_slot(unsigned char *base, int tp)
{
    ClSlot<T> v;
    v.h = reinterpret_cast<ClHdr *>(base);
    size_t o = sizeof(ClHdr);
    v.rp = reinterpret_cast<int *>(base + o);
    o += cl_al16(sizeof(int) * (size_t)(tp + 1 + 2 * CL_PAD));
    v.perm = reinterpret_cast<int *>(base + o);
    o += cl_al16(sizeof(int) * (size_t)(tp + 2 * CL_PAD));
    v.rec = reinterpret_cast<int *>(base + o);
    o += cl_al16(sizeof(int) * (size_t)(tp + 2 * CL_PAD));
    v.en = reinterpret_cast<int *>(base + o);
    o += cl_al16(sizeof(int) * (size_t)(CL_EDGE * tp + 2 * CL_PAD));
    v.cq = reinterpret_cast<T *>(base + o);
    o += cl_al16(sizeof(T) * (size_t)(tp + 2 * CL_PAD));
    v.ew = reinterpret_cast<T *>(base + o);
    return v;
}

// advance the tile cursor (s, q0, q1) of this CTA through its slices [sh0[s], sh1[s]) of
// the unit's steps; s = nl when there is no further tile
__device__ __forceinline__ void cl_next(const int *sh0, const int *sh1, int nl, int tp, int &s, int &q0, int &q1)
{
    if (s >= 0 && s < nl && q1 < sh1[s]) {
        q0 = q1;
        q1 = min(q0 + tp, sh1[s]);
        return;
    }
    for (++s; s < nl; ++s)
        if (sh1[s] > sh0[s]) {
            q0 = sh0[s];
            q1 = min(q0 + tp, sh1[s]);
            return;
        }
    s = nl;
    q0 = q1 = 0;
}

// thread 0, stage A of the next tile: header and its row offsets (rp[q0 .. q1])
template <typename T>
__device__ __forceinline__ void cl_stage_a(const TravParams &P, ClSlot<T> v, long long a, const int *sh0, const int *sh1,
                                           int nl, int tp, int &cs, int &cq0, int &cq1)
{
    cl_next(sh0, sh1, nl, tp, cs, cq0, cq1);
    v.h->s = cs;
    v.h->q0 = cq0;
    v.h->np = cq1 - cq0;
    if (cs >= nl) { mbar_arrive(&v.h->barA); return; }
    const long long i0 = a * (P.N + 1) + cq0, i1 = a * (P.N + 1) + cq1 + 1;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&v.h->barA, range_bytes<int>(i0, i1));
    v.h->o_rp = stage_range<int>(v.rp, P.rowptr, i0, i1, &v.h->barA);
}

// thread 0, stage B (row offsets visible): the structure of the tile
template <typename T>
__device__ __forceinline__ void cl_stage_b(const TravParams &P, ClSlot<T> v, long long a, long long ebase, int nl)
{
    if (v.h->s >= nl) { mbar_arrive(&v.h->barB); return; }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const int np = v.h->np;
    const int e0 = v.rp[v.h->o_rp], e1 = v.rp[v.h->o_rp + np];
    v.h->ne = e1 - e0;
    const long long p0 = a * P.N + v.h->q0, p1 = p0 + np;
    const long long g0 = ebase + e0, g1 = ebase + e1;
    const unsigned bytes = 2 * range_bytes<int>(p0, p1) + range_bytes<T>(p0, p1) + range_bytes<int>(g0, g1) +
                           range_bytes<T>(g0, g1);
    mbar_expect_tx(&v.h->barB, bytes);
    v.h->o_pos = stage_range<int>(v.perm, P.perm, p0, p1, &v.h->barB);
    stage_range<int>(v.rec, P.rec_slot, p0, p1, &v.h->barB);
    v.h->o_cq = stage_range<T>(v.cq, reinterpret_cast<const T *>(P.cq), p0, p1, &v.h->barB);
    v.h->o_en = stage_range<int>(v.en, P.enode, g0, g1, &v.h->barB);
    v.h->o_ew = stage_range<T>(v.ew, reinterpret_cast<const T *>(P.ew), g0, g1, &v.h->barB);
}

// Per-source base pointers of a traversal call, so that a unit's addresses are one 32-bit
// product and one add (every in-source offset is below 2^31: S N R < 2^31 per call).
template <typename T> struct ClBases {
    const T *in;     // input rows, indexed by node (forward, raw) or receiver slot (transpose, J)
    T *x;            // the transported field of the source, canonical order
    T *out;          // optional natural-order copy
    T *rec_out;      // forward J: d_rec rows of the source, by receiver slot
    T *g_out;        // transpose J without the source sum: g rows of the source, by node
    int ld_in, ld_x, ld_out, ld_aux;
    bool by_rec;     // input indexed by receiver slot (absent rows are zero)
    bool scale;      // multiply the input by C*M (forward J)
};

template <typename T, bool TR>
__device__ __forceinline__ ClBases<T> cl_bases(const TravParams &P, long long a)
{
    ClBases<T> b;
    const T *in = reinterpret_cast<const T *>(P.in);
    const bool J = P.mode == MODE_J;
    b.by_rec = TR && J;
    b.scale = !TR && J;
    if (b.by_rec) b.in = in + a * P.n_rec * P.ld_in;
    else b.in = in + ((!TR && J && P.shared_in) ? 0 : a * P.N * P.ld_in);
    b.x = reinterpret_cast<T *>(P.x) + a * P.N * P.ld_x;
    b.out = P.out ? reinterpret_cast<T *>(P.out) + a * P.N * P.ld_out : nullptr;
    T *aux = reinterpret_cast<T *>(P.aux);
    b.rec_out = (!TR && J && aux) ? aux + a * P.n_rec * P.ld_aux : nullptr;
    b.g_out = (TR && J && aux && !P.sum) ? aux + a * P.N * P.ld_aux : nullptr;
    b.ld_in = (int)P.ld_in;
    b.ld_x = (int)P.ld_x;
    b.ld_out = (int)P.ld_out;
    b.ld_aux = (int)P.ld_aux;
    return b;
}

// all threads: the input rows of the tile in slot v (structure visible) into L2
template <typename T>
__device__ __forceinline__ void cl_prefetch_input(const ClBases<T> &B, ClSlot<T> v, int nl, int rowb)
{
    if (v.h->s >= nl) return;
    const int np = v.h->np, op = v.h->o_pos;
    const int lines = (rowb + 127) >> 7;
    for (int q = threadIdx.x; q < np * lines; q += blockDim.x) {
        const int k = q / lines, c = q - k * lines;
        const int row = B.by_rec ? v.rec[op + k] : v.perm[op + k];
        if (row >= 0 && v.perm[op + k] >= 0)
            prefetch_l2(reinterpret_cast<const unsigned char *>(B.in + (unsigned)(row * B.ld_in)) + c * 128);
    }
}

// all threads: the tile in slot v.  A position's lanes (V-element vectors of right-hand
// sides) are split over G = lanes / W threads; thread (k0, g) handles lanes g, g + G, ...,
// g + (W-1) G of positions k0 + q * kstep, q < U = 4 / W.  The row of a position is
// decoded once per thread and shared by its W lanes, and every load of the thread (input
// rows, up to three upstream rows) is issued before any sum.
template <typename T, int V, int W, bool TR>
__device__ __forceinline__ void cl_compute(const ClBases<T> &B, ClSlot<T> v, int k0, int g, int kstep, int G)
{
    constexpr int U = 4 / W;
    const int np = v.h->np, p0 = v.h->q0;
    const int orp = v.h->o_rp, op = v.h->o_pos, ocq = v.h->o_cq, oen = v.h->o_en, oew = v.h->o_ew;
    const int ebx = v.rp[orp];
    const int lo = g * V, ls = G * V;      // element offset of the first lane, lane stride
    Pack<T, V> in[U][W], up[U][3][W];
    int node[U], e0[U], cnt[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
        const int k = k0 + q * kstep;
        node[q] = k < np ? v.perm[op + k] : -1;
        cnt[q] = 0;
        e0[q] = 0;
        if (node[q] < 0) continue;
        const int r0 = v.rp[orp + k];
        e0[q] = r0 - ebx;
        cnt[q] = v.rp[orp + k + 1] - r0;
        const int row = B.by_rec ? v.rec[op + k] : node[q];
        if (row >= 0) {
            const T *src = B.in + (unsigned)(row * B.ld_in + lo);
#pragma unroll
            for (int w = 0; w < W; ++w) in[q][w] = load_l2<T, V>(src + w * ls);
        } else {
#pragma unroll
            for (int w = 0; w < W; ++w)
#pragma unroll
                for (int i = 0; i < V; ++i) in[q][w].v[i] = T(0);
        }
#pragma unroll
        for (int e = 0; e < 3; ++e)
            if (e < cnt[q]) {
                const T *src = B.x + (unsigned)(v.en[oen + e0[q] + e] * B.ld_x + lo);
#pragma unroll
                for (int w = 0; w < W; ++w) up[q][e][w] = load_l2<T, V>(src + w * ls);
            }
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
        if (node[q] < 0) continue;
        const int k = k0 + q * kstep;
        const T c = v.cq[ocq + k];
        const T scale = B.scale ? c : T(1);
        Pack<T, V> acc[W];
#pragma unroll
        for (int w = 0; w < W; ++w)
#pragma unroll
            for (int i = 0; i < V; ++i) acc[w].v[i] = scale * in[q][w].v[i];
#pragma unroll
        for (int e = 0; e < 3; ++e)
            if (e < cnt[q]) {
                const T wt = v.ew[oew + e0[q] + e];
#pragma unroll
                for (int w = 0; w < W; ++w)
#pragma unroll
                    for (int i = 0; i < V; ++i) acc[w].v[i] += wt * up[q][e][w].v[i];
            }
        for (int e = 3; e < cnt[q]; ++e) {
            const T wt = v.ew[oew + e0[q] + e];
            const T *src = B.x + (unsigned)(v.en[oen + e0[q] + e] * B.ld_x + lo);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const Pack<T, V> xv = load_l2<T, V>(src + w * ls);
#pragma unroll
                for (int i = 0; i < V; ++i) acc[w].v[i] += wt * xv.v[i];
            }
        }
        T *dst = B.x + (unsigned)((p0 + k) * B.ld_x + lo);
#pragma unroll
        for (int w = 0; w < W; ++w) store<T, V>(dst + w * ls, acc[w]);
        if (B.out) {
            T *o = B.out + (unsigned)(node[q] * B.ld_out + lo);
#pragma unroll
            for (int w = 0; w < W; ++w) store<T, V>(o + w * ls, acc[w]);
        }
        if (B.rec_out) {
            const int rs = v.rec[op + k];
            if (rs >= 0) {
                T *o = B.rec_out + (unsigned)(rs * B.ld_aux + lo);
#pragma unroll
                for (int w = 0; w < W; ++w) store<T, V>(o + w * ls, acc[w]);
            }
        } else if (B.g_out) {
            T *o = B.g_out + (unsigned)(node[q] * B.ld_aux + lo);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                Pack<T, V> gv;
#pragma unroll
                for (int i = 0; i < V; ++i) gv.v[i] = c * acc[w].v[i];
                store<T, V>(o + w * ls, gv);
            }
        }
    }
}

// SCC blocks are rare; kept out of line so their registers do not weigh on the tile loop
template <typename T, bool TR>
__device__ __noinline__ void cl_block(const TravParams &P, int a, int b)
{
    run_block<T, TR>(P, a, b);
}

template <typename T, int V, bool TR, int W>
__global__ void __launch_bounds__(256, 2) k_traverse_cluster(const __grid_constant__ ClusterBatch B)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ int s_unit;
    __shared__ TravParams sP;
    const unsigned C = cl_ncta(), rank = cl_rank();
    const int tid = threadIdx.x;
    const int tp = B.tp;
    const size_t sb = cl_slot_bytes<T>(tp);
    int *sh0 = reinterpret_cast<int *>(dyn + CL_SLOTS * sb);   // this CTA's slice of every step
    int *sh1 = sh0 + B.tab;
    int *tab_blk = sh1 + B.tab;                                  // first block of every level
    auto slot = [&](int j) { return cl_slot<T>(dyn + (size_t)(j % CL_SLOTS) * sb, tp); };
    if (tid == 0)
        for (int q = 0; q < CL_SLOTS; ++q) {
            ClSlot<T> v = slot(q);
            mbar_init(&v.h->barA, 1);
            mbar_init(&v.h->barB, 1);
        }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    int uses = 0;   // tiles run through the slots so far (mbarrier phases)
    for (;;) {
        if (rank == 0 && tid == 0) s_unit = atomicAdd(B.ticket, 1);
        cl_sync();
        const int u = cl_load_remote(&s_unit, 0);
        cl_sync();                       // every CTA has read the ticket before rank 0 takes the next
        if (u >= B.unit_ptr[B.ntan]) break;
        int k = 0;
        while (u >= B.unit_ptr[k + 1]) ++k;
        {
            const int *src = reinterpret_cast<const int *>(&B.P[k]);
            int *dst = reinterpret_cast<int *>(&sP);
            for (int i = tid; i < (int)(sizeof(TravParams) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        const TravParams &P = sP;
        const int lanes = B.lanes[k];
        const long long a = __ldg(P.order + (u - B.unit_ptr[k]));
        const int nl = __ldg(P.nlev + a);
        const long long ebase = __ldg(P.ebase + a);
        {
            const int *lvl = P.lvl + a * (P.maxL + 1);
            for (int i = tid; i <= nl; i += blockDim.x) {
                tab_blk[i] = __ldg(P.blk_lvl + a * (P.maxL + 1) + i);
                if (i < nl) {
                    const int L = TR ? nl - 1 - i : i;
                    const int lo = __ldg(lvl + L), n = __ldg(lvl + L + 1) - lo;
                    sh0[i] = lo + n * (int)rank / (int)C;          // n * 16 < 2^31: int arithmetic
                    sh1[i] = lo + n * ((int)rank + 1) / (int)C;
                }
            }
        }
        // this thread's (position, lane group) and the tile size
        const int G = lanes / W;
        const int kstep = blockDim.x / G;
        const int k0 = tid / G, g = tid - k0 * G;
        const int tpu = min(tp, (4 / W) * kstep);
        const ClBases<T> bases = cl_bases<T, TR>(P, a);
        const int rowb = P.R * (int)sizeof(T);
        __syncthreads();
        // pipeline over this CTA's tiles; tile j uses slot (uses + j) % CL_SLOTS, and the
        // n-th use of a slot waits for mbarrier phase parity n & 1
        auto sl = [&](int j) { return slot(uses + j); };
        auto par = [&](int j) { return (unsigned)(((uses + j) / CL_SLOTS) & 1); };
        int cs = -1, cq0 = 0, cq1 = 0;     // tile cursor (thread 0)
        // prologue: row offsets of tiles 0..4, structure of tiles 0..2; visible before
        // iteration 0: the structure of tiles 0, 1 and the row offsets of tiles 0..3
        if (tid == 0) {
            for (int q = 0; q < 5; ++q) cl_stage_a<T>(P, sl(q), a, sh0, sh1, nl, tpu, cs, cq0, cq1);
            for (int q = 0; q < 3; ++q) {
                mbar_wait(&sl(q).h->barA, par(q), P);
                cl_stage_b<T>(P, sl(q), a, ebase, nl);
            }
            for (int q = 0; q < 2; ++q) mbar_wait(&sl(q).h->barB, par(q), P);
            mbar_wait(&sl(3).h->barA, par(3), P);
        }
        __syncthreads();
        cl_prefetch_input<T>(bases, sl(0), nl, rowb);
        int j = 0;
        for (int s = 0; s < nl; ++s) {
            for (;;) {
                ClSlot<T> cur = sl(j);
                if (cur.h->s != s) break;
                // visible here: the structure of tiles j, j+1 and the row offsets of tiles
                // up to j+3 (stage B of tile j+2 and stage A of tile j+4 were issued one
                // iteration ago)
                cl_prefetch_input<T>(bases, sl(j + 1), nl, rowb);
                if (tid == 0) {
                    cl_stage_b<T>(P, sl(j + 3), a, ebase, nl);
                    cl_stage_a<T>(P, sl(j + 5), a, sh0, sh1, nl, tpu, cs, cq0, cq1);
                }
                if (k0 < kstep) cl_compute<T, V, W, TR>(bases, cur, k0, g, kstep, G);
                if (tid == 0) {
                    mbar_wait(&sl(j + 2).h->barB, par(j + 2), P);
                    mbar_wait(&sl(j + 4).h->barA, par(j + 4), P);
                }
                __syncthreads();             // staged data visible; slot j is free
                ++j;
            }
            const int L = TR ? nl - 1 - s : s;
            for (int b = tab_blk[L] + (int)rank; b < tab_blk[L + 1]; b += C) cl_block<T, TR>(P, (int)a, b);
            cl_sync();
        }
        // tile indices j .. j+4 are empty: stage A has arrived on all of them, stage B on
        // j .. j+2; arrive stage B of the last two so that every index used each of its
        // slot's barriers exactly once, then advance the slots past them
        if (tid == 0) {
            cl_stage_b<T>(P, sl(j + 3), a, ebase, nl);
            cl_stage_b<T>(P, sl(j + 4), a, ebase, nl);
        }
        uses += j + 5;
        __syncthreads();
    }
    if (tid == 0)
        for (int q = 0; q < CL_SLOTS; ++q) {
            ClSlot<T> v = slot(q);
            mbar_inval(&v.h->barA);
            mbar_inval(&v.h->barB);
        }
}

// ---------------------------------------------------------------- multi-slot persistent schedule
// The persistent schedule with NS work items held by each CTA at once.  Every held item's
// structure and dependency list is copied into its own shared-memory slot with cp.async,
// and each thread's copies signal the slot's mbarrier (cp.async.mbarrier.arrive), so warp 0
// can see without waiting which slots have landed.  Warp 0 then polls the dependencies of
// every landed item in one round (one flag per lane) and hands the CTA the lowest-ticket
// item that is ready; a CTA that waited on one item in the single-slot schedule now
// computes another.  The computed slot takes the next ticket (taken during the compute)
// and its copies are issued behind it.  Progress: the lowest unfinished ticket has all
// its upstream items (lower tickets) done and its copies land unconditionally, so its
// CTA, which re-polls every held slot each round, picks it in bounded time.  Input rows
// are read in place (no tile) and prefetched into L2 once the slot's structure is in.
__device__ __forceinline__ void cp_async_mbar_arrive(unsigned long long *b)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *b, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
    return ok != 0;
}

// input rows of a landed slot into L2 (lanes of warp 0)
template <typename T, bool TR, int IM>
__device__ __forceinline__ void prefetch_inputs(const TravParams &P, const ItemStage<T, IM> &S, int lane)
{
    if (S.it.z < 0) return;
    const int np = S.it.w - S.it.z;
    const int rowb = P.R * (int)sizeof(T);
    for (int k = lane; k < np; k += 32) {
        const int v = S.perm[k];
        if (v < 0) continue;
        const T *src = input_row<T, TR>(P, S.it.x, v, S.rec[k]);
        if (src)
            for (int o = 0; o < rowb; o += 128) prefetch_l2(reinterpret_cast<const char *>(src) + o);
    }
}

// The tangents of one launch: one (the single-tangent call) or up to CL_MAXTAN (batched
// applies over several grids).  Tickets run over the items of all of them in a merged
// step-major order (step s of every tangent before step s + 1 of any), so an item's
// upstream items still have lower tickets.
struct MultiBatch {
    TravParams P[CL_MAXTAN];
    int G[CL_MAXTAN];            // lanes per position of each tangent
    int ntan;
    int nitems;                  // tickets: items of all the tangents
    const int2 *order;           // ticket -> {tangent, item}; nullptr: one tangent, ticket = item
    int *ticket;
};

// descriptor of ticket t into slot S (one thread)
template <typename T, int IM>
__device__ __forceinline__ void load_desc_multi(const MultiBatch &B, ItemStage<T, IM> &S, int t)
{
    S.tkt = t;
    S.nd = -1;
    if (t >= B.nitems) return;
    int k = 0, i = t;
    if (B.order) {
        const int2 o = B.order[t];
        k = o.x;
        i = o.y;
    }
    const TravParams &P = B.P[k];
    S.tan = k;
    S.idx = i;
    S.it = P.items[i];
    const int2 eb = P.ebeg[i];
    S.ebx = eb.x;
    S.eby = eb.y;
}

template <typename T, int V, bool TR, int NS, bool MT, int IM = ITEM_MAX>
__global__ void __launch_bounds__(256, 4) k_traverse_multi(const __grid_constant__ MultiBatch B)
{
    // MT: several tangents (slot k's item belongs to tangent stg[k].tan); else tangent 0
#define EIK_TAN(S) (MT ? (S).tan : 0)
    __shared__ ItemStage<T, IM> stg[NS];
    __shared__ __align__(8) unsigned long long bar[NS];
    __shared__ int s_pick, s_t;
    const int tid = threadIdx.x;
    const int ntk = B.nitems;
    const unsigned FULL = 0xffffffffu;
    unsigned ph = 0;                 // bit k: parity of the phase slot k's current copies complete
    unsigned hinted = 0;             // warp 0: bit k set once slot k's input rows were prefetched
    if (tid == 0) {
        for (int k = 0; k < NS; ++k) mbar_init(&bar[k], blockDim.x);
        for (int k = 0; k < NS; ++k) load_desc_multi(B, stg[k], atomicAdd(B.ticket, 1));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        if (stg[k].tkt < ntk) issue_structure<T>(B.P[EIK_TAN(stg[k])], stg[k]);
        cp_async_mbar_arrive(&bar[k]);
    }
    for (;;) {
        // ---- warp 0: the lowest-ticket held item whose copies landed and whose upstream
        // items are done (-1: nothing held, or a fault)
        if (tid < 32) {
            int pick = -1;
            const unsigned long long t0 = global_ns();
            for (int round = 0;; ++round) {
                unsigned held = 0, landed = 0;
#pragma unroll
                for (int k = 0; k < NS; ++k)
                    if (stg[k].tkt < ntk) {
                        held |= 1u << k;
                        if (mbar_test(&bar[k], (ph >> k) & 1)) landed |= 1u << k;
                    }
                if (!held) break;
                // one dependency flag per lane: slots in order, each its list (or its level counter)
                unsigned bad = 0;
                int base = 0;                           // pair index of slot k's first flag
#pragma unroll
                for (int k = 0; k < NS; ++k) {
                    if (!((landed >> k) & 1)) continue;
                    const ItemStage<T, IM> &S = stg[k];
                    if (S.it.y == 0) continue;          // first step: nothing upstream
                    const TravParams &P = B.P[EIK_TAN(S)];
                    const int nd = S.nd;
                    const int cnt = nd < 0 ? 1 : nd;
                    for (int j = ((tid - base) % 32 + 32) % 32; j < cnt; j += 32) {
                        bool ok;
                        if (nd < 0) {
                            const long long c = (long long)S.it.x * P.maxL + S.it.y - 1;
                            ok = ld_acquire(P.done + c) >= P.item_cnt[c];
                        } else {
                            ok = ld_acquire(P.item_done + S.deps[j]) >= 1;
                        }
                        if (!ok) bad |= 1u << k;
                    }
                    base += cnt;
                }
                bad = __reduce_or_sync(FULL, bad);
                const unsigned ready = landed & ~bad;
                if (ready) {
                    int best = -1;
#pragma unroll
                    for (int k = 0; k < NS; ++k)
                        if (((ready >> k) & 1) && (best < 0 || stg[k].tkt < stg[best].tkt)) best = k;
                    pick = best;
                    break;
                }
                // slots whose structure landed: their input rows into L2 while waiting
                const unsigned fresh = landed & ~hinted;
#pragma unroll
                for (int k = 0; k < NS; ++k)
                    if ((fresh >> k) & 1) prefetch_inputs<T, TR, IM>(B.P[EIK_TAN(stg[k])], stg[k], tid);
                hinted |= fresh;
                int stop = 0;
                if (tid == 0 && (round & 15) == 15) {
                    if (*(volatile int *)B.P[0].err != 0) stop = 1;
                    else if (global_ns() - t0 > B.P[0].timeout_ns) {
                        if (atomicCAS(B.P[0].err, 0, DEV_TIMEOUT) == 0) { B.P[0].err[1] = -1; B.P[0].err[2] = -1; B.P[0].err[3] = -1; }
                        stop = 1;
                    }
                }
                if (__shfl_sync(FULL, stop, 0)) break;
                __nanosleep(32);
            }
            if (tid == 0) s_pick = pick;
        }
        __syncthreads();             // (A) the picked item's upstream rows are complete
        const int b = s_pick;
        if (b < 0) break;
        ItemStage<T, IM> &C = stg[b];
        const int kt = EIK_TAN(C);
        const TravParams &P = B.P[kt];
        const int4 it = C.it;
        const int i = C.idx;
        if (tid == 1) s_t = atomicAdd(B.ticket, 1);
        if (it.z >= 0) run_stage_singletons<T, V, TR>(P, C, nullptr, B.G[kt]);
        else run_block<T, TR>(P, it.x, ~it.z);
        __syncthreads();             // (B) every row of the item written
        if (tid == 32) {
            fence_acq_rel_gpu();
            atomicAdd(P.done + (long long)it.x * P.maxL + it.y, 1);
            st_relaxed(P.item_done + i, 1);
        }
        if (tid == 1) load_desc_multi(B, C, s_t);
        ph ^= 1u << b;
        hinted &= ~(1u << b);
        __syncthreads();             // (C) the slot's next descriptor visible
        if (C.tkt < ntk) issue_structure<T>(B.P[EIK_TAN(C)], C);
        cp_async_mbar_arrive(&bar[b]);
    }
    cp_async_wait<0>();              // copies of slots never computed land before the CTA exits
#undef EIK_TAN
}

// g[j][r] = sum_a cq_a[j] lam_a[j][r] in source order.  FP64 path: FP64 products and
// sum.  FP32 path: FP32 products with a compensated (Kahan) FP32 sum, so the rounding
// error does not grow with the number of sources (B300's FP64 rate would make an FP64
// accumulation the bottleneck of this pass).  Loads are issued SUMB at a time.
constexpr int SUMB = 8;

template <typename T>
__global__ void k_source_sum(long long N, int S, int R, const T *__restrict__ cqn, const int *__restrict__ pos,
                             const T *__restrict__ lam, long long ld_lam, T *__restrict__ g, long long ld_g, int accumulate)
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
    g[j * ld_g + r] = accumulate ? g[j * ld_g + r] + acc : acc;
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
                                                        long long ld_g, int accumulate)
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
    if (j < N) {
        if (accumulate) {
            const Pack<T, V> old = load_ro<T, V>(g + j * ld_g + r);
#pragma unroll
            for (int u = 0; u < V; ++u) acc.v[u] = old.v[u] + acc.v[u];
        }
        store<T, V>(g + j * ld_g + r, acc);
    }
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
int ensure_workspace(Tangent *t, size_t vec_bytes, size_t blk_elems, bool TR)
{
    const bool own = split_lane(t, TR);
    void *&vec = own ? t->lane_t.ws_vec : t->ws_vec;
    size_t &vec_n = own ? t->lane_t.ws_vec_bytes : t->ws_vec_bytes;
    double *&blk = own ? t->lane_t.ws_blk : t->ws_blk;
    size_t &blk_n = own ? t->lane_t.ws_blk_elems : t->ws_blk_elems;
    if (vec_bytes > vec_n) {
        if (vec) cudaFree(vec);
        vec = nullptr;
        vec_n = 0;
        EIK_CHECK(cudaMalloc(&vec, vec_bytes));
        vec_n = vec_bytes;
    }
    if (blk_elems > blk_n) {
        if (blk) cudaFree(blk);
        blk = nullptr;
        blk_n = 0;
        EIK_CHECK(cudaMalloc(&blk, blk_elems * sizeof(double)));
        blk_n = blk_elems;
    }
    return EIK_OK;
}

int enable_split(Tangent *t)
{
    if (t->lane_t.ticket) return EIK_OK;
    Lane &L = t->lane_t;
    EIK_CHECK(cudaMalloc(&L.item_done, (size_t)std::max(t->nitems, 1) * sizeof(int) + 64));
    EIK_CHECK(cudaMalloc(&L.done, (size_t)t->S * std::max(t->maxL, 1) * sizeof(int) + 64));
    EIK_CHECK(cudaMalloc(&L.ticket, 4 * sizeof(int) + 64));
    EIK_CHECK(cudaMemset(L.ticket, 0, 4 * sizeof(int)));
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

template <typename T, int V, bool TR, int W>
static int launch_cluster_u(Tangent *t, ClusterBatch &B, int units, cudaStream_t st)
{
    auto kern = k_traverse_cluster<T, V, TR, W>;
    const int threads = t->opts.cluster_threads > 0 ? t->opts.cluster_threads : 256;
    const size_t dyn = CL_SLOTS * cl_slot_bytes<T>(B.tp) + 3 * (size_t)B.tab * sizeof(int);
    if (dyn > 200 * 1024) { set_error("cluster schedule: %zu bytes of shared memory needed", dyn); return EIK_ERR_INVALID; }
    EIK_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    EIK_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // active clusters of size c (cached per launch shape)
    auto fit = [&](int c, int *n) -> int {
        const long long key = ((long long)TR << 62) | ((long long)sizeof(T) << 56) | ((long long)V << 52) |
                              ((long long)W << 48) | ((long long)threads << 36) | ((long long)dyn << 8) | c;
        auto it = t->cluster_fit.find(key);
        if (it != t->cluster_fit.end()) { *n = it->second; return EIK_OK; }
        at[0].val.clusterDim.x = (unsigned)c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)c);
        int m = 0;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&m, kern, &cfg);
        if (e != cudaSuccess) { cudaGetLastError(); m = 0; }
        t->cluster_fit[key] = m;
        *n = m;
        return EIK_OK;
    };
    int C = t->opts.cluster_size, nact = 0;
    if (C > 0) {
        fit(C, &nact);
    } else {
        // the largest cluster that keeps every unit resident at once, else the size with the
        // most CTAs in flight
        static const int sizes[] = {16, 12, 8, 6, 4, 2, 1};
        int best = 1, best_ctas = -1;
        for (int c : sizes) {
            int m = 0;
            fit(c, &m);
            if (m >= units) { C = c; nact = m; break; }
            if (m * c > best_ctas) { best_ctas = m * c; best = c; nact = m; }
        }
        if (C <= 0) C = best;
    }
    if (nact <= 0) { set_error("cluster schedule: no cluster of %d CTAs x %d threads fits", C, threads); return EIK_ERR_INVALID; }
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(std::min(units, nact) * C));
    EIK_CHECK(cudaMemsetAsync(B.ticket, 0, sizeof(int), st));
    EIK_CHECK(cudaLaunchKernelEx(&cfg, kern, B));
    return EIK_OK;
}

template <typename T, int V, bool TR>
static int launch_cluster(Tangent *t, const TravParams &P, cudaStream_t st)
{
    if (t->opts.cluster_threads != 0 &&
        (t->opts.cluster_threads < 64 || t->opts.cluster_threads > 256 || t->opts.cluster_threads % 32)) {
        set_error("cluster_threads must be a multiple of 32 in 64..256");
        return EIK_ERR_INVALID;
    }
    if (t->opts.cluster_size < 0 || t->opts.cluster_size > 16) { set_error("cluster_size must be 0..16"); return EIK_ERR_INVALID; }
    ClusterBatch B{};
    B.P[0] = P;
    B.ntan = 1;
    B.unit_ptr[0] = 0;
    B.unit_ptr[1] = t->S;
    B.lanes[0] = P.R / V;
    const int threads = t->opts.cluster_threads > 0 ? t->opts.cluster_threads : 256;
    if (B.lanes[0] > threads) {
        set_error("cluster schedule: %d right-hand-side lanes exceed %d threads per CTA; set rhs_chunk", B.lanes[0], threads);
        return EIK_ERR_INVALID;
    }
    // lanes per thread: the widest of 4, 2, 1 that divides the lanes (pass_units caps it)
    const int cap = t->opts.pass_units > 0 ? t->opts.pass_units : 4;
    int W = 1;
    if (cap >= 4 && B.lanes[0] % 4 == 0) W = 4;
    else if (cap >= 2 && B.lanes[0] % 2 == 0) W = 2;
    B.tp = std::min(512, (4 / W) * (threads / (B.lanes[0] / W)));
    B.tab = t->maxL + 1;
    // keep the six slots and the level tables within 160 KB of shared memory
    while (B.tp > 32 && CL_SLOTS * cl_slot_bytes<T>(B.tp) + 3 * (size_t)B.tab * sizeof(int) > 160 * 1024) B.tp /= 2;
    B.ticket = P.ticket + 1;
    if (W == 4) return launch_cluster_u<T, V, TR, 4>(t, B, t->S, st);
    if (W == 2) return launch_cluster_u<T, V, TR, 2>(t, B, t->S, st);
    return launch_cluster_u<T, V, TR, 1>(t, B, t->S, st);
}

template <typename T, int V, bool TR>
static int launch_traverse(Tangent *t, TravParams &P, int G, cudaStream_t st)
{
    if (t->opts.schedule == EIK_SCHED_CLUSTER) return launch_cluster<T, V, TR>(t, P, st);
    if (t->opts.schedule == EIK_SCHED_SYNC) return launch_sync(t, P, (int)sizeof(T), V, TR, st);
    if (t->item_max > ITEM_MAX && t->opts.schedule != EIK_SCHED_PERSISTENT) {
        set_error("items of %d positions run in the persistent or cluster schedule only (build with chunk <= %d)",
                  t->item_max, ITEM_MAX);
        return EIK_ERR_INVALID;
    }
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
    // compute form: one vector per thread (default), or lane groups of W = pass_units vectors
    // per thread when W divides the lanes (measured slower on the 3-D apply workload: the
    // item is bound by dependent-instruction and memory latency, not by instruction count)
    const int lanes = P.R / V;
    const int want = t->opts.pass_units > 0 ? t->opts.pass_units : 1;
    if (t->opts.item_slots >= 2 && want <= 1) {
        // several items held per CTA (input rows read in place, prefetched into L2); items of
        // more than 64 positions (few right-hand sides) take two slots of the large capacity
        void (*mk)(MultiBatch) = t->item_max > ITEM_MAX ? k_traverse_multi<T, V, TR, 2, false, ITEM_CAP>
                                 : t->opts.item_slots >= 4 ? k_traverse_multi<T, V, TR, 4, false>
                                 : t->opts.item_slots == 3 ? k_traverse_multi<T, V, TR, 3, false>
                                                           : k_traverse_multi<T, V, TR, 2, false>;
        MultiBatch B{};
        B.P[0] = P;
        B.G[0] = G;
        B.ntan = 1;
        B.nitems = P.nitems;
        B.order = nullptr;
        B.ticket = P.ticket;
        int per_sm = t->opts.ctas_per_sm;
        if (per_sm <= 0) {
            EIK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mk, threads, 0));
            per_sm = std::max(per_sm, 1);
        }
        long long grid = std::min<long long>((long long)t->num_sms * per_sm, P.nitems);
        grid = std::max<long long>(grid, 1);
        EIK_CHECK(cudaMemsetAsync(P.done, 0, (size_t)t->S * t->maxL * sizeof(int), st));
        EIK_CHECK(cudaMemsetAsync(P.ticket, 0, sizeof(int), st));
        EIK_CHECK(cudaMemsetAsync(P.item_done, 0, (size_t)std::max(P.nitems, 1) * sizeof(int), st));
        mk<<<(unsigned)grid, threads, 0, st>>>(B);
        EIK_CHECK_LAUNCH();
        return EIK_OK;
    }
    void (*kern)(TravParams, int, int) = k_traverse_persistent<T, V, TR>;
    if (t->item_max > ITEM_MAX) kern = k_traverse_persistent<T, V, TR, 0, 1, ITEM_CAP>;   // large items (R small)
    else if (want >= 4 && lanes % 4 == 0 && lanes / 4 <= threads) kern = k_traverse_persistent<T, V, TR, 4, 1>;
    else if (want >= 2 && lanes % 2 == 0 && lanes / 2 <= threads) kern = k_traverse_persistent<T, V, TR, 2, 1>;
    EIK_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int per_sm = t->opts.ctas_per_sm;
    if (per_sm <= 0) {
        EIK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, dyn));
        per_sm = std::max(per_sm, 1);
    }
    long long grid = std::min<long long>((long long)t->num_sms * per_sm, P.nitems);
    grid = std::max<long long>(grid, 1);
    EIK_CHECK(cudaMemsetAsync(P.done, 0, (size_t)t->S * t->maxL * sizeof(int), st));
    EIK_CHECK(cudaMemsetAsync(P.ticket, 0, sizeof(int), st));
    EIK_CHECK(cudaMemsetAsync(P.item_done, 0, (size_t)std::max(P.nitems, 1) * sizeof(int), st));
    kern<<<(unsigned)grid, threads, dyn, st>>>(P, G, tile_bytes);
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
int source_sum(Tangent *t, int w, void *g, long long ld_g, int dtype, cudaStream_t st, bool accumulate)
{
    NvtxRange range("source sum");
    const int acc = accumulate ? 1 : 0;
    const void *xp = lane_ws(t, true);    // the reverse field of the last transpose traversal
    const int V = dtype == EIK_F32 ? 4 : 2;
    const int L = w / V;
    if (w % V == 0 && ld_g % V == 0 && aligned16(xp) && aligned16(g) && L <= 256) {
        const int rows = std::min(SUM_ROWS, std::max(1, 256 / L));
        const unsigned blocks = (unsigned)((t->N + rows - 1) / rows);
        if (dtype == EIK_F32)
            k_source_sum_vec<float, 4><<<blocks, rows * L, 0, st>>>(t->N, t->S, w, rows, t->cqn32, t->pos,
                                                                    (const float *)xp, (long long)w, (float *)g, ld_g, acc);
        else
            k_source_sum_vec<double, 2><<<blocks, rows * L, 0, st>>>(t->N, t->S, w, rows, t->cqn64, t->pos,
                                                                     (const double *)xp, (long long)w, (double *)g, ld_g, acc);
    } else {
        const long long n = t->N * w;
        const unsigned blocks = (unsigned)((n + 255) / 256);
        if (dtype == EIK_F32)
            k_source_sum<float><<<blocks, 256, 0, st>>>(t->N, t->S, w, t->cqn32, t->pos, (const float *)xp, (long long)w,
                                                        (float *)g, ld_g, acc);
        else
            k_source_sum<double><<<blocks, 256, 0, st>>>(t->N, t->S, w, t->cqn64, t->pos, (const double *)xp, (long long)w,
                                                         (double *)g, ld_g, acc);
    }
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

// launch parameters of one traversal call (a column chunk of w right-hand sides starting
// at the given input/output pointers; row strides R)
static TravParams make_params(Tangent *t, bool TR, int mode, const void *inp, int shared_in, int w, int R, void *xp,
                              void *outp, void *auxp, int sum_sources, int dtype)
{
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
    const bool own = split_lane(t, TR);
    P.done = own ? t->lane_t.done : t->done;
    P.ticket = own ? t->lane_t.ticket : t->ticket;
    P.err = t->err;
    P.deps = TR ? t->deps_bwd : t->deps_fwd;
    // while a test hold is in place every item takes the level wait it targets
    P.ndeps = t->opts.item_deps && t->holds.empty() ? (TR ? t->ndeps_bwd : t->ndeps_fwd) : nullptr;
    P.item_done = own ? t->lane_t.item_done : t->item_done;
    P.blk_desc = t->blk_desc; P.blk_off = t->blk_off; P.binv = t->binv; P.ws = own ? t->lane_t.ws_blk : t->ws_blk;
    P.lu = t->lu; P.piv = t->piv; P.blk_lu_min = t->opts.block_lu_min;
    P.timeout_ns = (unsigned long long)(t->opts.wait_timeout_s * 1e9);
    P.lvl = t->lvl_d; P.blk_lvl = t->blk_lvl_d; P.nlev = t->nlev_d; P.order = t->order_d;
    return P;
}

int traverse(Tangent *t, bool TR, int mode, const void *in, int shared_in, int R, void *out_full, void *out_aux,
             int sum_sources, int dtype, cudaStream_t st)
{
    NvtxRange range(TR ? (mode == MODE_J ? "J^T traversal" : "A^-T solve") : (mode == MODE_J ? "J traversal" : "A^-1 solve"));
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
    int rc = ensure_workspace(t, need_vec, (size_t)t->ws_rows * Rc, TR);
    if (rc) return rc;
    for (int r0 = 0; r0 < R; r0 += Rc) {
        const int w = std::min(Rc, R - r0);
        const char *inp = static_cast<const char *>(in) + r0 * esz;
        char *xp = static_cast<char *>(lane_ws(t, TR));
        char *outp = out_full ? static_cast<char *>(out_full) + r0 * esz : nullptr;
        char *auxp = out_aux ? static_cast<char *>(out_aux) + r0 * esz : nullptr;
        TravParams P = make_params(t, TR, mode, inp, shared_in, w, R, xp, outp, auxp, sum_sources, dtype);
        if (dtype == EIK_F32) rc = TR ? dispatch_v<float, true>(t, P, st) : dispatch_v<float, false>(t, P, st);
        else rc = TR ? dispatch_v<double, true>(t, P, st) : dispatch_v<double, false>(t, P, st);
        if (rc) return rc;
        if (!TR && mode == MODE_J && t->pts.K > 0) {
            // point sources: the seed rows' share sigma_a z_a (linear in the model input)
            rc = seed_sigma(t, inp, shared_in, (long long)R, w, dtype, st);
            if (!rc && auxp && t->n_rec > 0) rc = seed_add(t, t->n_rec, w, t->pts.zrec, auxp, (long long)R, dtype, st);
            if (!rc && outp) rc = seed_add(t, t->N, w, t->pts.z, outp, (long long)R, dtype, st);
            if (rc) return rc;
        }
        if (TR && mode == MODE_J && sum_sources && out_aux) {
            rc = source_sum(t, w, auxp, (long long)R, dtype, st, sum_sources == 2);
            if (rc) return rc;
        }
        if (TR && mode == MODE_J && t->pts.K > 0 && out_aux) {
            // point sources: M^T Phi^T sum_q r_q lam_q, added in source order
            rc = seed_scatter(t, w, auxp, (long long)R, sum_sources == 0, nullptr, 0, 0, nullptr, dtype, st);
            if (rc) return rc;
        }
    }
    return EIK_OK;
}

// ---------------------------------------------------------------- batched tangents
template <typename T, int V, bool TR>
static int launch_batch(Tangent *const *ts, int ntan, const TravParams *Ps, const int *R, cudaStream_t st)
{
    Tangent *t0 = ts[0];
    ClusterBatch B{};
    B.ntan = ntan;
    B.unit_ptr[0] = 0;
    int min_lanes = 1 << 30, W = 4, tab = 0;
    for (int k = 0; k < ntan; ++k) {
        B.P[k] = Ps[k];
        B.unit_ptr[k + 1] = B.unit_ptr[k] + ts[k]->S;
        B.lanes[k] = R[k] / V;
        min_lanes = std::min(min_lanes, B.lanes[k]);
        if (B.lanes[k] % 4) W = std::min(W, B.lanes[k] % 2 ? 1 : 2);
        tab = std::max(tab, ts[k]->maxL + 1);
    }
    const int cap = t0->opts.pass_units > 0 ? t0->opts.pass_units : 4;
    W = std::min(W, cap >= 4 ? 4 : (cap >= 2 ? 2 : 1));
    const int threads = t0->opts.cluster_threads > 0 ? t0->opts.cluster_threads : 256;
    for (int k = 0; k < ntan; ++k)
        if (B.lanes[k] / W > threads) {
            set_error("batch: %d right-hand-side lanes exceed %d threads per CTA", B.lanes[k], threads);
            return EIK_ERR_INVALID;
        }
    B.tp = std::min(512, (4 / W) * (threads / std::max(1, min_lanes / W)));
    B.tab = tab;
    while (B.tp > 32 && CL_SLOTS * cl_slot_bytes<T>(B.tp) + 3 * (size_t)B.tab * sizeof(int) > 160 * 1024) B.tp /= 2;
    B.ticket = Ps[0].ticket + 1;
    const int units = B.unit_ptr[ntan];
    if (W == 4) return launch_cluster_u<T, V, TR, 4>(t0, B, units, st);
    if (W == 2) return launch_cluster_u<T, V, TR, 2>(t0, B, units, st);
    return launch_cluster_u<T, V, TR, 1>(t0, B, units, st);
}

// ticket -> {tangent, item} of a merged step-major order: runs {tangent, first item, items,
// first ticket}, in ticket order
__global__ void k_batch_order(int total, const int4 *__restrict__ runs, int nruns, int2 *__restrict__ order)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int lo = 0, hi = nruns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (runs[mid].w <= t) lo = mid;
        else hi = mid - 1;
    }
    const int4 r = runs[lo];
    order[t] = make_int2(r.x, r.y + (t - r.w));
}

// One persistent launch over the items of several tangents (multi-slot kernel): tickets in
// a merged step-major order, step s of every tangent before step s + 1 of any.
template <typename T, int V, bool TR>
static int launch_multi_batch(Tangent *const *ts, int ntan, const TravParams *Ps, const int *R, cudaStream_t st)
{
    Tangent *t0 = ts[0];
    MultiBatch B{};
    B.ntan = ntan;
    int smax = 0;
    for (int k = 0; k < ntan; ++k) {
        B.P[k] = Ps[k];
        const int lanes = R[k] / V;
        int G = 1;
        while (G < lanes && G < 32) G <<= 1;
        B.G[k] = G;
        smax = std::max(smax, ts[k]->maxL);
    }
    std::vector<int4> &runs = t0->batch_runs;
    runs.clear();
    long long tk = 0;
    for (int s = 0; s < smax; ++s)
        for (int k = 0; k < ntan; ++k) {
            if (s >= ts[k]->maxL) continue;
            const std::vector<int> &sp = TR ? ts[k]->step_ptr_bwd : ts[k]->step_ptr_fwd;
            const int n = sp[s + 1] - sp[s];
            if (n <= 0) continue;
            runs.push_back(make_int4(k, sp[s], n, (int)tk));
            tk += n;
        }
    if (tk >= (1ll << 31)) { set_error("batch: more than 2^31 - 1 work items"); return EIK_ERR_INVALID; }
    B.nitems = (int)tk;
    const size_t need = (size_t)std::max<long long>(tk, 1) * sizeof(int2) + runs.size() * sizeof(int4) + 64;
    if (need > t0->batch_bytes) {
        if (t0->batch_buf) cudaFree(t0->batch_buf);
        t0->batch_buf = nullptr;
        t0->batch_bytes = 0;
        EIK_CHECK(cudaMalloc(&t0->batch_buf, need));
        t0->batch_bytes = need;
    }
    int2 *order = reinterpret_cast<int2 *>(t0->batch_buf);
    int4 *runs_d = reinterpret_cast<int4 *>(reinterpret_cast<char *>(t0->batch_buf) +
                                            ((size_t)std::max<long long>(tk, 1) * sizeof(int2) + 15) / 16 * 16);
    if (!runs.empty()) {
        EIK_CHECK(cudaMemcpyAsync(runs_d, runs.data(), runs.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
        k_batch_order<<<(unsigned)((tk + 255) / 256), 256, 0, st>>>((int)tk, runs_d, (int)runs.size(), order);
        EIK_CHECK_LAUNCH();
    }
    B.order = order;
    B.ticket = Ps[0].ticket;
    const int slots = std::max(2, std::min(4, t0->opts.item_slots));
    void (*mk)(MultiBatch) = slots >= 4 ? k_traverse_multi<T, V, TR, 4, true>
                             : slots == 3 ? k_traverse_multi<T, V, TR, 3, true> : k_traverse_multi<T, V, TR, 2, true>;
    const int threads = 256;
    int per_sm = t0->opts.ctas_per_sm;
    if (per_sm <= 0) {
        EIK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mk, threads, 0));
        per_sm = std::max(per_sm, 1);
    }
    long long grid = std::min<long long>((long long)t0->num_sms * per_sm, std::max<long long>(tk, 1));
    for (int k = 0; k < ntan; ++k) {
        EIK_CHECK(cudaMemsetAsync(Ps[k].done, 0, (size_t)ts[k]->S * ts[k]->maxL * sizeof(int), st));
        EIK_CHECK(cudaMemsetAsync(Ps[k].item_done, 0, (size_t)std::max(Ps[k].nitems, 1) * sizeof(int), st));
    }
    EIK_CHECK(cudaMemsetAsync(B.ticket, 0, sizeof(int), st));
    mk<<<(unsigned)grid, threads, 0, st>>>(B);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

int traverse_batch(Tangent *const *ts, int ntan, bool TR, const void *const *in, const int *R, void *const *out,
                   int dtype, cudaStream_t st)
{
    NvtxRange range(TR ? "J^T batch" : "J batch");
    for (int k = 0; k < ntan; ++k)
        if (ts[k] && ts[k]->pts.K > 0) { set_error("batched applies take tangents of node sources only"); return EIK_ERR_INVALID; }
    if (ntan < 1 || ntan > CL_MAXTAN) { set_error("batch: 1..%d tangents", CL_MAXTAN); return EIK_ERR_INVALID; }
    if (dtype != EIK_F32 && dtype != EIK_F64) { set_error("bad dtype"); return EIK_ERR_INVALID; }
    const size_t esz = dtype == EIK_F32 ? 4 : 8;
    TravParams Ps[CL_MAXTAN];
    int V = dtype == EIK_F32 ? 4 : 2;
    for (int k = 0; k < ntan; ++k) {
        Tangent *t = ts[k];
        if (!t || !in[k] || !out[k] || R[k] <= 0) { set_error("batch: bad arguments of tangent %d", k); return EIK_ERR_INVALID; }
        if (t->n_rec == 0) { set_error("batch: tangent %d has no receivers", k); return EIK_ERR_INVALID; }
        if (!aligned16(in[k]) || !aligned16(out[k])) { set_error("device buffers must be 16-byte aligned"); return EIK_ERR_INVALID; }
        if (t->device != ts[0]->device) { set_error("batch: tangents on different devices"); return EIK_ERR_INVALID; }
        for (int j = 0; j < k; ++j)
            if (ts[j] == t) { set_error("batch: tangent %d appears twice", k); return EIK_ERR_INVALID; }
        while (R[k] % V) V >>= 1;
        // every right-hand side of every tangent in one pass: the workspace holds them all
        int rc = ensure_workspace(t, (size_t)t->S * t->N * R[k] * esz, (size_t)t->ws_rows * R[k], TR);
        if (rc) return rc;
    }
    for (int k = 0; k < ntan; ++k)
        Ps[k] = make_params(ts[k], TR, MODE_J, in[k], TR ? 0 : 1, R[k], R[k], lane_ws(ts[k], TR), nullptr,
                            TR ? nullptr : out[k], TR ? 1 : 0, dtype);
    int rc;
    // the persistent (multi-slot) schedule unless the first tangent asks for the cluster one or
    // a tangent's items exceed the slot capacity
    bool persistent = ts[0]->opts.schedule != EIK_SCHED_CLUSTER;
    for (int k = 0; k < ntan; ++k) persistent = persistent && ts[k]->item_max <= ITEM_MAX;
    if (persistent) {
        if (dtype == EIK_F32) {
            if (V == 4) rc = TR ? launch_multi_batch<float, 4, true>(ts, ntan, Ps, R, st) : launch_multi_batch<float, 4, false>(ts, ntan, Ps, R, st);
            else if (V == 2) rc = TR ? launch_multi_batch<float, 2, true>(ts, ntan, Ps, R, st) : launch_multi_batch<float, 2, false>(ts, ntan, Ps, R, st);
            else rc = TR ? launch_multi_batch<float, 1, true>(ts, ntan, Ps, R, st) : launch_multi_batch<float, 1, false>(ts, ntan, Ps, R, st);
        } else {
            if (V == 2) rc = TR ? launch_multi_batch<double, 2, true>(ts, ntan, Ps, R, st) : launch_multi_batch<double, 2, false>(ts, ntan, Ps, R, st);
            else rc = TR ? launch_multi_batch<double, 1, true>(ts, ntan, Ps, R, st) : launch_multi_batch<double, 1, false>(ts, ntan, Ps, R, st);
        }
    } else if (dtype == EIK_F32) {
        if (V == 4) rc = TR ? launch_batch<float, 4, true>(ts, ntan, Ps, R, st) : launch_batch<float, 4, false>(ts, ntan, Ps, R, st);
        else if (V == 2) rc = TR ? launch_batch<float, 2, true>(ts, ntan, Ps, R, st) : launch_batch<float, 2, false>(ts, ntan, Ps, R, st);
        else rc = TR ? launch_batch<float, 1, true>(ts, ntan, Ps, R, st) : launch_batch<float, 1, false>(ts, ntan, Ps, R, st);
    } else {
        if (V == 2) rc = TR ? launch_batch<double, 2, true>(ts, ntan, Ps, R, st) : launch_batch<double, 2, false>(ts, ntan, Ps, R, st);
        else rc = TR ? launch_batch<double, 1, true>(ts, ntan, Ps, R, st) : launch_batch<double, 1, false>(ts, ntan, Ps, R, st);
    }
    if (rc) return rc;
    if (TR)
        for (int k = 0; k < ntan; ++k) {
            rc = source_sum(ts[k], R[k], out[k], (long long)R[k], dtype, st);
            if (rc) return rc;
        }
    return EIK_OK;
}

}  // namespace eik
