// Level-synchronous schedule of the block traversals B_a / B_a^T (Prop. 3, Sec. 4.3-4.4).
//
// One cooperative launch (every CTA resident) in which all sources advance together: global
// step s holds, for every source, the next level of its traversal (forward levels in
// increasing order, the transpose's in decreasing order).  Within a step no row depends on
// another (the levels are longest-path levels of the condensation), so a step's work is
// one flat list of units cut into equal contiguous slices, one per CTA, and one grid-wide
// barrier separates consecutive steps.  A nontrivial SCC block takes two steps of its
// source: the first forms its right-hand side b_C (one unit per block row, FP64, into the
// block workspace), the second multiplies by A_C^-1 (one unit per block row), so a block's
// FP64 work is spread over the grid like any other row and the source's later levels move
// one step down.
//
// Unit records.  Once per tangent and direction the step table is turned into one record
// per unit, in step order: {node, position, receiver slot, entries | kind | source} and
// {first three upstream positions, first entry}.  A CTA's slice of a step is then one
// contiguous run of records, copied into a three-slot shared-memory ring with cp.async two
// steps ahead; after arriving at a step's barrier the CTA prefetches the input rows of the
// step after next into L2.  None of that data is written by the traversal, so all of
// it moves while the barrier completes; after the wait only the upstream gathers of the
// transported field, the sums and the stores remain.
//
// Tasks: task = (unit, lane), lane = V consecutive right-hand sides.  A thread takes ILP
// tasks at a time and issues all their loads before summing any.  The arithmetic of a row
// (input x C*M, then the upstream terms in edge order; block rows in FP64 with the explicit
// inverse) is the same sequence of operations as in the other schedules.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "eik_internal.h"
#include "eik_trav.h"
#include "eik_vec.cuh"

namespace eik {

enum : int { SK_POS = 0, SK_BRHS = 1, SK_BMUL = 2, SK_SKIP = 3 };   // unit kinds
constexpr int SY_UMAX = 512;       // units per CTA and ring slot (wider slices run in chunks)
constexpr int SY_EDGES = 3;        // upstream positions held in a record; further ones are read in place

// record word 3: entries | kind << 4 | source << 8
__host__ __device__ __forceinline__ int sy_meta(int cnt, int kind, int a) { return cnt | (kind << 4) | (a << 8); }

// the row arithmetic with its rounding steps spelled out (a product, then one fused
// multiply-add per upstream term), so that no contraction choice of the compiler changes it
__device__ __forceinline__ float sy_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double sy_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float sy_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double sy_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void prefetch_line_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ void sy_cp16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void sy_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void sy_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// the input row a singleton task reads (nullptr: zero input), as node_input reads it
template <typename T, bool TR>
__device__ __forceinline__ const T *sy_input_row(const TravParams &P, long long a, int v, int rec)
{
    const T *in = reinterpret_cast<const T *>(P.in);
    if (!TR) return in + ((P.mode == MODE_J && P.shared_in ? 0 : a * P.N) + v) * P.ld_in;
    if (P.mode == MODE_J) return rec >= 0 ? in + (a * P.n_rec + rec) * P.ld_in : nullptr;
    return in + (a * P.N + v) * P.ld_in;
}

// One unit record (48 bytes for FP32, 64 for FP64; a whole number of 16-byte chunks).
template <typename T> struct SyRec {
    int v, p, rec, meta;        // node, position, receiver slot (-1), entries | kind << 4 | source << 8;
                                // block units: block id, block row, -1, meta
    int en[SY_EDGES];           // first upstream positions
    int eg;                     // global index of the row's first entry (rows with more entries)
    T cq;                       // C*M of the position
    T w[SY_EDGES];              // first weights
};
static_assert(sizeof(SyRec<float>) == 48 && sizeof(SyRec<double>) == 64, "record layout");

// Unit records of one direction and precision: unit u (global index over all steps) lies in
// the last segment whose first global unit is <= u.  Segments are {kind << 24 | source,
// first position or block, units, -}.
template <typename T>
__global__ void k_sync_records(int total, const int4 *__restrict__ seg, const int *__restrict__ seg_g, int nseg,
                               long long N, const int *__restrict__ perm, const int *__restrict__ rowptr,
                               const int *__restrict__ enode, const T *__restrict__ ew, const T *__restrict__ cq,
                               const long long *__restrict__ ebase, const int *__restrict__ rec_slot,
                               SyRec<T> *__restrict__ out)
{
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= total) return;
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_g[mid] <= u) lo = mid;
        else hi = mid - 1;
    }
    const int4 g = seg[lo];
    const int kind = g.x >> 24, a = g.x & 0xffffff;
    const int off = (int)(u - seg_g[lo]);
    SyRec<T> r;
    r.rec = -1;
    r.eg = 0;
    r.cq = T(0);
#pragma unroll
    for (int e = 0; e < SY_EDGES; ++e) {
        r.en[e] = 0;
        r.w[e] = T(0);
    }
    if (kind != SK_POS) {            // block row: block id, row
        r.v = g.y;
        r.p = off;
        r.meta = sy_meta(0, kind, a);
    } else {
        const int p = g.y + off;
        const long long ap = (long long)a * N + p;
        r.v = perm[ap];
        r.p = p;
        if (r.v < 0) {
            r.meta = sy_meta(0, SK_SKIP, a);     // member of a nontrivial block
        } else {
            const int r0 = rowptr[(long long)a * (N + 1) + p], cnt = rowptr[(long long)a * (N + 1) + p + 1] - r0;
            const long long eb = ebase[a] + r0;
            r.rec = rec_slot[ap];
            r.meta = sy_meta(cnt, SK_POS, a);
            r.eg = (int)eb;
            r.cq = cq[ap];
#pragma unroll
            for (int e = 0; e < SY_EDGES; ++e)
                if (e < cnt) {
                    r.en[e] = enode[eb + e];
                    r.w[e] = ew[eb + e];
                }
        }
    }
    out[u] = r;
}

// One block unit (row m of block b of source a) for lanes [r, r + V): the right-hand side
// b_m = q_m + sum over external upstream entries (SK_BRHS, into the block workspace), or
// x_m = (A_C^-1 b)_m (SK_BMUL; the transpose reads A_C^-1 transposed) with the stores of a
// solved position.  FP64 throughout, in the operation order of the other schedules.
template <typename T, int V, bool TR>
__device__ __noinline__ void sy_block_unit(const TravParams &P, int kind, int a, int b, int m, int r)
{
    const int4 d = __ldg(&P.blk_desc[b]);
    const int p0 = d.y, k = d.z;
    const long long luo = __ldg(&P.blk_off[3 * b]), wso = __ldg(&P.blk_off[3 * b + 2]);
    const int R = P.R;
    const long long N = P.N;
    const int p = p0 + m;
    const long long ap = (long long)a * N + p;
    const int v = ~__ldg(P.perm + ap);
    const int rec = __ldg(P.rec_slot + ap);
    const T *in = reinterpret_cast<const T *>(P.in);
    T *x = reinterpret_cast<T *>(P.x) + (long long)a * N * P.ld_x;
    double *W = P.ws + wso * R;
    if (kind == SK_BRHS) {
        const int *rp = P.rowptr + (long long)a * (N + 1);
        const long long eb = __ldg(P.ebase + a);
        const int e0 = __ldg(rp + p), e1 = __ldg(rp + p + 1);
        if (!EIK_POSITION_OK(P, a, p, v, e0, e1 - e0, -1, P.enode + eb, rec)) return;
        double acc[V];
#pragma unroll
        for (int u = 0; u < V; ++u) {
            if (!TR) {
                if (P.mode == MODE_J)
                    acc[u] = sy_mul(__ldg(P.cq64 + ap), (double)in[((P.shared_in ? 0 : (long long)a * N) + v) * P.ld_in + r + u]);
                else
                    acc[u] = (double)in[((long long)a * N + v) * P.ld_in + r + u];
            } else {
                if (P.mode == MODE_J) acc[u] = rec >= 0 ? (double)in[((long long)a * P.n_rec + rec) * P.ld_in + r + u] : 0.0;
                else acc[u] = (double)in[((long long)a * N + v) * P.ld_in + r + u];
            }
        }
        // the external upstream entries (at most 2 x ndim), all loads issued first
        double wv[MAX_ROW];
        T xv[MAX_ROW][V];
#pragma unroll
        for (int j = 0; j < MAX_ROW; ++j)
            if (e0 + j < e1) {
                wv[j] = __ldg(P.ew64 + eb + e0 + j);
                const T *xr = x + (long long)__ldg(P.enode + eb + e0 + j) * P.ld_x + r;
#pragma unroll
                for (int u = 0; u < V; ++u) xv[j][u] = __ldcg(xr + u);
            }
#pragma unroll
        for (int j = 0; j < MAX_ROW; ++j)
            if (e0 + j < e1) {
#pragma unroll
                for (int u = 0; u < V; ++u) acc[u] = sy_fma(wv[j], (double)xv[j][u], acc[u]);
            }
#pragma unroll
        for (int u = 0; u < V; ++u) W[(long long)m * R + r + u] = acc[u];
        return;
    }
    // x_m = sum_c A_C^-1[m][c] b_c in order of c, the loads of SY_BCH terms issued together
    constexpr int SY_BCH = 8;
    const double *Ainv = P.binv + luo;
    double val[V];
#pragma unroll
    for (int u = 0; u < V; ++u) val[u] = 0.0;
    for (int c0 = 0; c0 < k; c0 += SY_BCH) {
        double av[SY_BCH], wv[SY_BCH][V];
#pragma unroll
        for (int j = 0; j < SY_BCH; ++j)
            if (c0 + j < k) {
                const int c = c0 + j;
                av[j] = TR ? __ldg(Ainv + (long long)c * k + m) : __ldg(Ainv + (long long)m * k + c);
#pragma unroll
                for (int u = 0; u < V; ++u) wv[j][u] = __ldcg(W + (long long)c * R + r + u);
            }
#pragma unroll
        for (int j = 0; j < SY_BCH; ++j)
            if (c0 + j < k) {
#pragma unroll
                for (int u = 0; u < V; ++u) val[u] = sy_fma(av[j], wv[j][u], val[u]);
            }
    }
    T *aux = reinterpret_cast<T *>(P.aux);
#pragma unroll
    for (int u = 0; u < V; ++u) {
        x[(long long)p * P.ld_x + r + u] = (T)val[u];
        if (P.out) reinterpret_cast<T *>(P.out)[((long long)a * N + v) * P.ld_out + r + u] = (T)val[u];
        if (P.mode == MODE_J && aux) {
            if (!TR) {
                if (rec >= 0) aux[((long long)a * P.n_rec + rec) * P.ld_aux + r + u] = (T)val[u];
            } else if (!P.sum) {
                aux[((long long)a * N + v) * P.ld_aux + r + u] = (T)(__ldg(P.cq64 + ap) * val[u]);
            }
        }
    }
}


// the loads of one singleton task: input row and up to SY_EDGES upstream rows
template <typename T, int V> struct SyLoad {
    Pack<T, V> q;
    Pack<T, V> up[SY_EDGES];
};

// issue the loads of task (record R, lanes [r, r + V)); x is the source's field at column r
template <typename T, int V, bool TR>
__device__ __forceinline__ void sy_issue(const TravParams &P, const SyRec<T> &R, int r, SyLoad<T, V> &L)
{
    const int cnt = R.meta & 15, a = R.meta >> 8;
    const T *x = reinterpret_cast<const T *>(P.x) + (long long)a * P.N * P.ld_x + r;
#pragma unroll
    for (int e = 0; e < SY_EDGES; ++e)
        if (e < cnt) L.up[e] = load_l2<T, V>(x + (long long)R.en[e] * P.ld_x);
    const T *src = sy_input_row<T, TR>(P, a, R.v, R.rec);
    if (src) {
        L.q = load_ro<T, V>(src + r);
    } else {
#pragma unroll
        for (int u = 0; u < V; ++u) L.q.v[u] = T(0);
    }
}

template <typename T, int V, bool TR>
__device__ __forceinline__ void sy_finish(const TravParams &P, const SyRec<T> &R, int r, SyLoad<T, V> &L)
{
    const int cnt = R.meta & 15, a = R.meta >> 8;
    const T scale = (!TR && P.mode == MODE_J) ? R.cq : T(1);
    Pack<T, V> acc;
#pragma unroll
    for (int u = 0; u < V; ++u) acc.v[u] = sy_mul(scale, L.q.v[u]);
#pragma unroll
    for (int e = 0; e < SY_EDGES; ++e)
        if (e < cnt) {
#pragma unroll
            for (int u = 0; u < V; ++u) acc.v[u] = sy_fma(R.w[e], L.up[e].v[u], acc.v[u]);
        }
    T *x = reinterpret_cast<T *>(P.x) + (long long)a * P.N * P.ld_x;
    if (cnt > SY_EDGES) {       // rows with more upstream entries than a record holds (rare)
        const T *ew = reinterpret_cast<const T *>(P.ew);
        for (int e = SY_EDGES; e < cnt; ++e) {
            const T w = __ldg(ew + R.eg + e);
            const Pack<T, V> xv = load_l2<T, V>(x + (long long)__ldg(P.enode + R.eg + e) * P.ld_x + r);
#pragma unroll
            for (int u = 0; u < V; ++u) acc.v[u] = sy_fma(w, xv.v[u], acc.v[u]);
        }
    }
    node_output<T, V, TR>(P, a, R.v, R.p, R.rec, R.cq, r, x, acc);
}

// checked build: the indices of a singleton record against their arrays
template <typename T>
__device__ __forceinline__ bool sy_record_ok(const TravParams &P, const SyRec<T> &R)
{
    const int a = R.meta >> 8;
    const long long eb = __ldg(P.ebase + a);
    return EIK_POSITION_OK(P, a, R.p, R.v, (int)(R.eg - eb), R.meta & 15, -1, P.enode + eb, R.rec);
}

// All tasks of nu singleton records of a ring slot (every thread).  Thread tid owns lane
// tid % lanes of units tid / lanes + k * upt (upt = units per pass); ILP units at a time,
// all their loads issued before any sum.
template <typename T, int V, bool TR, int ILP>
__device__ __forceinline__ void sy_compute(const TravParams &P, const SyRec<T> *rs, int nu, int lanes, int upt)
{
    const int i0 = threadIdx.x / lanes;
    if (i0 >= upt) return;
    const int r = (threadIdx.x - i0 * lanes) * V;
    for (int ib = i0; ib < nu; ib += ILP * upt) {
        SyLoad<T, V> L[ILP];
        bool on[ILP];
#pragma unroll
        for (int q = 0; q < ILP; ++q) {
            const int i = ib + q * upt;
            on[q] = false;
            if (i >= nu) continue;
            const SyRec<T> &R = rs[i];
            if (((R.meta >> 4) & 15) != SK_POS || !sy_record_ok<T>(P, R)) continue;
            on[q] = true;
            sy_issue<T, V, TR>(P, R, r, L[q]);
        }
#pragma unroll
        for (int q = 0; q < ILP; ++q)
            if (on[q]) sy_finish<T, V, TR>(P, rs[ib + q * upt], r, L[q]);
    }
}

// block records of a step dealt to this CTA: j = first + blockIdx.x + k * gridDim.x (every
// thread; records read in place)
template <typename T, int V, bool TR>
__device__ __noinline__ void sy_blocks(const TravParams &P, const SyRec<T> *__restrict__ recs, long long first,
                                       long long end)
{
    const int lanes = P.R / V;
    const long long mine = end - first > blockIdx.x ? (end - first - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    for (long long t = threadIdx.x; t < mine * lanes; t += blockDim.x) {
        const long long q = t / lanes;
        const long long j = first + blockIdx.x + q * gridDim.x;
        const int v = __ldg(&recs[j].v), m = __ldg(&recs[j].p), meta = __ldg(&recs[j].meta);
        const int kind = (meta >> 4) & 15;
        if (kind == SK_BRHS || kind == SK_BMUL) sy_block_unit<T, V, TR>(P, kind, meta >> 8, v, m, (int)(t - q * lanes) * V);
    }
}

// this CTA's singleton slice [u0, u1) (global record indices) of every global step, into a
// shared table (every thread; the 64-bit divisions run once per step and CTA)
__device__ __forceinline__ void sy_slices(const int *__restrict__ step_base, int nsteps, int2 *sl)
{
    for (int s = threadIdx.x; s < nsteps; s += blockDim.x) {
        const long long b = __ldg(step_base + 2 * s), ns = __ldg(step_base + 2 * s + 1);
        sl[s] = make_int2((int)(b + ns * blockIdx.x / gridDim.x), (int)(b + ns * (blockIdx.x + 1) / gridDim.x));
    }
}

// cp.async of records [u0, u0 + nu) into a ring slot (every thread; not committed here)
template <typename T>
__device__ __forceinline__ void sy_fetch(const SyRec<T> *__restrict__ recs, long long u0, int nu, SyRec<T> *slot)
{
    constexpr int C = sizeof(SyRec<T>) / 16;
    const char *src = reinterpret_cast<const char *>(recs + u0);
    char *dst = reinterpret_cast<char *>(slot);
    for (int i = threadIdx.x; i < C * nu; i += blockDim.x) sy_cp16(dst + 16 * i, src + 16 * i);
}

// prefetch into L2 the input rows of the singleton records of a slot
template <typename T, bool TR>
__device__ __forceinline__ void sy_prefetch(const TravParams &P, const SyRec<T> *rs, int nu)
{
    const int rowb = P.R * (int)sizeof(T);
    for (int i = threadIdx.x; i < nu; i += blockDim.x) {
        const SyRec<T> &R = rs[i];
        if (((R.meta >> 4) & 15) != SK_POS) continue;
        const T *src = sy_input_row<T, TR>(P, R.meta >> 8, R.v, R.rec);
        if (src)
            for (int o = 0; o < rowb; o += 128) prefetch_line_l2(reinterpret_cast<const char *>(src) + o);
    }
}

// Every CTA of the cooperative launch runs this loop over the global steps; steps end at a
// grid-wide barrier (one counter: each CTA adds 1 after its stores, then waits until the
// counter reaches (s + 1) x CTAs).  Ring slot s % 3 holds the first chunk of step s's
// singleton records; the records of step s + 2 are fetched while step s computes, the
// step's block records follow, dealt round-robin over the CTAs.  The wait is bounded by
// globaltimer: past the time-out the fault is latched and every CTA leaves (they also
// leave when another one latched a fault), so the launch ends in bounded time with
// EIK_ERR_TIMEOUT.
template <typename T, int V, bool TR, int NT, int ILP>
__global__ void __launch_bounds__(NT, 1)
    k_traverse_sync(const __grid_constant__ TravParams P, const SyRec<T> *__restrict__ recs,
                    const int *__restrict__ step_base, int nsteps, unsigned *bar, int hold_step)
{
    extern __shared__ __align__(16) unsigned char ring_raw[];     // 3 slots x SY_UMAX records, slice table
    SyRec<T> *ring = reinterpret_cast<SyRec<T> *>(ring_raw);
    int2 *sl = reinterpret_cast<int2 *>(ring_raw + 3 * SY_UMAX * sizeof(SyRec<T>));
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    const int lanes = P.R / V, upt = NT / lanes;
    auto slot = [&](int s) { return ring + (size_t)(s % 3) * SY_UMAX; };
    auto first_n = [&](int s) { return min(sl[s].y - sl[s].x, SY_UMAX); };
    auto fetch_first = [&](int s) {
        if (s < nsteps) sy_fetch<T>(recs, sl[s].x, first_n(s), slot(s));
        sy_commit();
    };
    sy_slices(step_base, nsteps, sl);
    __syncthreads();
    fetch_first(0);
    fetch_first(1);
    sy_wait<0>();                  // records of steps 0 and 1
    __syncthreads();
    if (nsteps > 0) sy_prefetch<T, TR>(P, slot(0), first_n(0));
    if (nsteps > 1) sy_prefetch<T, TR>(P, slot(1), first_n(1));
    for (int s = 0; s < nsteps; ++s) {
        fetch_first(s + 2);        // one group per step, possibly empty
        const int u0 = sl[s].x, u1 = sl[s].y;
        for (int c0 = u0; c0 < u1; c0 += SY_UMAX) {
            const int nu = min(u1 - c0, SY_UMAX);
            if (c0 != u0) {        // slices wider than one slot: the rest in place
                __syncthreads();
                sy_fetch<T>(recs, c0, nu, slot(s));
                sy_commit();
                sy_wait<0>();
                __syncthreads();
            }
            sy_compute<T, V, TR, ILP>(P, slot(s), nu, lanes, upt);
        }
        const int b0 = __ldg(step_base + 2 * s) + __ldg(step_base + 2 * s + 1), b1 = __ldg(step_base + 2 * s + 2);
        if (b1 > b0) sy_blocks<T, V, TR>(P, recs, b0, b1);
        // ---- arrive: every store of this CTA for step s, then the counter
        __syncthreads();
        if (tid == 0 && !(s == hold_step && blockIdx.x == 0)) {   // (a test hold: CTA 0 skips one arrival)
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        }
        if (s + 1 == nsteps) break;
        // ---- records of step s + 2 visible; their input rows into L2 (two steps ahead of use)
        sy_wait<0>();
        __syncthreads();
        if (s + 2 < nsteps) sy_prefetch<T, TR>(P, slot(s + 2), first_n(s + 2));
        // ---- wait for step s everywhere
        if (tid == 0) {
            int ok = 1;
            const unsigned target = (unsigned)(s + 1) * gridDim.x;
            if (ld_acquire_u32(bar) < target) {
                const unsigned long long t0 = global_ns();
                for (int n = 0;; ++n) {
                    if (ld_acquire_u32(bar) >= target) break;
                    if ((n & 63) == 63) {
                        if (*(volatile int *)P.err != 0) { ok = 0; break; }
                        if (global_ns() - t0 > P.timeout_ns) {
                            if (atomicCAS(P.err, 0, DEV_TIMEOUT) == 0) { P.err[1] = -1; P.err[2] = s; P.err[3] = (int)blockIdx.x; }
                            ok = 0;
                            break;
                        }
                    }
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
    }
    sy_wait<0>();                  // no copy outlives the CTA
}

// ---------------------------------------------------------------- host side
// Step table and unit records of one direction and precision: per source, its levels in
// traversal order, one global step each, plus one more step after every level that holds
// nontrivial blocks (their inverse products).  Built once per tangent, direction and
// precision (synchronizes).
template <typename T>
static int sync_table(Tangent *t, bool TR)
{
    const int d = TR ? 1 : 0, f = sizeof(T) == 4 ? 0 : 1;
    if (t->sync_rec[d][f]) return EIK_OK;
    const int S = t->S, maxL = t->maxL;
    if (S >= (1 << 23)) { set_error("level-synchronous schedule: at most 2^23 - 1 sources"); return EIK_ERR_INVALID; }
    const std::vector<long long> &eb_host = TR ? t->tbase : t->ebase;
    if (!eb_host.empty() && eb_host.back() >= (1ll << 31)) {
        set_error("level-synchronous schedule: more than 2^31 - 1 upstream entries in one direction");
        return EIK_ERR_INVALID;
    }
    std::vector<std::vector<int4>> steps;
    auto put = [&](int s, int4 g) {
        if ((int)steps.size() <= s) steps.resize(s + 1);
        steps[s].push_back(g);
    };
    size_t bi = 0;           // blocks are ordered by (source, level)
    for (int a = 0; a < S; ++a) {
        const int nl = t->nlev[a];
        const size_t b_first = bi;
        while (bi < t->blocks.size() && t->blocks[bi].src == a) ++bi;
        std::vector<std::pair<size_t, size_t>> by_level(nl, {0, 0});   // blocks of each level
        for (size_t b = b_first; b < bi; ++b) {
            const int L = t->blocks[b].level;
            if (L < 0 || L >= nl) { set_error("block %zu of source %d has level %d of %d", b, a, L, nl); return EIK_ERR_INVALID; }
            if (by_level[L].second == 0) by_level[L].first = b;
            by_level[L].second = b + 1;
        }
        int s = 0;
        for (int i = 0; i < nl; ++i) {
            const int L = TR ? nl - 1 - i : i;
            const long long p0 = t->level_ptr[(size_t)a * (maxL + 1) + L], p1 = t->level_ptr[(size_t)a * (maxL + 1) + L + 1];
            if (p1 > p0) put(s, make_int4(a | (SK_POS << 24), (int)p0, (int)(p1 - p0), 0));
            const auto br = by_level[L];
            if (br.second > br.first) {
                for (size_t b = br.first; b < br.second; ++b) put(s, make_int4(a | (SK_BRHS << 24), (int)b, t->blocks[b].k, 0));
                for (size_t b = br.first; b < br.second; ++b) put(s + 1, make_int4(a | (SK_BMUL << 24), (int)b, t->blocks[b].k, 0));
                s += 2;
            } else {
                s += 1;
            }
        }
    }
    std::vector<int4> seg;
    std::vector<int> seg_g, base(2 * steps.size() + 2, 0);     // per step {first record, singleton records}
    long long total = 0;
    for (size_t s = 0; s < steps.size(); ++s) {
        // singleton rows first (cut into contiguous CTA slices), then the block rows (dealt
        // round-robin over the CTAs, so that a block's FP64 rows spread over the grid)
        std::stable_partition(steps[s].begin(), steps[s].end(), [](const int4 &g) { return (g.x >> 24) == SK_POS; });
        base[2 * s] = (int)total;
        long long ns = 0;
        for (const int4 &g : steps[s])
            if ((g.x >> 24) == SK_POS) ns += g.z;
        base[2 * s + 1] = (int)ns;
        for (const int4 &g : steps[s]) {
            seg.push_back(g);
            seg_g.push_back((int)total);
            total += g.z;
            if (total >= (1ll << 30)) { set_error("level-synchronous schedule: more than 2^30 rows in one direction"); return EIK_ERR_INVALID; }
        }
    }
    base[2 * steps.size()] = (int)total;
    int4 *seg_d = nullptr;
    int *segg_d = nullptr, *base_d = t->sync_base[d];
    SyRec<T> *rec_d = nullptr;
    cudaError_t e = cudaMalloc(&seg_d, std::max<size_t>(seg.size(), 1) * sizeof(int4));
    if (e == cudaSuccess) e = cudaMalloc(&segg_d, std::max<size_t>(seg_g.size(), 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&rec_d, std::max<long long>(total, 1) * sizeof(SyRec<T>));
    if (e == cudaSuccess && !base_d) e = cudaMalloc(&base_d, base.size() * sizeof(int));
    if (e == cudaSuccess && !seg.empty()) e = cudaMemcpy(seg_d, seg.data(), seg.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !seg_g.empty()) e = cudaMemcpy(segg_d, seg_g.data(), seg_g.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base_d, base.data(), base.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && total > 0) {
        const T *ew = reinterpret_cast<const T *>(sizeof(T) == 4 ? (const void *)(TR ? t->dn_w32 : t->up_w32)
                                                                 : (const void *)(TR ? t->dn_w64 : t->up_w64));
        const T *cq = reinterpret_cast<const T *>(sizeof(T) == 4 ? (const void *)t->cq32 : (const void *)t->cq64);
        k_sync_records<T><<<(unsigned)((total + 255) / 256), 256>>>(
            (int)total, seg_d, segg_d, (int)seg.size(), t->N, t->perm, TR ? t->cptr : t->rowptr,
            TR ? t->dn_node : t->up_node, ew, cq, TR ? t->tbase_d : t->ebase_d, t->rec_slot, rec_d);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (seg_d) cudaFree(seg_d);
    if (segg_d) cudaFree(segg_d);
    if (e != cudaSuccess) {
        if (rec_d) cudaFree(rec_d);
        if (base_d && base_d != t->sync_base[d]) cudaFree(base_d);
        return cuda_fail(e, "level-synchronous step table", __FILE__, __LINE__);
    }
    t->sync_rec[d][f] = rec_d;
    t->sync_base[d] = base_d;
    t->sync_steps[d] = (int)steps.size();
    return EIK_OK;
}

int prepare_sync(Tangent *t, int dtype)
{
    int rc = EIK_OK;
    if (dtype != EIK_F64) {
        rc = sync_table<float>(t, false);
        if (!rc) rc = sync_table<float>(t, true);
    }
    if (!rc && dtype != EIK_F32) {
        rc = sync_table<double>(t, false);
        if (!rc) rc = sync_table<double>(t, true);
    }
    if (!rc && !t->sync_bar) EIK_CHECK(cudaMalloc(&t->sync_bar, 2 * 32 * sizeof(unsigned)));
    return rc;
}

template <typename T, int V, bool TR>
static int launch_sync_t(Tangent *t, const TravParams &P, cudaStream_t st)
{
    const int d = TR ? 1 : 0, f = sizeof(T) == 4 ? 0 : 1;
    if (!t->sync_rec[d][f] || !t->sync_bar) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        EIK_CHECK(cudaStreamIsCapturing(st, &cs));
        if (cs != cudaStreamCaptureStatusNone) {
            set_error("level-synchronous schedule: its step tables are built on first use; run one traversal of this "
                      "precision before capturing");
            return EIK_ERR_INVALID;
        }
        int rc = prepare_sync(t, sizeof(T) == 4 ? EIK_F32 : EIK_F64);
        if (rc) return rc;
    }
    if (P.blk_lu_min > 0) {
        for (const Block &b : t->blocks)
            if (b.k >= P.blk_lu_min) {
                set_error("level-synchronous schedule: blocks are applied by their inverse; block_lu_min must be 0 "
                          "(a block of %d nodes would take the LU tier)", b.k);
                return EIK_ERR_INVALID;
            }
    }
    // one CTA per SM: 1024 threads with one unit in flight each (default), or fewer threads
    // with 2 or 4 units in flight each (pass_units)
    void (*kern)(TravParams, const SyRec<T> *, const int *, int, unsigned *, int) = k_traverse_sync<T, V, TR, 1024, 1>;
    int threads = 1024;
    if (t->opts.pass_units == 2) { kern = k_traverse_sync<T, V, TR, 768, 2>; threads = 768; }
    else if (t->opts.pass_units == 3) { kern = k_traverse_sync<T, V, TR, 1024, 2>; threads = 1024; }
    else if (t->opts.pass_units >= 4) { kern = k_traverse_sync<T, V, TR, 512, 4>; threads = 512; }
    if (P.R / V > threads) {
        set_error("level-synchronous schedule: %d right-hand-side lanes exceed %d threads per CTA; set rhs_chunk", P.R / V, threads);
        return EIK_ERR_INVALID;
    }
    const size_t dyn = 3 * SY_UMAX * sizeof(SyRec<T>) + (size_t)t->sync_steps[d] * sizeof(int2);
    if (dyn > 220 * 1024) { set_error("level-synchronous schedule: %d steps exceed the shared slice table", t->sync_steps[d]); return EIK_ERR_INVALID; }
    EIK_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int per_sm = 0;
    EIK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, dyn));
    if (per_sm < 1) { set_error("level-synchronous schedule: the kernel does not fit on an SM"); return EIK_ERR_INVALID; }
    unsigned *bar = t->sync_bar + 32 * d;
    EIK_CHECK(cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(t->num_sms * per_sm));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // while a test hold (tangent_debug_hold) is in place, CTA 0 skips its arrival at one step,
    // so every CTA's bounded barrier wait runs out
    const int hold = t->holds.empty() ? -1 : (int)std::min<long long>(t->holds[0] % t->maxL, t->sync_steps[d] - 1);
    EIK_CHECK(cudaLaunchKernelEx(&cfg, kern, P, (const SyRec<T> *)t->sync_rec[d][f], (const int *)t->sync_base[d],
                                 t->sync_steps[d], bar, hold));
    return EIK_OK;
}

int launch_sync(Tangent *t, const TravParams &P, int esz, int V, bool TR, cudaStream_t st)
{
    if (esz == 4) {
        if (V == 4) return TR ? launch_sync_t<float, 4, true>(t, P, st) : launch_sync_t<float, 4, false>(t, P, st);
        if (V == 2) return TR ? launch_sync_t<float, 2, true>(t, P, st) : launch_sync_t<float, 2, false>(t, P, st);
        return TR ? launch_sync_t<float, 1, true>(t, P, st) : launch_sync_t<float, 1, false>(t, P, st);
    }
    if (V == 2) return TR ? launch_sync_t<double, 2, true>(t, P, st) : launch_sync_t<double, 2, false>(t, P, st);
    return TR ? launch_sync_t<double, 1, true>(t, P, st) : launch_sync_t<double, 1, false>(t, P, st);
}

}  // namespace eik
