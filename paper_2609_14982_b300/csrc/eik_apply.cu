// Phase III of Algorithm 1: the stored block traversals B_a (forward, A^-1) and B_a^T
// (reverse, A^-T) for all sources and right-hand sides (Prop. 3, Sec. 4.3-4.4).
//
// Data layout (right-hand-side index fastest):
//   per-source vectors [S][N][R] in natural node order, so a node's R values are one
//   contiguous, vector-loadable run; the structure (rows, weights, C*M, receiver slots)
//   is stored per source in the canonical level order, so one level is a contiguous
//   slice of every structure array.
// Work: a work item is (source, step, position range) of singleton components of one
//   level, or one nontrivial SCC block.  Items are ordered step-major across sources.
//   Persistent schedule: CTAs take items by ticket; an item of step t waits (bounded)
//   until every item of step t-1 of its own source has completed.  Since tickets are
//   handed out in order, every item waited on is held by a running CTA: no deadlock.
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

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct TravParams {
    int S, R, n_rec, maxL, nitems;
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
    void *x;               // dT or lam [S][N][R]
    void *aux;             // forward: d_rec [S][n_rec][R]; transpose (no sum): g [S][N][R]
    const int4 *items;
    const int *item_cnt;   // [S][maxL] items per (source, step) of this direction
    int *done;             // [S][maxL]
    int *ticket;
    int *err;              // {code, source, step, item}
    const int4 *blk_desc;
    const long long *blk_off;
    const double *lu;
    const int *piv;
    double *ws;
    unsigned long long timeout_ns;
};

// ---------------------------------------------------------------- singleton items
// Each group of G lanes owns one node at a time; lane l handles right-hand sides
// l*V .. l*V+V-1, then strides by G*V.
template <typename T, int V, bool TR>
__device__ __forceinline__ void run_singletons(const TravParams &P, int a, int p0, int p1, int G)
{
    const int lane = threadIdx.x % G, slot = threadIdx.x / G, nslot = blockDim.x / G;
    const long long N = P.N;
    const int R = P.R;
    const int *perm = P.perm + a * N;
    const int *rp = P.rowptr + a * (N + 1);
    const long long eb = P.ebase[a];
    const int *en = P.enode + eb;
    const T *ew = reinterpret_cast<const T *>(P.ew) + eb;
    const T *cq = reinterpret_cast<const T *>(P.cq) + a * N;
    const int *rs = P.rec_slot + a * N;
    const T *in = reinterpret_cast<const T *>(P.in);
    T *x = reinterpret_cast<T *>(P.x) + a * N * R;
    T *aux = reinterpret_cast<T *>(P.aux);
    for (int p = p0 + slot; p < p1; p += nslot) {
        const int v = __ldg(perm + p);
        if (v < 0) continue;                      // member of a nontrivial block
        const int e0 = __ldg(rp + p), e1 = __ldg(rp + p + 1);
        const int rec = __ldg(rs + p);
        const T c = __ldg(cq + p);
        for (int r = lane * V; r < R; r += G * V) {
            Pack<T, V> acc;
            if (!TR) {
                if (P.mode == MODE_J) {
                    const T *src = in + ((P.shared_in ? 0 : (long long)a * N) + v) * R + r;
                    Pack<T, V> q = load_ro<T, V>(src);
#pragma unroll
                    for (int k = 0; k < V; ++k) acc.v[k] = c * q.v[k];
                } else {
                    acc = load_ro<T, V>(in + ((long long)a * N + v) * R + r);
                }
            } else {
                if (P.mode == MODE_J) {
                    if (rec >= 0) acc = load_ro<T, V>(in + ((long long)a * P.n_rec + rec) * R + r);
                    else {
#pragma unroll
                        for (int k = 0; k < V; ++k) acc.v[k] = T(0);
                    }
                } else {
                    acc = load_ro<T, V>(in + ((long long)a * N + v) * R + r);
                }
            }
            for (int e = e0; e < e1; ++e) {
                const int j = __ldg(en + e);
                const T w = __ldg(ew + e);
                Pack<T, V> xj = load_l2<T, V>(x + (long long)j * R + r);
#pragma unroll
                for (int k = 0; k < V; ++k) acc.v[k] += w * xj.v[k];
            }
            store<T, V>(x + (long long)v * R + r, acc);
            if (P.mode == MODE_J && aux) {
                if (!TR) {
                    if (rec >= 0) store<T, V>(aux + ((long long)a * P.n_rec + rec) * R + r, acc);
                } else if (!P.sum) {
                    Pack<T, V> gv;
#pragma unroll
                    for (int k = 0; k < V; ++k) gv.v[k] = c * acc.v[k];
                    store<T, V>(aux + ((long long)a * N + v) * R + r, gv);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- block items
// FP64 solve of one nontrivial SCC block for all right-hand sides (Sec. 4.3):
// forward: b = q_C + W_ext x_ext, then P, L, U; transpose: b = r_C + W_ext^T lam_ext,
// then U^T, L^T, P^T.  Right-hand sides are independent, one thread each.
template <typename T, bool TR>
__device__ void run_block(const TravParams &P, int a, int b)
{
    const int4 d = P.blk_desc[b];
    const int p0 = d.y, k = d.z;
    const long long luo = P.blk_off[3 * b], pvo = P.blk_off[3 * b + 1], wso = P.blk_off[3 * b + 2];
    const int R = P.R;
    const long long N = P.N;
    const int *perm = P.perm + a * N;
    const int *rp = P.rowptr + a * (N + 1);
    const long long eb = P.ebase[a];
    const int *en = P.enode + eb;
    const double *ew = P.ew64 + eb;
    const T *in = reinterpret_cast<const T *>(P.in);
    T *x = reinterpret_cast<T *>(P.x) + a * N * R;
    T *aux = reinterpret_cast<T *>(P.aux);
    double *W = P.ws + wso * R;
    const double *LU = P.lu + luo;
    const int *pv = P.piv + pvo;
    for (long long idx = threadIdx.x; idx < (long long)k * R; idx += blockDim.x) {
        const int m = (int)(idx / R), r = (int)(idx % R);
        const int p = p0 + m;
        const int v = ~__ldg(perm + p);
        double acc;
        const int rec = P.rec_slot[a * N + p];
        if (!TR) {
            if (P.mode == MODE_J)
                acc = P.cq64[a * N + p] * (double)in[((P.shared_in ? 0 : (long long)a * N) + v) * R + r];
            else
                acc = (double)in[((long long)a * N + v) * R + r];
        } else {
            if (P.mode == MODE_J) acc = rec >= 0 ? (double)in[((long long)a * P.n_rec + rec) * R + r] : 0.0;
            else acc = (double)in[((long long)a * N + v) * R + r];
        }
        for (int e = rp[p]; e < rp[p + 1]; ++e) acc += ew[e] * (double)__ldcg(x + (long long)en[e] * R + r);
        W[(long long)m * R + r] = acc;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        double *bcol = W + r;
        if (!TR) {
            for (int m = 0; m < k; ++m) {
                int q = pv[m];
                if (q != m) { double t = bcol[(long long)m * R]; bcol[(long long)m * R] = bcol[(long long)q * R]; bcol[(long long)q * R] = t; }
            }
            for (int m = 0; m < k; ++m) {
                double acc = bcol[(long long)m * R];
                for (int c = 0; c < m; ++c) acc -= LU[(long long)m * k + c] * bcol[(long long)c * R];
                bcol[(long long)m * R] = acc;
            }
            for (int m = k - 1; m >= 0; --m) {
                double acc = bcol[(long long)m * R];
                for (int c = m + 1; c < k; ++c) acc -= LU[(long long)m * k + c] * bcol[(long long)c * R];
                bcol[(long long)m * R] = acc / LU[(long long)m * k + m];
            }
        } else {
            for (int m = 0; m < k; ++m) {
                double acc = bcol[(long long)m * R];
                for (int c = 0; c < m; ++c) acc -= LU[(long long)c * k + m] * bcol[(long long)c * R];
                bcol[(long long)m * R] = acc / LU[(long long)m * k + m];
            }
            for (int m = k - 1; m >= 0; --m) {
                double acc = bcol[(long long)m * R];
                for (int c = m + 1; c < k; ++c) acc -= LU[(long long)c * k + m] * bcol[(long long)c * R];
                bcol[(long long)m * R] = acc;
            }
            for (int m = k - 1; m >= 0; --m) {
                int q = pv[m];
                if (q != m) { double t = bcol[(long long)m * R]; bcol[(long long)m * R] = bcol[(long long)q * R]; bcol[(long long)q * R] = t; }
            }
        }
    }
    __syncthreads();
    for (long long idx = threadIdx.x; idx < (long long)k * R; idx += blockDim.x) {
        const int m = (int)(idx / R), r = (int)(idx % R);
        const int p = p0 + m;
        const int v = ~perm[p];
        const double val = W[(long long)m * R + r];
        x[(long long)v * R + r] = (T)val;
        if (P.mode == MODE_J && aux) {
            const int rec = P.rec_slot[a * N + p];
            if (!TR) {
                if (rec >= 0) aux[((long long)a * P.n_rec + rec) * R + r] = (T)val;
            } else if (!P.sum) {
                aux[((long long)a * N + v) * R + r] = (T)(P.cq64[a * N + p] * val);
            }
        }
    }
}

template <typename T, int V, bool TR>
__device__ __forceinline__ void run_item(const TravParams &P, int4 it, int G)
{
    if (it.z >= 0) run_singletons<T, V, TR>(P, it.x, it.z, it.w, G);
    else run_block<T, TR>(P, it.x, ~it.z);
}

// ---------------------------------------------------------------- persistent schedule
template <typename T, int V, bool TR>
__global__ void __launch_bounds__(256) k_traverse_persistent(TravParams P, int G)
{
    __shared__ int s_item;
    __shared__ int s_ok;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.ticket, 1);
        __syncthreads();
        const int i = s_item;
        if (i >= P.nitems) break;
        const int4 it = P.items[i];
        if (threadIdx.x == 0) {
            int ok = 1;
            if (it.y > 0) {
                const int *flag = P.done + (long long)it.x * P.maxL + it.y - 1;
                const int need = P.item_cnt[(long long)it.x * P.maxL + it.y - 1];
                const unsigned long long t0 = global_ns();
                while (ld_acquire(flag) < need) {
                    if (*(volatile int *)P.err != 0) { ok = 0; break; }
                    if (global_ns() - t0 > P.timeout_ns) {
                        if (atomicCAS(P.err, 0, DEV_TIMEOUT) == 0) { P.err[1] = it.x; P.err[2] = it.y; P.err[3] = i; }
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        run_item<T, V, TR>(P, it, G);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(P.done + (long long)it.x * P.maxL + it.y, 1);
        }
    }
}

// ---------------------------------------------------------------- per-level schedule
template <typename T, int V, bool TR>
__global__ void __launch_bounds__(256) k_traverse_step(TravParams P, int G, int first)
{
    run_item<T, V, TR>(P, P.items[first + blockIdx.x], G);
}

// g[j][r] = sum_a cq_a[j] lam_a[j][r], in source order (FP64 accumulation)
template <typename T>
__global__ void k_source_sum(long long N, int S, int R, const T *__restrict__ cqn, const T *__restrict__ lam,
                             const double *__restrict__ cqn64, T *__restrict__ g)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= N * R) return;
    long long j = idx / R;
    double acc = 0.0;
    for (int a = 0; a < S; ++a) acc += cqn64[(long long)a * N + j] * (double)lam[(long long)a * N * R + idx];
    g[idx] = (T)acc;
    (void)cqn;
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

template <typename T, int V, bool TR>
static int launch_traverse(Tangent *t, TravParams &P, int G, cudaStream_t st)
{
    const int threads = 256;
    if (t->opts.schedule == EIK_SCHED_LEVELS) {
        const std::vector<int> &sp = TR ? t->step_ptr_bwd : t->step_ptr_fwd;
        for (int s = 0; s < t->maxL; ++s) {
            int n = sp[s + 1] - sp[s];
            if (n > 0) k_traverse_step<T, V, TR><<<n, threads, 0, st>>>(P, G, sp[s]);
        }
        EIK_CHECK_LAUNCH();
        return EIK_OK;
    }
    int per_sm = t->opts.ctas_per_sm;
    if (per_sm <= 0) {
        EIK_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traverse_persistent<T, V, TR>, threads, 0));
        per_sm = std::max(per_sm, 1);
    }
    long long grid = std::min<long long>((long long)t->num_sms * per_sm, P.nitems);
    grid = std::max<long long>(grid, 1);
    EIK_CHECK(cudaMemsetAsync(P.done, 0, (size_t)t->S * t->maxL * sizeof(int), st));
    EIK_CHECK(cudaMemsetAsync(P.ticket, 0, sizeof(int), st));
    k_traverse_persistent<T, V, TR><<<(unsigned)grid, threads, 0, st>>>(P, G);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

template <typename T, bool TR>
static int dispatch_v(Tangent *t, TravParams &P, cudaStream_t st)
{
    // widest vector that divides R and keeps every row 16-byte aligned when possible
    const int R = P.R;
    int V = 1;
    if (sizeof(T) == 4 && R % 4 == 0) V = 4;
    else if (R % 2 == 0) V = 2;
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
    const size_t vec_bytes = (size_t)t->S * t->N * R * esz;
    void *x = out_full;
    size_t need_vec = x ? 0 : vec_bytes;
    int rc = ensure_workspace(t, need_vec, (size_t)t->ws_rows * R);
    if (rc) return rc;
    if (!x) x = t->ws_vec;
    TravParams P{};
    P.S = t->S; P.R = R; P.n_rec = t->n_rec; P.maxL = t->maxL; P.nitems = t->nitems; P.N = t->N;
    P.mode = mode; P.shared_in = shared_in; P.sum = sum_sources;
    P.perm = t->perm;
    P.rowptr = TR ? t->cptr : t->rowptr;
    P.enode = TR ? t->dn_node : t->up_node;
    P.ew = dtype == EIK_F32 ? (const void *)(TR ? t->dn_w32 : t->up_w32) : (const void *)(TR ? t->dn_w64 : t->up_w64);
    P.ew64 = TR ? t->dn_w64 : t->up_w64;
    P.ebase = nullptr;
    P.cq = dtype == EIK_F32 ? (const void *)t->cq32 : (const void *)t->cq64;
    P.cq64 = t->cq64;
    P.rec_slot = t->rec_slot;
    P.in = in; P.x = x; P.aux = out_aux;
    P.items = TR ? t->items_bwd : t->items_fwd;
    P.item_cnt = t->item_cnt + (TR ? (size_t)t->S * t->maxL : 0);
    P.done = t->done; P.ticket = t->ticket; P.err = t->err;
    P.blk_desc = t->blk_desc; P.blk_off = t->blk_off; P.lu = t->lu; P.piv = t->piv; P.ws = t->ws_blk;
    P.timeout_ns = (unsigned long long)(t->opts.wait_timeout_s * 1e9);
    // per-source edge bases live on the device next to the items
    static_assert(sizeof(long long) == 8, "");
    P.ebase = TR ? reinterpret_cast<const long long *>(t->tbase_d) : reinterpret_cast<const long long *>(t->ebase_d);
    if (dtype == EIK_F32) rc = TR ? dispatch_v<float, true>(t, P, st) : dispatch_v<float, false>(t, P, st);
    else rc = TR ? dispatch_v<double, true>(t, P, st) : dispatch_v<double, false>(t, P, st);
    if (rc) return rc;
    if (TR && mode == MODE_J && sum_sources && out_aux) {
        long long n = t->N * R;
        unsigned blocks = (unsigned)((n + 255) / 256);
        if (dtype == EIK_F32)
            k_source_sum<float><<<blocks, 256, 0, st>>>(t->N, t->S, R, t->cqn32, (const float *)x, t->cqn64, (float *)out_aux);
        else
            k_source_sum<double><<<blocks, 256, 0, st>>>(t->N, t->S, R, t->cqn64, (const double *)x, t->cqn64, (double *)out_aux);
        EIK_CHECK_LAUNCH();
    }
    return EIK_OK;
}

}  // namespace eik
