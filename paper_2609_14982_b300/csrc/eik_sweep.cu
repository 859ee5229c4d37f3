// The plain form the block traversal is compared with: directional sweeping of the
// same frozen operator (Sec. 3.6), i.e. Gauss-Seidel over the 2^ndim logical
// orderings, cycled to a tolerance.  On the device each ordering is run hyperplane by
// hyperplane: with the axis directions of ordering o, the nodes of one hyperplane
// sum_d i'_d = h depend only on hyperplanes h-1 (already updated) and h+1 (old
// values), which reproduces the lexicographic Gauss-Seidel sweep exactly.  All
// sources and right-hand sides of a hyperplane are updated in one launch, and one
// cycle's launches (2^ndim orderings x hyperplanes) are replayed from a CUDA graph.
//
// The operator is held in a slotted stencil form, built once per precision: for every
// (source, node) 2 ndim weights, slot 2d + (side > 0) for the neighbour across the face
// of axis d on that side, zero where there is no dependency.  The forward form holds
// w_ij of row i at the slot of its upstream neighbour j; the transposed form holds w_ij
// at row j, in the slot of its downstream neighbour i, so A^T is swept with the same
// gather as A.  The FP32 path reads FP32 weights and accumulates in FP32 (the
// precision of the traversal it is compared with); the stopping test takes max |dx| and
// max |x| per cycle with one atomic per warp into one of 64 slots.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "eik_internal.h"
#include "eik_vec.cuh"

namespace eik {

constexpr int SW_SLOTS = 64;          // spread of the stopping-test maxima

struct SweepParams {
    GridDesc g;
    int S, R, order, h;
    int lo0, hi0;                     // range of the first logical coordinate on the hyperplane
    const void *w;                    // slotted weights [S][N][2 ndim] (T)
    const void *b;
    void *x;
    unsigned int *flags;              // [2][SW_SLOTS] float bit patterns: max |dx|, max |x|
};

// slotted form of one source's rows: forward (row i, slot of upstream j) or transposed
// (row j, slot of downstream i); every (row, slot) is written by exactly one edge
template <typename T>
__global__ void k_sweep_slots(GridDesc g, long long SN, const int *__restrict__ cnt, const int *__restrict__ node,
                              const double *__restrict__ w, int transpose, T *__restrict__ out)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= SN) return;
    const int slots = 2 * g.ndim;
    const long long a = v / g.N, i = v - a * g.N;
    for (int e = 0; e < cnt[v]; ++e) {
        const long long j = node[v * slots + e];
        const long long diff = j - i;
        int d = 0, side = 0;
        for (int q = 0; q < g.ndim; ++q) {
            if (diff == g.st[q]) { d = q; side = 1; }
            if (diff == -g.st[q]) { d = q; side = -1; }
        }
        if (!transpose) {
            out[v * slots + 2 * d + (side > 0)] = (T)w[v * slots + e];
        } else {   // at row j, the neighbour across the face towards i is on the other side
            out[(a * g.N + j) * slots + 2 * d + (side < 0)] = (T)w[v * slots + e];
        }
    }
}

template <typename T, int V, int ND>
__global__ void __launch_bounds__(256) k_sweep_plane(SweepParams P)
{
    const GridDesc &g = P.g;
    constexpr int nd = ND, slots = 2 * ND;
    const int RV = P.R / V;
    const int n1 = g.n[1], n2 = nd == 3 ? g.n[2] : 1;
    // 3-D: cells enumerate (c0, c2) and c1 = h - c0 - c2 (the last axis is the shortest)
    const unsigned span = (unsigned)(P.hi0 - P.lo0 + 1) * (unsigned)(nd == 3 ? n2 : 1);
    // blockIdx.y = source; the x threads of a source cover (cell of the hyperplane, lane),
    // 32-bit index arithmetic (a hyperplane of one source holds < 2^31 units)
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    float dx = 0.f, ax = 0.f;
    if (t < span * (unsigned)RV) {
        const int a = blockIdx.y;
        const unsigned cell = t / (unsigned)RV;
        const int rv = (int)(t - cell * (unsigned)RV);
        int c0, c1, c2;
        bool on = true;
        if (nd == 3) {
            const unsigned q0 = cell / (unsigned)n2;
            c0 = P.lo0 + (int)q0;
            c2 = (int)(cell - q0 * (unsigned)n2);
            c1 = P.h - c0 - c2;
            on = c1 >= 0 && c1 < n1;
        } else {
            c0 = P.lo0 + (int)cell;
            c1 = P.h - c0;
            c2 = 0;
            on = c1 >= 0 && c1 < n1;
        }
        if (on) {
            // undo the axis reversals of this ordering
            const int i0 = (P.order & 1) ? g.n[0] - 1 - c0 : c0;
            const int i1 = (P.order & 2) ? n1 - 1 - c1 : c1;
            const int i2 = (P.order & 4) ? n2 - 1 - c2 : c2;
            const long long i = nd == 3 ? ((long long)i0 * n1 + i1) * n2 + i2 : (long long)i0 * n1 + i1;
            const long long base = (long long)a * g.N;
            const T *b = reinterpret_cast<const T *>(P.b) + base * P.R;
            T *x = reinterpret_cast<T *>(P.x) + base * P.R;
            const T *w = reinterpret_cast<const T *>(P.w) + (base + i) * slots;
            const int r = rv * V;
            // every load of the update first: right-hand side, old value, weights and the
            // neighbours across faces with a dependency; then the sum in slot order
            Pack<T, V> acc = load_ro<T, V>(b + i * P.R + r);
            const Pack<T, V> old = load_l2<T, V>(x + i * P.R + r);
            T wq[slots];
            Pack<T, V> xj[slots];
#pragma unroll
            for (int q = 0; q < slots; ++q) wq[q] = __ldg(w + q);
#pragma unroll
            for (int q = 0; q < slots; ++q)
                if (wq[q] != T(0)) {
                    const long long j = (q & 1) ? i + g.st[q >> 1] : i - g.st[q >> 1];
                    xj[q] = load_l2<T, V>(x + j * P.R + r);
                }
#pragma unroll
            for (int q = 0; q < slots; ++q)
                if (wq[q] != T(0)) {
#pragma unroll
                    for (int u = 0; u < V; ++u) acc.v[u] += wq[q] * xj[q].v[u];
                }
            store<T, V>(x + i * P.R + r, acc);
#pragma unroll
            for (int u = 0; u < V; ++u) {
                dx = fmaxf(dx, fabsf((float)(acc.v[u] - old.v[u])));
                ax = fmaxf(ax, fabsf((float)acc.v[u]));
            }
        }
    }
    // one atomic per warp for each maximum, spread over SW_SLOTS words
    for (int o = 16; o > 0; o >>= 1) {
        dx = fmaxf(dx, __shfl_xor_sync(0xffffffffu, dx, o));
        ax = fmaxf(ax, __shfl_xor_sync(0xffffffffu, ax, o));
    }
    if ((threadIdx.x & 31) == 0 && (dx > 0.f || ax > 0.f)) {
        const int slot = (int)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % SW_SLOTS);
        atomicMax(P.flags + slot, __float_as_uint(dx));
        atomicMax(P.flags + SW_SLOTS + slot, __float_as_uint(ax));
    }
}

template <typename T, int V, int ND>
static int launch_cycle_nd(const SweepParams &P0, long long S, int R, cudaStream_t st)
{
    const GridDesc &g = P0.g;
    const int nd = g.ndim, nord = 1 << nd;
    int hmax = 0;
    for (int d = 0; d < nd; ++d) hmax += g.n[d] - 1;
    SweepParams P = P0;
    for (int o = 0; o < nord; ++o) {
        P.order = o;
        for (int h = 0; h <= hmax; ++h) {
            const int rest = hmax - (g.n[0] - 1);
            P.h = h;
            P.lo0 = std::max(0, h - rest);
            P.hi0 = std::min(g.n[0] - 1, h);
            const long long span = (long long)(P.hi0 - P.lo0 + 1) * (nd == 3 ? g.n[2] : 1);
            const long long n = span * (R / V);
            k_sweep_plane<T, V, ND><<<dim3((unsigned)((n + 255) / 256), (unsigned)S), 256, 0, st>>>(P);
        }
    }
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

template <typename T, int V>
static int launch_cycle(const SweepParams &P0, long long S, int R, cudaStream_t st)
{
    return P0.g.ndim == 3 ? launch_cycle_nd<T, V, 3>(P0, S, R, st) : launch_cycle_nd<T, V, 2>(P0, S, R, st);
}

// the slotted weights of one direction and precision (built on first use)
static int sweep_weights(Tangent *t, bool transpose, int dtype, const void **out, cudaStream_t st)
{
    const int k = (transpose ? 2 : 0) + (dtype == EIK_F32 ? 1 : 0);
    const size_t esz = dtype == EIK_F32 ? 4 : 8;
    const long long SN = (long long)t->S * t->N;
    const int slots = 2 * t->grid.ndim;
    if (!t->sweep_w[k]) {
        EIK_CHECK(cudaMalloc(&t->sweep_w[k], (size_t)SN * slots * esz));
        EIK_CHECK(cudaMemsetAsync(t->sweep_w[k], 0, (size_t)SN * slots * esz, st));
        const unsigned blocks = (unsigned)((SN + 255) / 256);
        if (dtype == EIK_F32)
            k_sweep_slots<float><<<blocks, 256, 0, st>>>(t->grid, SN, t->nrow_cnt, t->nrow_node, t->nrow_w, transpose,
                                                         (float *)t->sweep_w[k]);
        else
            k_sweep_slots<double><<<blocks, 256, 0, st>>>(t->grid, SN, t->nrow_cnt, t->nrow_node, t->nrow_w, transpose,
                                                          (double *)t->sweep_w[k]);
        EIK_CHECK_LAUNCH();
    }
    *out = t->sweep_w[k];
    return EIK_OK;
}

int sweep(Tangent *t, bool transpose, const void *b, int R, void *x, int dtype, const eik_opts *opts, int *cycles,
          cudaStream_t st)
{
    NvtxRange range(transpose ? "sweep A^T" : "sweep A");
    if (dtype != EIK_F32 && dtype != EIK_F64) { set_error("bad dtype"); return EIK_ERR_INVALID; }
    if (opts->sweep_max_cycles < 1) { set_error("sweep_max_cycles must be positive"); return EIK_ERR_INVALID; }
    const size_t esz = dtype == EIK_F32 ? 4 : 8;
    const void *w = nullptr;
    int rc = sweep_weights(t, transpose, dtype, &w, st);
    if (rc) return rc;
    if (!t->sweep_flags) EIK_CHECK(cudaMalloc(&t->sweep_flags, 2 * SW_SLOTS * sizeof(unsigned int)));
    EIK_CHECK(cudaMemsetAsync(x, 0, (size_t)t->S * t->N * R * esz, st));
    SweepParams P{};
    P.g = t->grid; P.S = t->S; P.R = R;
    P.w = w; P.b = b; P.x = x; P.flags = t->sweep_flags;
    const int V = dtype == EIK_F32 ? (R % 4 == 0 ? 4 : 1) : (R % 2 == 0 ? 2 : 1);
    auto cycle = [&](cudaStream_t s) -> int {
        if (dtype == EIK_F32) return V == 4 ? launch_cycle<float, 4>(P, t->S, R, s) : launch_cycle<float, 1>(P, t->S, R, s);
        return V == 2 ? launch_cycle<double, 2>(P, t->S, R, s) : launch_cycle<double, 1>(P, t->S, R, s);
    };
    // one cycle's launches as a CUDA graph, replayed per cycle and kept for later calls
    // with the same buffers (direct launches while the caller is capturing the stream)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    EIK_CHECK(cudaStreamIsCapturing(st, &cs));
    cudaGraphExec_t exec = nullptr;
    if (cs == cudaStreamCaptureStatusNone) {
        const std::vector<long long> key = {transpose ? 1 : 0, dtype, R, (long long)(uintptr_t)b, (long long)(uintptr_t)x};
        cudaGraphExec_t &slot = t->sweep_graphs[key];
        if (!slot) {
            if (!t->cap_stream) EIK_CHECK(cudaStreamCreateWithFlags(&t->cap_stream, cudaStreamNonBlocking));
            EIK_CHECK(cudaStreamBeginCapture(t->cap_stream, cudaStreamCaptureModeThreadLocal));
            rc = cycle(t->cap_stream);
            cudaGraph_t gr = nullptr;
            cudaError_t e = cudaStreamEndCapture(t->cap_stream, &gr);
            if (rc) { if (gr) cudaGraphDestroy(gr); return rc; }
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
            e = cudaGraphInstantiate(&slot, gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) { slot = nullptr; return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__); }
        }
        exec = slot;
    }
    int used = -1;
    for (int cyc = 1; cyc <= opts->sweep_max_cycles && rc == EIK_OK; ++cyc) {
        cudaError_t e = cudaMemsetAsync(t->sweep_flags, 0, 2 * SW_SLOTS * sizeof(unsigned int), st);
        if (e != cudaSuccess) { rc = cuda_fail(e, "memset", __FILE__, __LINE__); break; }
        if (exec) {
            e = cudaGraphLaunch(exec, st);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaGraphLaunch", __FILE__, __LINE__); break; }
        } else {
            rc = cycle(st);
            if (rc) break;
        }
        unsigned int h[2 * SW_SLOTS];
        e = cudaMemcpyAsync(h, t->sweep_flags, sizeof h, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = cuda_fail(e, "sweep sync", __FILE__, __LINE__); break; }
        float dmax = 0.f, xmax = 0.f;
        for (int q = 0; q < SW_SLOTS; ++q) {
            float a, c;
            std::memcpy(&a, &h[q], 4);
            std::memcpy(&c, &h[SW_SLOTS + q], 4);
            dmax = std::max(dmax, a);
            xmax = std::max(xmax, c);
        }
        if ((double)dmax <= opts->sweep_tol * (double)xmax) { used = cyc; break; }
    }
    if (rc) return rc;
    if (cycles) *cycles = used < 0 ? opts->sweep_max_cycles : used;
    if (used < 0) { set_error("sweeping did not converge in %d cycles", opts->sweep_max_cycles); return EIK_ERR_NOT_CONVERGED; }
    return EIK_OK;
}

}  // namespace eik
