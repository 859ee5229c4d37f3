// Launch parameters of the block traversals and the device helpers that every traversal
// schedule shares (device code only; not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include "eik_internal.h"
#include "eik_vec.cuh"

namespace eik {

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
    const double *lu;      // block LU factors (P A_C = L U, rows swapped in place) and pivots
    const int *piv;
    int blk_lu_min;        // blocks of at least this size use the LU substitution (0: never)
    double *ws;
    unsigned long long timeout_ns;
    // cluster schedule: [S][maxL+1] first position / first block of each level, [S] level
    // counts, [S] sources in the order clusters take them
    const int *lvl;
    const int *blk_lvl;
    const int *nlev;
    const int *order;
};

constexpr int MAX_ROW = 6;   // at most 2 * ndim faces per row

// Checked build (compiled with -DEIK_CHECKED, the library's debug mode in place of a
// sanitizer): before a position is computed, its node, its row's edge range in the staged
// arrays, every upstream position and its receiver slot are checked against their arrays;
// a bad one latches DEV_BAD_INDEX {source, position, value} and the position is skipped.
// The normal build compiles the check away.
#ifdef EIK_CHECKED
static __device__ __noinline__ bool position_ok(const TravParams &P, long long a, int pos, int v, int e0, int cnt, int staged,
                                         const int *en, int rec)
{
    long long bad = -1;
    if (v < 0 || v >= P.N) bad = v;
    else if (e0 < 0 || cnt < 0 || cnt > MAX_ROW || (staged >= 0 && e0 + cnt > staged)) bad = e0 + cnt;
    else if (rec >= P.n_rec) bad = rec;
    else
        for (int e = 0; e < cnt; ++e)
            if (en[e0 + e] < 0 || en[e0 + e] >= P.N) { bad = en[e0 + e]; break; }
    if (bad < 0) return true;
    if (atomicCAS(P.err, 0, DEV_BAD_INDEX) == 0) { P.err[1] = (int)a; P.err[2] = pos; P.err[3] = (int)bad; }
    return false;
}
#define EIK_POSITION_OK(P, a, pos, v, e0, cnt, staged, en, rec) position_ok(P, a, pos, v, e0, cnt, staged, en, rec)
#else
#define EIK_POSITION_OK(P, a, pos, v, e0, cnt, staged, en, rec) true
#endif

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

// the traversal launch of the level-synchronous schedule (eik_sync.cu)
int launch_sync(Tangent *t, const TravParams &P, int esz, int V, bool TR, cudaStream_t st);

}  // namespace eik
