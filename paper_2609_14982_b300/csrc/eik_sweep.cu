// The plain form the block traversal is compared with: directional sweeping of the
// same frozen operator (Sec. 3.6), i.e. Gauss-Seidel over the 2^ndim logical
// orderings, cycled to a tolerance.  On the device each ordering is run hyperplane by
// hyperplane: with the axis directions of ordering o, the nodes of one hyperplane
// sum_d i'_d = h depend only on hyperplanes h-1 (already updated) and h+1 (old
// values), which reproduces the lexicographic Gauss-Seidel sweep exactly.  All
// sources and right-hand sides of a hyperplane are updated in one launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "eik_internal.h"

namespace eik {

struct SweepParams {
    GridDesc g;
    int S, R, transpose, order, h;
    int lo0, hi0;                 // range of the first logical coordinate on the hyperplane
    const int *cnt, *nnode;       // natural full rows [S][N], [S][N][2 ndim]
    const double *nw;
    const void *b;
    void *x;
    unsigned int *dmax, *xmax;    // float bit patterns of max |dx|, max |x| (non-negative)
};

template <typename T>
__global__ void k_sweep_plane(SweepParams P)
{
    const GridDesc &g = P.g;
    const int nd = g.ndim, slots = 2 * nd;
    long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int n1 = g.n[1], n2 = nd == 3 ? g.n[2] : 1;
    const long long span = (long long)(P.hi0 - P.lo0 + 1) * (nd == 3 ? n1 : 1);
    const long long per_src = span * P.R;
    if (tid >= per_src * P.S) return;
    const int a = (int)(tid / per_src);
    long long rem = tid - a * per_src;
    const int r = (int)(rem % P.R);
    long long cell = rem / P.R;
    int c0, c1, c2;
    if (nd == 3) {
        c0 = P.lo0 + (int)(cell / n1);
        c1 = (int)(cell % n1);
        c2 = P.h - c0 - c1;
        if (c2 < 0 || c2 >= n2) return;
    } else {
        c0 = P.lo0 + (int)cell;
        c1 = P.h - c0;
        c2 = 0;
        if (c1 < 0 || c1 >= n1) return;
    }
    // undo the axis reversals of this ordering
    int i0 = (P.order & 1) ? g.n[0] - 1 - c0 : c0;
    int i1 = (P.order & 2) ? n1 - 1 - c1 : c1;
    int i2 = (P.order & 4) ? n2 - 1 - c2 : c2;
    long long i = nd == 3 ? ((long long)i0 * n1 + i1) * n2 + i2 : (long long)i0 * n1 + i1;
    const long long N = g.N, base = (long long)a * N;
    const T *b = reinterpret_cast<const T *>(P.b) + base * P.R;
    T *x = reinterpret_cast<T *>(P.x) + base * P.R;
    double acc = (double)b[i * P.R + r];
    if (!P.transpose) {
        const long long v = base + i;
        for (int e = 0; e < P.cnt[v]; ++e)
            acc += P.nw[v * slots + e] * (double)x[(long long)P.nnode[v * slots + e] * P.R + r];
    } else {
        int c[3] = {i0, i1, i2};
        for (int d = 0; d < nd; ++d)
            for (int side = -1; side <= 1; side += 2) {
                int at = c[d] + side;
                if (at < 0 || at >= g.n[d]) continue;
                long long u = i + side * g.st[d];
                long long vu = base + u;
                for (int e = 0; e < P.cnt[vu]; ++e)
                    if (P.nnode[vu * slots + e] == (int)i) acc += P.nw[vu * slots + e] * (double)x[u * P.R + r];
            }
    }
    T nv = (T)acc;
    float dx = fabsf((float)((double)nv - (double)x[i * P.R + r]));
    x[i * P.R + r] = nv;
    float ax = fabsf((float)nv);
    atomicMax(P.dmax, __float_as_uint(dx));
    atomicMax(P.xmax, __float_as_uint(ax));
}

int sweep(Tangent *t, bool transpose, const void *b, int R, void *x, int dtype, const eik_opts *opts, int *cycles,
          cudaStream_t st)
{
    if (dtype != EIK_F32 && dtype != EIK_F64) { set_error("bad dtype"); return EIK_ERR_INVALID; }
    const GridDesc &g = t->grid;
    const size_t esz = dtype == EIK_F32 ? 4 : 8;
    EIK_CHECK(cudaMemsetAsync(x, 0, (size_t)t->S * t->N * R * esz, st));
    unsigned int *flags;
    EIK_CHECK(cudaMalloc(&flags, 2 * sizeof(unsigned int)));
    SweepParams P{};
    P.g = g; P.S = t->S; P.R = R; P.transpose = transpose;
    P.cnt = t->nrow_cnt; P.nnode = t->nrow_node; P.nw = t->nrow_w;
    P.b = b; P.x = x; P.dmax = flags; P.xmax = flags + 1;
    const int nd = g.ndim;
    const int nord = 1 << nd;
    int hmax = 0;
    for (int d = 0; d < nd; ++d) hmax += g.n[d] - 1;
    int used = -1;
    int rc = EIK_OK;
    for (int cyc = 1; cyc <= opts->sweep_max_cycles; ++cyc) {
        cudaError_t e = cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned int), st);
        if (e != cudaSuccess) { rc = cuda_fail(e, "memset", __FILE__, __LINE__); break; }
        for (int o = 0; o < nord; ++o) {
            P.order = o;
            for (int h = 0; h <= hmax; ++h) {
                int rest = hmax - (g.n[0] - 1);
                P.h = h;
                P.lo0 = std::max(0, h - rest);
                P.hi0 = std::min(g.n[0] - 1, h);
                long long span = (long long)(P.hi0 - P.lo0 + 1) * (nd == 3 ? g.n[1] : 1);
                long long n = span * R * t->S;
                unsigned blocks = (unsigned)((n + 255) / 256);
                if (dtype == EIK_F32) k_sweep_plane<float><<<blocks, 256, 0, st>>>(P);
                else k_sweep_plane<double><<<blocks, 256, 0, st>>>(P);
            }
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) { rc = cuda_fail(e, "sweep launch", __FILE__, __LINE__); break; }
        unsigned int h[2];
        e = cudaMemcpyAsync(h, flags, sizeof h, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = cuda_fail(e, "sweep sync", __FILE__, __LINE__); break; }
        float dmax, xmax;
        std::memcpy(&dmax, &h[0], 4);
        std::memcpy(&xmax, &h[1], 4);
        if ((double)dmax <= opts->sweep_tol * (double)xmax) { used = cyc; break; }
    }
    cudaFree(flags);
    if (rc) return rc;
    if (cycles) *cycles = used;
    if (used < 0) { set_error("sweeping did not converge in %d cycles", opts->sweep_max_cycles); return EIK_ERR_NOT_CONVERGED; }
    return EIK_OK;
}

}  // namespace eik
