// Cell-based velocity model (the inversion cells of Sec. 5.3, one per grid hexahedron):
// the node <- cell averaging map and its transpose.  With it a Jacobian action on cells
// is J_cells p = J (A_avg p) and J_cells^T y = A_avg^T (J^T y), J taking the tangent's
// velocity model map.  A node's perturbation is the mean over its adjacent cells (a
// reading; the paper gives no formula).  Cells are indexed like nodes on the grid of
// extents n_d - 1.  Both directions are gathers (no atomics), vectors [.][R] with the
// right-hand side fastest.
#include <cuda_runtime.h>

#include "eik_internal.h"

namespace eik {

struct CellGrid {
    int nd;
    int n[3];            // node extents
    long long nst[3];    // node strides
    long long cst[3];    // cell strides (extents n_d - 1)
};

static CellGrid make_cells(int ndim, const int *n)
{
    CellGrid c{};
    c.nd = ndim;
    long long sn = 1, sc = 1;
    for (int d = ndim - 1; d >= 0; --d) {
        c.n[d] = n[d];
        c.nst[d] = sn;
        c.cst[d] = sc;
        sn *= n[d];
        sc *= n[d] - 1;
    }
    return c;
}

__device__ __forceinline__ int n_adjacent(const CellGrid &C, const int *i)
{
    int k = 1;
    for (int d = 0; d < C.nd; ++d) k *= (i[d] > 0 && i[d] < C.n[d] - 1) ? 2 : 1;
    return k;
}

// p_node[j][r] = mean over the cells adjacent to node j of p_cell[c][r]
template <typename T>
__global__ void k_cells_to_nodes(CellGrid C, long long N, int R, const T *__restrict__ pc, T *__restrict__ pn)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= N * R) return;
    const long long j = t / R;
    const int r = (int)(t - j * R);
    int i[3] = {0, 0, 0};
    for (int d = 0; d < C.nd; ++d) i[d] = (int)((j / C.nst[d]) % C.n[d]);
    double acc = 0.0;
    for (int o = 0; o < (1 << C.nd); ++o) {
        long long c = 0;
        bool in = true;
        for (int d = 0; d < C.nd; ++d) {
            const int ci = i[d] - ((o >> d) & 1);
            in = in && ci >= 0 && ci <= C.n[d] - 2;
            c += (long long)ci * C.cst[d];
        }
        if (in) acc += (double)pc[c * R + r];
    }
    pn[t] = (T)(acc / n_adjacent(C, i));
}

// g_cell[c][r] = sum over the corner nodes j of cell c of g_node[j][r] / n_adj(j)
template <typename T>
__global__ void k_nodes_to_cells(CellGrid C, long long NC, int R, const T *__restrict__ gn, T *__restrict__ gc)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= NC * R) return;
    const long long c = t / R;
    const int r = (int)(t - c * R);
    int ci[3] = {0, 0, 0};
    for (int d = 0; d < C.nd; ++d) ci[d] = (int)((c / C.cst[d]) % (C.n[d] - 1));
    double acc = 0.0;
    for (int o = 0; o < (1 << C.nd); ++o) {
        int i[3] = {0, 0, 0};
        long long j = 0;
        for (int d = 0; d < C.nd; ++d) {
            i[d] = ci[d] + ((o >> d) & 1);
            j += (long long)i[d] * C.nst[d];
        }
        acc += (double)gn[j * R + r] / n_adjacent(C, i);
    }
    gc[t] = (T)acc;
}

template <typename T>
static int cells_map(int ndim, const int *n, const void *in, int R, void *out, bool to_nodes, cudaStream_t st)
{
    const CellGrid C = make_cells(ndim, n);
    long long N = 1, NC = 1;
    for (int d = 0; d < ndim; ++d) { N *= n[d]; NC *= n[d] - 1; }
    const long long work = (to_nodes ? N : NC) * R;
    const unsigned blocks = (unsigned)((work + 255) / 256);
    if (to_nodes) k_cells_to_nodes<T><<<blocks, 256, 0, st>>>(C, N, R, (const T *)in, (T *)out);
    else k_nodes_to_cells<T><<<blocks, 256, 0, st>>>(C, NC, R, (const T *)in, (T *)out);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

int cell_map(int ndim, const int *n, const void *in, int R, void *out, bool to_nodes, int dtype, cudaStream_t st)
{
    return dtype == EIK_F32 ? cells_map<float>(ndim, n, in, R, out, to_nodes, st)
                            : cells_map<double>(ndim, n, in, R, out, to_nodes, st);
}

static int cells_entry(const eik_grid *g, const void *in, int R, void *out, int dtype, bool to_nodes,
                       eik_stream stream)
{
    if (!g || (g->ndim != 2 && g->ndim != 3) || !in || !out || R <= 0 || (dtype != EIK_F32 && dtype != EIK_F64)) {
        set_error("bad model cell map arguments");
        return EIK_ERR_INVALID;
    }
    for (int d = 0; d < g->ndim; ++d)
        if (g->n[d] < 2) { set_error("grid needs >= 2 nodes per axis"); return EIK_ERR_INVALID; }
    return cell_map(g->ndim, g->n, in, R, out, to_nodes, dtype, (cudaStream_t)stream);
}

}  // namespace eik

extern "C" int model_cells_to_nodes(const eik_grid *g, const void *p_cell, int R, void *p_node, int dtype,
                                    eik_stream stream)
{
    return eik::cells_entry(g, p_cell, R, p_node, dtype, true, stream);
}

extern "C" int model_nodes_to_cells(const eik_grid *g, const void *g_node, int R, void *g_cell, int dtype,
                                    eik_stream stream)
{
    return eik::cells_entry(g, g_node, R, g_cell, dtype, false, stream);
}
