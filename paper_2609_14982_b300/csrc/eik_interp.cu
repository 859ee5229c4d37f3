// Off-grid receivers (Sec. 4.4's P_a for receivers between grid nodes): P_a samples the
// transported field multilinearly at each receiver's fractional logical position (a
// reading; the paper gives no formula), and P_a^T spreads receiver data onto the
// 2^ndim corner nodes with the same weights.  D_a = 0 for node sources; for point
// sources (eik_points.cu) a receiver in the source's cell is carried by D_a instead.
//   J:   traverse (receivers not fused), then gather each receiver's corners from the
//        canonical-order workspace through pos.
//   J^T: build the dense reverse input P^T y (a gather over the receivers touching each
//        node, no atomics), traverse it as a raw A^-T solve, then the source sum C^T M^T.
// Right-hand sides beyond rhs_chunk are processed in column chunks through a staging
// buffer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "eik_internal.h"

namespace eik {

// out[a][k][r] (row stride ld_out) = sum over corners of w * x_a[pos_a[node]][r]
template <typename T>
__global__ void k_ip_sample(int S, int n_ip, int K, long long N, int w, const int *__restrict__ ip_node,
                            const double *__restrict__ ip_w, const int *__restrict__ pos, const T *__restrict__ x,
                            T *__restrict__ out, long long ld_out)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)S * n_ip * w) return;
    const long long ar = t / w;
    const int r = (int)(t - ar * w);
    const long long a = ar / n_ip;
    double acc = 0.0;
    for (int c = 0; c < K; ++c) {
        const long long e = ar * K + c;
        const int node = ip_node[e];
        acc += ip_w[e] * (double)x[(a * N + pos[a * N + node]) * w + r];
    }
    out[ar * ld_out + r] = (T)acc;
}

// dense[a][node][r] = sum over the corner entries at node of w * y[a][receiver][r]
template <typename T>
__global__ void k_ip_spread(int S, int n_ip, int K, int n_ipt, long long N, int w, const int *__restrict__ ipt_node,
                            const int *__restrict__ ipt_ptr, const int *__restrict__ ipt_e, const double *__restrict__ ip_w,
                            const T *__restrict__ y, long long ld_y, T *__restrict__ dense)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)S * n_ipt * w) return;
    const long long at = t / w;
    const int r = (int)(t - at * w);
    const long long a = at / n_ipt;
    const int node = ipt_node[at];
    if (node < 0) return;
    const int *ptr = ipt_ptr + a * (n_ipt + 1) + (at - a * n_ipt);
    const int *ent = ipt_e + a * (long long)n_ip * K;
    const double *wa = ip_w + a * (long long)n_ip * K;
    double acc = 0.0;
    for (int q = ptr[0]; q < ptr[1]; ++q) {
        const int e = ent[q];
        acc += wa[e] * (double)y[(a * n_ip + e / K) * ld_y + r];
    }
    dense[(a * N + node) * w + r] = (T)acc;
}

static int ensure_ws_in(Tangent *t, size_t bytes)
{
    if (t->ws_in_bytes >= bytes) return EIK_OK;
    if (t->ws_in) cudaFree(t->ws_in);
    t->ws_in = nullptr;
    t->ws_in_bytes = 0;
    cudaError_t e = cudaMalloc(&t->ws_in, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (interp staging)", __FILE__, __LINE__);
    t->ws_in_bytes = bytes;
    return EIK_OK;
}

static int chunk_width(const Tangent *t, int R, int dtype)
{
    int Rc = R;
    if (t->opts.rhs_chunk > 0 && t->opts.rhs_chunk < R) {
        Rc = t->opts.rhs_chunk;
        const int unit = dtype == EIK_F32 ? 4 : 2;
        if (R % unit == 0) Rc = std::max(unit, Rc / unit * unit);
    }
    return Rc;
}

template <typename T>
static int apply_interp(Tangent *t, const void *ds, int shared, int R, void *d_rec, int dtype, cudaStream_t st)
{
    const long long N = t->N;
    const int S = t->S;
    const int Rc = chunk_width(t, R, dtype);
    const long long rows = shared ? N : N * S;
    if (Rc < R) {
        int rc = ensure_ws_in(t, (size_t)rows * Rc * sizeof(T));
        if (rc) return rc;
    }
    for (int r0 = 0; r0 < R; r0 += Rc) {
        const int w = std::min(Rc, R - r0);
        const void *in = ds;
        if (Rc < R) {   // this chunk's columns, packed [rows][w]
            EIK_CHECK(cudaMemcpy2DAsync(t->ws_in, w * sizeof(T), static_cast<const T *>(ds) + r0, R * sizeof(T),
                                        w * sizeof(T), rows, cudaMemcpyDeviceToDevice, st));
            in = t->ws_in;
        }
        int rc = traverse(t, false, MODE_J, in, shared, w, nullptr, nullptr, 0, dtype, st);
        if (rc) return rc;
        const long long n = (long long)S * t->n_ip * w;
        k_ip_sample<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S, t->n_ip, t->ip_k, N, w, t->ip_node, t->ip_w,
                                                                    t->pos, (const T *)t->ws_vec,
                                                                    static_cast<T *>(d_rec) + r0, (long long)R);
        EIK_CHECK_LAUNCH();
        if (t->pts.K > 0) {   // point sources: seed rows through z, and D for direct receivers
            rc = seed_add(t, t->n_ip, w, t->pts.ip_zeta, static_cast<T *>(d_rec) + r0, (long long)R, dtype, st);
            if (rc) return rc;
        }
    }
    return EIK_OK;
}

template <typename T>
static int apply_interp_T(Tangent *t, const void *y, int R, void *g, int dtype, cudaStream_t st)
{
    const long long N = t->N;
    const int S = t->S;
    const int Rc = chunk_width(t, R, dtype);
    int rc = ensure_ws_in(t, (size_t)S * N * Rc * sizeof(T));
    if (rc) return rc;
    for (int r0 = 0; r0 < R; r0 += Rc) {
        const int w = std::min(Rc, R - r0);
        EIK_CHECK(cudaMemsetAsync(t->ws_in, 0, (size_t)S * N * w * sizeof(T), st));
        const long long n = (long long)S * t->n_ipt * w;
        if (n > 0)
            k_ip_spread<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                S, t->n_ip, t->ip_k, t->n_ipt, N, w, t->ipt_node, t->ipt_ptr, t->ipt_e, t->ip_w,
                static_cast<const T *>(y) + r0, (long long)R, (T *)t->ws_in);
        EIK_CHECK_LAUNCH();
        rc = traverse(t, true, MODE_RAW, t->ws_in, 0, w, nullptr, nullptr, 0, dtype, st);
        if (rc) return rc;
        rc = source_sum(t, w, static_cast<T *>(g) + r0, (long long)R, dtype, st);
        if (rc) return rc;
        if (t->pts.K > 0) {   // point sources: M^T Phi^T (r . lam_seeds + rho . y_direct)
            rc = seed_scatter(t, w, static_cast<T *>(g) + r0, (long long)R, false, static_cast<const T *>(y) + r0,
                              (long long)R, t->n_ip, t->pts.ip_rho, dtype, st);
            if (rc) return rc;
        }
    }
    return EIK_OK;
}

int set_receivers_interp(Tangent *t, int n_rec, const double *f)
{
    const int nd = t->grid.ndim, S = t->S, K = 1 << nd;
    void *old[] = {t->ip_node, t->ip_w, t->ipt_node, t->ipt_ptr, t->ipt_e};
    for (void *p : old) if (p) cudaFree(p);
    t->ip_node = nullptr; t->ip_w = nullptr; t->ipt_node = nullptr; t->ipt_ptr = nullptr; t->ipt_e = nullptr;
    t->n_ip = 0; t->ip_k = K; t->n_ipt = 0;
    if (n_rec == 0) return EIK_OK;
    const size_t ne = (size_t)S * n_rec * K;
    std::vector<int> node(ne);
    std::vector<double> wt(ne);
    std::vector<double> rho((size_t)S * n_rec, -1.0);   // direct receivers of point sources
    long long stride[3] = {1, 1, 1};
    long long acc = 1;
    for (int d = nd - 1; d >= 0; --d) { stride[d] = acc; acc *= t->grid.n[d]; }
    for (size_t q = 0; q < (size_t)S * n_rec; ++q) {
        int base[3] = {0, 0, 0};
        double tt[3] = {0, 0, 0};
        for (int d = 0; d < nd; ++d) {
            const double fd = f[q * nd + d];
            if (!(fd >= 0.0 && fd <= t->grid.n[d] - 1)) {
                set_error("receiver %zu coordinate %d = %g outside [0, %d]", q % n_rec, d, fd, t->grid.n[d] - 1);
                return EIK_ERR_INVALID;
            }
            base[d] = std::min((int)std::floor(fd), t->grid.n[d] - 2);
            tt[d] = fd - base[d];
        }
        for (int c = 0; c < K; ++c) {
            double wv = 1.0;
            long long j = 0;
            for (int d = 0; d < nd; ++d) {
                const int o = (c >> (nd - 1 - d)) & 1;   // corner order: last axis fastest
                wv *= o ? tt[d] : 1.0 - tt[d];
                j += (long long)(base[d] + o) * stride[d];
            }
            node[q * K + c] = (int)j;
            wt[q * K + c] = wv;
        }
        if (t->pts.K > 0) {
            // D_a: a receiver inside its source's cell takes the source treatment's value
            // s_src |x_r - x_src| (its P row is zeroed); the corners of the two cells coincide
            const size_t a = q / n_rec;
            bool same = true;
            for (int d = 0; d < nd; ++d) same = same && base[d] == t->pts.base[a * 3 + d];
            if (same) {
                double xr[3] = {0.0, 0.0, 0.0};
                for (int c = 0; c < K; ++c)
                    for (int d = 0; d < nd; ++d) xr[d] = xr[d] + wt[q * K + c] * t->pts.corner_xyz[(a * 8 + c) * 3 + d];
                double acc = 0.0;
                for (int d = 0; d < nd; ++d) {
                    const double dd = xr[d] - t->pts.xs_host[a * 3 + d];
                    acc = acc + dd * dd;
                }
                rho[q] = std::sqrt(acc);
                for (int c = 0; c < K; ++c) wt[q * K + c] = 0.0;
            }
        }
    }
    // P^T: per source, the touched nodes ascending and their corner entries
    std::vector<std::vector<std::pair<int, int>>> bys(S);
    int n_ipt = 0;
    for (int a = 0; a < S; ++a) {
        auto &v = bys[a];
        v.reserve((size_t)n_rec * K);
        for (int e = 0; e < n_rec * K; ++e) v.emplace_back(node[(size_t)a * n_rec * K + e], e);
        std::sort(v.begin(), v.end());
        int u = 0;
        for (size_t k = 0; k < v.size(); ++k) u += (k == 0 || v[k].first != v[k - 1].first);
        n_ipt = std::max(n_ipt, u);
    }
    std::vector<int> tn((size_t)S * n_ipt, -1), tp((size_t)S * (n_ipt + 1), 0), te(ne);
    for (int a = 0; a < S; ++a) {
        const auto &v = bys[a];
        int u = -1;
        for (size_t k = 0; k < v.size(); ++k) {
            if (k == 0 || v[k].first != v[k - 1].first) {
                ++u;
                tn[(size_t)a * n_ipt + u] = v[k].first;
                tp[(size_t)a * (n_ipt + 1) + u] = (int)k;
            }
            te[(size_t)a * n_rec * K + k] = v[k].second;
        }
        for (int q = u + 1; q <= n_ipt; ++q) tp[(size_t)a * (n_ipt + 1) + q] = (int)v.size();
    }
    cudaError_t e = cudaMalloc((void **)&t->ip_node, ne * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&t->ip_w, ne * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&t->ipt_node, std::max<size_t>(tn.size(), 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&t->ipt_ptr, tp.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&t->ipt_e, ne * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(t->ip_node, node.data(), ne * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->ip_w, wt.data(), ne * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !tn.empty()) e = cudaMemcpy(t->ipt_node, tn.data(), tn.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->ipt_ptr, tp.data(), tp.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->ipt_e, te.data(), ne * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "tangent_set_receivers", __FILE__, __LINE__);
    t->n_ip = n_rec;
    t->n_ipt = n_ipt;
    if (t->pts.K > 0) return seed_interp_setup(t, rho, nullptr);
    return EIK_OK;
}

int apply_interp_entry(Tangent *t, const void *ds, int shared, int R, void *d_rec, int dtype, cudaStream_t st)
{
    if (t->n_ip == 0) { set_error("no off-grid receivers set (tangent_set_receivers)"); return EIK_ERR_INVALID; }
    return dtype == EIK_F32 ? apply_interp<float>(t, ds, shared, R, d_rec, dtype, st)
                            : apply_interp<double>(t, ds, shared, R, d_rec, dtype, st);
}

int apply_interp_T_entry(Tangent *t, const void *y, int R, void *g, int dtype, cudaStream_t st)
{
    if (t->n_ip == 0) { set_error("no off-grid receivers set (tangent_set_receivers)"); return EIK_ERR_INVALID; }
    return dtype == EIK_F32 ? apply_interp_T<float>(t, y, R, g, dtype, st)
                            : apply_interp_T<double>(t, y, R, g, dtype, st);
}

}  // namespace eik
