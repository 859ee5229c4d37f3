// Off-grid point sources: the source treatment behind the seed rows of Sec. 3.1-3.2 and
// the direct term D_a of Sec. 4.4 (Eq. source-jacobian, Eq. source-transpose).  The paper
// supplies the seed rows from a differentiated source treatment without printing it;
// this file implements one reading:
//   * a source sits at fractional logical coordinates f; its cell has corner base
//     b_d = min(floor(f_d), n_d - 2), local coordinates t = f - b, and corner q (axis 0
//     the most significant bit of q) the multilinear weight phi_q = prod_d (t_d or 1 - t_d);
//   * x_src = sum_q phi_q x_q and s_src = sum_q phi_q s_q; the state is the factored solve
//     with T0 = s_src |x - x_src|, every corner kept at T = s_src r_q, r_q = |x_q - x_src|;
//   * the corners are identity (seed) rows of A, and differentiating T_q = s_src r_q gives
//     their right-hand side q_q = r_q sum_k phi_k ds_k;
//   * an off-grid receiver inside the source cell is predicted by the source treatment
//     itself, T_r = s_src |x_r - x_src|: its row of P is zero and its row of D is
//     |x_r - x_src| phi.
// The traversal kernels are not touched.  A is linear, so the seed rows' contribution
// to J p is sigma_a z_a with sigma_a = sum_k phi_k (M p)_k and the fixed field
// z_a = A_a^-1 e_a (e_a = r on the seed rows), formed once per tangent; J^T y gains
// M^T Phi^T (sum_q r_q lam_q + sum_direct rho y).  Compiled with -fmad=false (the point
// data are the same IEEE sequence as in the state solve).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "eik_internal.h"

namespace eik {

// one thread per source: corners, weights, position, slowness and seed distances
__global__ void k_point_source(GridDesc g, int S, const double *__restrict__ xyz, const double *__restrict__ s,
                               const double *__restrict__ f, int *__restrict__ node, double *__restrict__ phi,
                               double *__restrict__ xs, double *__restrict__ ss, double *__restrict__ r,
                               double *__restrict__ cxyz)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= S) return;
    const int nd = g.ndim, K = 1 << nd;
    int base[3];
    double t[3];
    for (int d = 0; d < nd; ++d) {
        const double fd = f[a * 3 + d];
        base[d] = min((int)floor(fd), g.n[d] - 2);
        t[d] = fd - base[d];
    }
    double x[3] = {0.0, 0.0, 0.0};
    double sv = 0.0;
    for (int q = 0; q < K; ++q) {
        long long nq = 0;
        double w = 1.0;
        for (int d = 0; d < nd; ++d) {
            const int o = (q >> (nd - 1 - d)) & 1;
            nq = nq * g.n[d] + base[d] + o;
            w = w * (o ? t[d] : 1.0 - t[d]);
        }
        node[a * 8 + q] = (int)nq;
        phi[a * 8 + q] = w;
        for (int c = 0; c < 3; ++c) cxyz[(a * 8 + q) * 3 + c] = c < nd ? xyz[nq * nd + c] : 0.0;
        for (int c = 0; c < nd; ++c) x[c] = x[c] + w * xyz[nq * nd + c];
        sv = sv + w * s[nq];
    }
    for (int q = K; q < 8; ++q) { node[a * 8 + q] = -1; phi[a * 8 + q] = 0.0; r[a * 8 + q] = 0.0; }
    for (int c = 0; c < 3; ++c) xs[a * 3 + c] = c < nd ? x[c] : 0.0;
    ss[a] = sv;
    for (int q = 0; q < K; ++q) {
        const long long nq = node[a * 8 + q];
        double acc = 0.0;
        for (int c = 0; c < nd; ++c) {
            const double dd = xyz[nq * nd + c] - x[c];
            acc = acc + dd * dd;
        }
        r[a * 8 + q] = sqrt(acc);
    }
}

// phim = phi x the model factor at each corner (Sec. 2.3: 1, -s^2 or -s)
__global__ void k_point_phim(int S, int model, const int *__restrict__ node, const double *__restrict__ phi,
                             const double *__restrict__ s, double *__restrict__ phim)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= S * 8) return;
    const int k = node[e];
    if (k < 0) { phim[e] = 0.0; return; }
    const double si = s[k];
    const double m = model == EIK_MODEL_SLOWNESS ? 1.0 : (model == EIK_MODEL_VELOCITY ? -(si * si) : -si);
    phim[e] = phi[e] * m;
}

// e[a][node_q] = r_q (the seed rows' response to a unit source slowness change)
__global__ void k_seed_unit(int S, long long N, const int *__restrict__ node, const double *__restrict__ r,
                            double *__restrict__ e)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S * 8) return;
    const int k = node[i];
    if (k >= 0) e[(long long)(i / 8) * N + k] = r[i];
}

// zsel[a][j] = z[a][nodes[a][j]]
__global__ void k_gather_z(int S, int n, long long N, const int *__restrict__ nodes, const double *__restrict__ z,
                           double *__restrict__ out)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)S * n) return;
    const long long a = i / n;
    out[i] = z[a * N + nodes[i]];
}

// sigma[a][r] = sum_q phim_q in[row(node_q)][r]   (FP64, corner order)
template <typename T>
__global__ void k_seed_sigma(int S, int K, long long N, int w, const int *__restrict__ node,
                             const double *__restrict__ phim, const T *__restrict__ in, int shared_in, long long ld_in,
                             double *__restrict__ sigma)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S * w) return;
    const int a = i / w, r = i - a * w;
    const T *base = in + (shared_in ? 0 : (long long)a * N * ld_in);
    double acc = 0.0;
    for (int q = 0; q < K; ++q) acc = acc + phim[a * 8 + q] * (double)base[(long long)node[a * 8 + q] * ld_in + r];
    sigma[i] = acc;
}

// out[a][j][r] += sigma[a][r] * zeta[a][j]
template <typename T>
__global__ void k_seed_add(int S, long long n, int w, const double *__restrict__ sigma, const double *__restrict__ zeta,
                           T *__restrict__ out, long long ld)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)S * n * w) return;
    const long long aj = i / w;
    const int r = (int)(i - aj * w);
    const long long a = aj / n;
    T *o = out + aj * ld + r;
    *o = (T)((double)*o + sigma[a * w + r] * zeta[aj]);
}

// J^T: per column, in source order (deterministic):
//   tau_a = sum_q r_q lam_a[pos(node_q)] + sum_j rho_j y_a[j]   (rho_j < 0: not direct)
//   g[(a) node_q] += phim_q tau_a
template <typename T>
__global__ void k_seed_scatter(int S, int K, long long N, int w, const int *__restrict__ node,
                               const double *__restrict__ phim, const double *__restrict__ rq,
                               const int *__restrict__ pos, const T *__restrict__ lam, int n_y,
                               const double *__restrict__ rho, const T *__restrict__ y, long long ld_y,
                               T *__restrict__ g, long long ld_g, int per_source)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= w) return;
    for (int a = 0; a < S; ++a) {
        double tau = 0.0;
        for (int q = 0; q < K; ++q) {
            const int k = node[a * 8 + q];
            tau = tau + rq[a * 8 + q] * (double)lam[((long long)a * N + pos[(long long)a * N + k]) * w + r];
        }
        if (rho)
            for (int j = 0; j < n_y; ++j) {
                const double rj = rho[(long long)a * n_y + j];
                if (rj >= 0.0) tau = tau + rj * (double)y[((long long)a * n_y + j) * ld_y + r];
            }
        T *ga = g + (per_source ? (long long)a * N * ld_g : 0);
        for (int q = 0; q < K; ++q) {
            T *o = ga + (long long)node[a * 8 + q] * ld_g + r;
            *o = (T)((double)*o + phim[a * 8 + q] * tau);
        }
    }
}

// zeta of the interpolated receivers: rho for a direct receiver, else sum_k w_k z[node_k]
__global__ void k_ip_zeta(int S, int n_ip, int K, long long N, const int *__restrict__ ip_node,
                          const double *__restrict__ ip_w, const double *__restrict__ rho, const double *__restrict__ z,
                          double *__restrict__ zeta)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)S * n_ip) return;
    const long long a = i / n_ip;
    if (rho[i] >= 0.0) { zeta[i] = rho[i]; return; }
    double acc = 0.0;
    for (int c = 0; c < K; ++c) acc = acc + ip_w[i * K + c] * z[a * N + ip_node[i * K + c]];
    zeta[i] = acc;
}

static unsigned nblk(long long n) { return (unsigned)((n + 255) / 256); }

int point_sources(const GridDesc &g, const double *xyz, const double *s, int S, const double *f_host, PointData &pd,
                  cudaStream_t st)
{
    const int nd = g.ndim;
    for (int a = 0; a < S; ++a)
        for (int d = 0; d < nd; ++d) {
            const double v = f_host[a * nd + d];
            if (!(v >= 0.0 && v <= g.n[d] - 1)) {
                set_error("point source %d: coordinate %d = %g outside [0, %d]", a, d, v, g.n[d] - 1);
                return EIK_ERR_INVALID;
            }
        }
    std::vector<double> f3((size_t)S * 3, 0.0);
    for (int a = 0; a < S; ++a)
        for (int d = 0; d < nd; ++d) f3[(size_t)a * 3 + d] = f_host[a * nd + d];
    pd.S = S;
    pd.K = 1 << nd;
    pd.base.assign((size_t)S * 3, 0);
    for (int a = 0; a < S; ++a)
        for (int d = 0; d < nd; ++d) pd.base[(size_t)a * 3 + d] = std::min((int)std::floor(f3[(size_t)a * 3 + d]), g.n[d] - 2);
    cudaError_t e = cudaSuccess;
    auto get = [&](auto **p, size_t n) { if (e == cudaSuccess) e = cudaMalloc(p, std::max<size_t>(n, 1) * sizeof(**p)); };
    get(&pd.f, (size_t)S * 3);
    get(&pd.node, (size_t)S * 8);
    get(&pd.phi, (size_t)S * 8);
    get(&pd.phim, (size_t)S * 8);
    get(&pd.xs, (size_t)S * 3);
    get(&pd.ss, (size_t)S);
    get(&pd.r, (size_t)S * 8);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (point sources)", __FILE__, __LINE__);
    e = cudaMemcpyAsync(pd.f, f3.data(), f3.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__);
    double *cxyz = nullptr;
    EIK_CHECK(cudaMalloc(&cxyz, (size_t)S * 24 * sizeof(double)));
    k_point_source<<<nblk(S), 256, 0, st>>>(g, S, xyz, s, pd.f, pd.node, pd.phi, pd.xs, pd.ss, pd.r, cxyz);
    e = cudaGetLastError();
    pd.xs_host.resize((size_t)S * 3);
    pd.corner_xyz.resize((size_t)S * 24);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pd.xs_host.data(), pd.xs, (size_t)S * 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pd.corner_xyz.data(), cxyz, (size_t)S * 24 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(cxyz);
    if (e != cudaSuccess) return cuda_fail(e, "point sources", __FILE__, __LINE__);
    return EIK_OK;
}

void free_point_data(PointData &pd)
{
    void *p[] = {pd.f, pd.node, pd.phi, pd.phim, pd.xs, pd.ss, pd.r, pd.z, pd.zrec, pd.sigma, pd.ip_rho, pd.ip_zeta};
    for (void *q : p) if (q) cudaFree(q);
    pd = PointData{};
}

int point_tangent_setup(Tangent *t, const double *s, cudaStream_t st)
{
    PointData &pd = t->pts;
    const long long N = t->N;
    const int S = t->S;
    k_point_phim<<<nblk(S * 8), 256, 0, st>>>(S, t->model, pd.node, pd.phi, s, pd.phim);
    EIK_CHECK_LAUNCH();
    // z_a = A_a^-1 e_a, e_a = r on the seed rows (FP64 raw forward solve)
    double *e = nullptr;
    EIK_CHECK(cudaMalloc(&pd.z, (size_t)S * N * sizeof(double)));
    EIK_CHECK(cudaMalloc(&e, (size_t)S * N * sizeof(double)));
    int rc = EIK_OK;
    cudaError_t ce = cudaMemsetAsync(e, 0, (size_t)S * N * sizeof(double), st);
    if (ce == cudaSuccess) {
        k_seed_unit<<<nblk(S * 8), 256, 0, st>>>(S, N, pd.node, pd.r, e);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) rc = cuda_fail(ce, "seed right-hand side", __FILE__, __LINE__);
    if (!rc) rc = traverse(t, false, MODE_RAW, e, 0, 1, pd.z, nullptr, 0, EIK_F64, st);
    if (!rc) {
        ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) rc = cuda_fail(ce, "cudaStreamSynchronize", __FILE__, __LINE__);
    }
    cudaFree(e);
    if (rc) return rc;
    if (t->n_rec > 0) {
        EIK_CHECK(cudaMalloc(&pd.zrec, (size_t)S * t->n_rec * sizeof(double)));
        k_gather_z<<<nblk((long long)S * t->n_rec), 256, 0, st>>>(S, t->n_rec, N, t->rec_nat, pd.z, pd.zrec);
        EIK_CHECK_LAUNCH();
    }
    return EIK_OK;
}

static int ensure_sigma(PointData &pd, int w)
{
    if (pd.sigma_cols >= w) return EIK_OK;
    if (pd.sigma) cudaFree(pd.sigma);
    pd.sigma = nullptr;
    pd.sigma_cols = 0;
    EIK_CHECK(cudaMalloc(&pd.sigma, (size_t)pd.S * w * sizeof(double)));
    pd.sigma_cols = w;
    return EIK_OK;
}

int seed_sigma(Tangent *t, const void *in, int shared_in, long long ld_in, int w, int dtype, cudaStream_t st)
{
    PointData &pd = t->pts;
    int rc = ensure_sigma(pd, w);
    if (rc) return rc;
    const int n = t->S * w;
    if (dtype == EIK_F32)
        k_seed_sigma<float><<<nblk(n), 256, 0, st>>>(t->S, pd.K, t->N, w, pd.node, pd.phim, (const float *)in, shared_in,
                                                     ld_in, pd.sigma);
    else
        k_seed_sigma<double><<<nblk(n), 256, 0, st>>>(t->S, pd.K, t->N, w, pd.node, pd.phim, (const double *)in,
                                                      shared_in, ld_in, pd.sigma);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

int seed_add(Tangent *t, long long n, int w, const double *zeta, void *out, long long ld, int dtype, cudaStream_t st)
{
    const long long tot = (long long)t->S * n * w;
    if (tot == 0) return EIK_OK;
    if (dtype == EIK_F32)
        k_seed_add<float><<<nblk(tot), 256, 0, st>>>(t->S, n, w, t->pts.sigma, zeta, (float *)out, ld);
    else
        k_seed_add<double><<<nblk(tot), 256, 0, st>>>(t->S, n, w, t->pts.sigma, zeta, (double *)out, ld);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

int seed_scatter(Tangent *t, int w, void *g, long long ld_g, bool per_source, const void *y, long long ld_y,
                 int n_y, const double *rho, int dtype, cudaStream_t st)
{
    PointData &pd = t->pts;
    const unsigned blocks = (unsigned)((w + 63) / 64);
    if (dtype == EIK_F32)
        k_seed_scatter<float><<<blocks, 64, 0, st>>>(t->S, pd.K, t->N, w, pd.node, pd.phim, pd.r, t->pos,
                                                    (const float *)lane_ws(t, true), n_y, rho, (const float *)y, ld_y,
                                                    (float *)g, ld_g, per_source ? 1 : 0);
    else
        k_seed_scatter<double><<<blocks, 64, 0, st>>>(t->S, pd.K, t->N, w, pd.node, pd.phim, pd.r, t->pos,
                                                     (const double *)lane_ws(t, true), n_y, rho, (const double *)y, ld_y,
                                                     (double *)g, ld_g, per_source ? 1 : 0);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

int seed_interp_setup(Tangent *t, const std::vector<double> &rho_host, cudaStream_t st)
{
    PointData &pd = t->pts;
    if (pd.ip_rho) cudaFree(pd.ip_rho);
    if (pd.ip_zeta) cudaFree(pd.ip_zeta);
    pd.ip_rho = pd.ip_zeta = nullptr;
    const long long n = (long long)t->S * t->n_ip;
    if (n == 0) return EIK_OK;
    EIK_CHECK(cudaMalloc(&pd.ip_rho, n * sizeof(double)));
    EIK_CHECK(cudaMalloc(&pd.ip_zeta, n * sizeof(double)));
    EIK_CHECK(cudaMemcpyAsync(pd.ip_rho, rho_host.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    k_ip_zeta<<<nblk(n), 256, 0, st>>>(t->S, t->n_ip, t->ip_k, t->N, t->ip_node, t->ip_w, pd.ip_rho, pd.z, pd.ip_zeta);
    EIK_CHECK_LAUNCH();
    EIK_CHECK(cudaStreamSynchronize(st));
    return EIK_OK;
}

}  // namespace eik
