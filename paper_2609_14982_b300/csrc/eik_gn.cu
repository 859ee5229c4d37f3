// The augmented Gauss-Newton operator of Sec. 4.5 (Eq. augmented-ls, Eq.
// augmented-actions) on a built tangent, and LSMR (Fong and Saunders, 2011) on it with
// every vector operation and scalar on the device (one iteration can be captured in a
// CUDA graph):
//   K p   = [ W_d J p ; lam R p ; lam S p ],              S = gamma diag(1 / v_k)
//   K^T y = J^T W_d y_d + lam R^T y_R + lam S^T y_S.
// One model vector (R = 1 right-hand side).  J and J^T are the stored block traversals;
// W_d, R and S are applied in the epilogues of the Krylov vector updates, so a K p or
// K^T y costs one traversal plus one pass over the K-space vector.
// R (not defined in the paper): unit first differences along every logical axis,
// (R p)_row = p[i + e_d] - p[i]; rows axis by axis, within an axis in the linear order of
// the lower node i.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "eik_internal.h"
#include "eik_krylov.h"

namespace eik {

// logical grid for R: extents and strides (natural node order, last axis fastest)
struct RoughGrid {
    int nd;
    int n[3];
    long long stride[3];
    long long r0[4];      // first row of each axis block; r0[nd] = number of rows
};

static RoughGrid make_rough(const GridDesc &g)
{
    RoughGrid r{};
    r.nd = g.ndim;
    for (int d = 0; d < g.ndim; ++d) r.n[d] = g.n[d];
    long long st = 1;
    for (int d = g.ndim - 1; d >= 0; --d) { r.stride[d] = st; st *= g.n[d]; }
    r.r0[0] = 0;
    for (int d = 0; d < g.ndim; ++d) {
        long long c = 1;
        for (int e = 0; e < g.ndim; ++e) c *= (e == d ? g.n[e] - 1 : g.n[e]);
        r.r0[d + 1] = r.r0[d] + c;
    }
    return r;
}

// lower node of row q (0 <= q < rows of axis d): the rows of axis d enumerate, in natural
// order, the nodes with i_d <= n_d - 2, i.e. a grid whose extent along d is n_d - 1
__device__ __forceinline__ long long rough_lower(const RoughGrid &R, int d, long long q)
{
    long long node = 0;
    for (int e = R.nd - 1; e >= 0; --e) {
        const long long m = e == d ? R.n[e] - 1 : R.n[e];
        const long long i = q % m;
        q /= m;
        node += i * R.stride[e];
    }
    return node;
}

// row of axis d whose lower node is `node` (requires i_d <= n_d - 2)
__device__ __forceinline__ long long rough_row(const RoughGrid &R, int d, long long node)
{
    long long q = 0;
    for (int e = 0; e < R.nd; ++e) {
        const long long i = (node / R.stride[e]) % R.n[e];
        const long long m = e == d ? R.n[e] - 1 : R.n[e];
        q = q * m + i;
    }
    return R.r0[d] + q;
}

// K-space vector out = K p (given Jp at the receivers), or, with coef_slot >= 0,
// u = K p - sc[coef_slot] * u; partial[block] = sum of squares of the result
template <typename T>
__global__ void k_gn_forward(long long nd, long long N, RoughGrid R, double lam, const double *__restrict__ wd,
                             const double *__restrict__ sdiag, const T *__restrict__ jp, const T *__restrict__ p,
                             T *__restrict__ u, const double *sc, int coef_slot, double *partial)
{
    __shared__ double red[LB];
    const long long nR = R.r0[R.nd], n = nd + nR + N;
    const bool axpby = coef_slot >= 0;
    const double coef = axpby ? sc[coef_slot] : 0.0;
    double acc = 0.0;
    for (long long e = blockIdx.x * (long long)LB + threadIdx.x; e < n; e += (long long)gridDim.x * LB) {
        double kv;
        if (e < nd) {
            kv = wd[e] * (double)jp[e];
        } else if (e < nd + nR) {
            const long long q = e - nd;
            int d = 0;
            while (q >= R.r0[d + 1]) ++d;
            const long long lo = rough_lower(R, d, q - R.r0[d]);
            kv = lam * ((double)p[lo + R.stride[d]] - (double)p[lo]);
        } else {
            const long long j = e - nd - nR;
            kv = lam * sdiag[j] * (double)p[j];
        }
        const double val = axpby ? kv - coef * (double)u[e] : kv;
        const T tv = (T)val;
        u[e] = tv;
        acc += (double)tv * (double)tv;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = LB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (partial && threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// yw = W_d y_d (the data block, weighted for the transpose traversal)
template <typename T>
__global__ void k_gn_weight(long long nd, const double *__restrict__ wd, const T *__restrict__ y, T *__restrict__ yw)
{
    for (long long e = blockIdx.x * (long long)LB + threadIdx.x; e < nd; e += (long long)gridDim.x * LB)
        yw[e] = (T)(wd[e] * (double)y[e]);
}

// model vector out = g + lam R^T y_R + lam S y_S (g = J^T W_d y_d from the traversal), or
// with coef_slot >= 0, v = that - sc[coef_slot] * v; partial sums of squares as above.
// R^T is gathered per node (no atomics): + y of the row where the node is upper, - y of
// the row where it is lower, axis by axis.
template <typename T>
__global__ void k_gn_transpose(long long nd, long long N, RoughGrid R, double lam, const double *__restrict__ sdiag,
                               const T *__restrict__ g, const T *__restrict__ y, T *__restrict__ v, const double *sc,
                               int coef_slot, double *partial)
{
    __shared__ double red[LB];
    const long long nR = R.r0[R.nd];
    const T *yR = y + nd, *yS = y + nd + nR;
    const bool axpby = coef_slot >= 0;
    const double coef = axpby ? sc[coef_slot] : 0.0;
    double acc = 0.0;
    for (long long j = blockIdx.x * (long long)LB + threadIdx.x; j < N; j += (long long)gridDim.x * LB) {
        double rt = 0.0;
        for (int d = 0; d < R.nd; ++d) {
            const long long i = (j / R.stride[d]) % R.n[d];
            if (i > 0) rt += (double)yR[rough_row(R, d, j - R.stride[d])];
            if (i < R.n[d] - 1) rt -= (double)yR[rough_row(R, d, j)];
        }
        const double kt = (double)g[j] + lam * rt + lam * sdiag[j] * (double)yS[j];
        const double val = axpby ? kt - coef * (double)v[j] : kt;
        const T tv = (T)val;
        v[j] = tv;
        acc += (double)tv * (double)tv;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = LB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (partial && threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_gn_sdiag(long long N, double gamma, const double *__restrict__ vk, double *__restrict__ sdiag)
{
    for (long long j = blockIdx.x * (long long)LB + threadIdx.x; j < N; j += (long long)gridDim.x * LB)
        sdiag[j] = gamma / vk[j];
}

// ---------------------------------------------------------------- LSMR state on the device
// Slots of the scalar array (names follow Fong and Saunders' recurrences).
enum {
    M_ALPHA = 0, M_BETA, M_ALPHABAR, M_ZETABAR, M_RHO, M_RHOBAR, M_CBAR, M_SBAR, M_ZETA,
    M_BETADD, M_BETAD, M_RHODOT, M_THETATILDE, M_TAUTILDE, M_DONE2, M_NORMA2,
    M_NORMR, M_NORMX, M_NORMB,
    M_CHBAR, M_CX, M_CH,          // coefficients of the vector updates of the step
    M_NSCAL = 32
};

// start: beta_1 and alpha_1 are in their slots (b normalised, v = A^T u normalised)
__global__ void k_m_start(double *sc)
{
    const double alpha = sc[M_ALPHA], beta = sc[M_BETA];
    sc[M_ALPHABAR] = alpha;
    sc[M_ZETABAR] = alpha * beta;
    sc[M_RHO] = 1.0;
    sc[M_RHOBAR] = 1.0;
    sc[M_CBAR] = 1.0;
    sc[M_SBAR] = 0.0;
    sc[M_ZETA] = 0.0;
    sc[M_BETADD] = beta;
    sc[M_BETAD] = 0.0;
    sc[M_RHODOT] = 1.0;
    sc[M_THETATILDE] = 0.0;
    sc[M_TAUTILDE] = 0.0;
    sc[M_DONE2] = 0.0;
    sc[M_NORMA2] = alpha * alpha;
    sc[M_NORMR] = beta;
    sc[M_NORMB] = beta;
    sc[M_NORMX] = 0.0;
}

__device__ __forceinline__ double safe_div(double a, double b) { return b != 0.0 ? a / b : 0.0; }

// one step of the rotations, given beta_{k+1} and alpha_{k+1} in their slots:
// P_k on B_k, Pbar_k on [R_k^T; theta e_k^T], the coefficients of the h / hbar / x
// updates, and Ptilde_{k-1} with the forward substitution that carries |r_k|
__global__ void k_m_step(double *sc)
{
    const double alpha = sc[M_ALPHA], beta = sc[M_BETA];
    sc[M_NORMA2] += beta * beta + alpha * alpha;
    // P_k
    const double alphabar = sc[M_ALPHABAR];
    const double rho_prev = sc[M_RHO];
    const double rho = hypot(alphabar, beta);
    const double c = safe_div(alphabar, rho), s = safe_div(beta, rho);
    const double theta = s * alpha;
    sc[M_ALPHABAR] = c * alpha;
    // Pbar_k
    const double rhobar_prev = sc[M_RHOBAR], zeta_prev = sc[M_ZETA];
    const double cbar_prev = sc[M_CBAR], sbar_prev = sc[M_SBAR], zetabar = sc[M_ZETABAR];
    const double thetabar = sbar_prev * rho;
    const double rhobar = hypot(cbar_prev * rho, theta);
    const double cbar = safe_div(cbar_prev * rho, rhobar), sbar = safe_div(theta, rhobar);
    const double zeta = cbar * zetabar;
    sc[M_ZETABAR] = -sbar * zetabar;
    sc[M_RHO] = rho;
    sc[M_RHOBAR] = rhobar;
    sc[M_CBAR] = cbar;
    sc[M_SBAR] = sbar;
    sc[M_ZETA] = zeta;
    // hbar = h - chbar hbar ; x += cx hbar ; h = v - ch h
    sc[M_CHBAR] = safe_div(thetabar * rho, rho_prev * rhobar_prev);
    sc[M_CX] = safe_div(zeta, rho * rhobar);
    sc[M_CH] = safe_div(theta, rho);
    // |r_k|: P_k on the rotated right-hand side, then Ptilde_{k-1}
    const double betadd = sc[M_BETADD];
    const double betahat = c * betadd;
    sc[M_BETADD] = -s * betadd;
    const double rhodot = sc[M_RHODOT], betad = sc[M_BETAD];
    const double rhotilde = hypot(rhodot, thetabar);
    const double ctilde = safe_div(rhodot, rhotilde), stilde = safe_div(thetabar, rhotilde);
    const double thetatilde_prev = sc[M_THETATILDE];
    const double thetatilde = stilde * rhobar;
    const double rhodot_new = ctilde * rhobar;
    const double betatilde = ctilde * betad + stilde * betahat;
    const double betad_new = -stilde * betad + ctilde * betahat;
    const double tautilde = safe_div(zeta_prev - thetatilde_prev * sc[M_TAUTILDE], rhotilde);
    const double taudot = safe_div(zeta - thetatilde * tautilde, rhodot_new);
    const double done2 = sc[M_DONE2] + (betatilde - tautilde) * (betatilde - tautilde);
    sc[M_THETATILDE] = thetatilde;
    sc[M_RHODOT] = rhodot_new;
    sc[M_BETAD] = betad_new;
    sc[M_TAUTILDE] = tautilde;
    sc[M_DONE2] = done2;
    const double bdd = sc[M_BETADD];
    sc[M_NORMR] = sqrt(done2 + (betad_new - taudot) * (betad_new - taudot) + bdd * bdd);
}

// hbar = h - chbar hbar ; x = x + cx hbar ; h = v - ch h ; partial sums of x^2
template <typename T>
__global__ void k_m_update(long long n, T *__restrict__ x, T *__restrict__ h, T *__restrict__ hbar,
                           const T *__restrict__ v, const double *sc, double *partial)
{
    __shared__ double red[LB];
    const double chbar = sc[M_CHBAR], cx = sc[M_CX], ch = sc[M_CH];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)LB + threadIdx.x; i < n; i += (long long)gridDim.x * LB) {
        const double hi = (double)h[i];
        const T hb = (T)(hi - chbar * (double)hbar[i]);
        hbar[i] = hb;
        const T xi = (T)((double)x[i] + cx * (double)hb);
        x[i] = xi;
        h[i] = (T)((double)v[i] - ch * hi);
        acc += (double)xi * (double)xi;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int hh = LB / 2; hh > 0; hh >>= 1) {
        if (threadIdx.x < hh) red[threadIdx.x] += red[threadIdx.x + hh];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

}  // namespace eik

using namespace eik;

struct eik_tangent { Tangent *impl; };

struct eik_gn {
    eik_tangent *t = nullptr;
    int dtype = EIK_F64;
    int cells = 0;                 // model on the cells (one per grid hexahedron), not the nodes
    long long N = 0, nd = 0, nR = 0, n_rows = 0;   // N: model size (nodes or cells)
    void *pn = nullptr, *gc = nullptr;             // cells: node-space input of J, cell-space J^T
    RoughGrid R{};
    double lam = 0.0, gamma = 0.0;
    double *wd = nullptr, *sdiag = nullptr;                 // device copies of W_d and gamma / v_k
    void *u = nullptr, *v = nullptr, *h = nullptr, *hbar = nullptr, *x = nullptr;
    void *jp = nullptr, *yw = nullptr, *g = nullptr;       // J v at receivers, W_d u_d, J^T W_d u_d
    double *sc = nullptr, *partial = nullptr;
    int nb_rows = 1, nb_model = 1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int iters = 0;
};

namespace {

int nblocks(long long n)
{
    long long b = (n + LB - 1) / LB;
    return (int)(b < 1 ? 1 : (b < LMAXB ? b : LMAXB));
}

// K p into out (coef_slot < 0) or u = K p - sc[coef] u with partial sums
template <typename T>
int gn_forward(eik_gn *G, const void *p, void *out, int coef_slot, double *partial, cudaStream_t st)
{
    const void *pj = p;
    if (G->cells) {   // J acts on the nodal perturbation A p
        const GridDesc &gd = G->t->impl->grid;
        int rc = cell_map(gd.ndim, gd.n, p, 1, G->pn, true, G->dtype, st);
        if (rc) return rc;
        pj = G->pn;
    }
    int rc = traverse(G->t->impl, false, MODE_J, pj, 1, 1, nullptr, G->jp, 0, G->dtype, st);
    if (rc) return rc;
    k_gn_forward<T><<<G->nb_rows, LB, 0, st>>>(G->nd, G->N, G->R, G->lam, G->wd, G->sdiag, (const T *)G->jp,
                                               (const T *)p, (T *)out, G->sc, coef_slot, partial);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

// K^T y into out (coef_slot < 0) or v = K^T y - sc[coef] v with partial sums
template <typename T>
int gn_transpose(eik_gn *G, const void *y, void *out, int coef_slot, double *partial, cudaStream_t st)
{
    k_gn_weight<T><<<nblocks(G->nd), LB, 0, st>>>(G->nd, G->wd, (const T *)y, (T *)G->yw);
    EIK_CHECK_LAUNCH();
    int rc = traverse(G->t->impl, true, MODE_J, G->yw, 0, 1, nullptr, G->g, 1, G->dtype, st);
    if (rc) return rc;
    const void *gm = G->g;
    if (G->cells) {   // A^T (J^T W_d y_d)
        const GridDesc &gd = G->t->impl->grid;
        rc = cell_map(gd.ndim, gd.n, G->g, 1, G->gc, false, G->dtype, st);
        if (rc) return rc;
        gm = G->gc;
    }
    k_gn_transpose<T><<<G->nb_model, LB, 0, st>>>(G->nd, G->N, G->R, G->lam, G->sdiag, (const T *)gm,
                                                  (const T *)y, (T *)out, G->sc, coef_slot, partial);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

template <typename T>
int lsmr_begin(eik_gn *G, const void *b, cudaStream_t st)
{
    const size_t es = sizeof(T);
    EIK_CHECK(cudaMemcpyAsync(G->u, b, G->n_rows * es, cudaMemcpyDeviceToDevice, st));
    // beta_1 u_1 = b
    k_l_axpby_sq<T><<<G->nb_rows, LB, 0, st>>>(G->n_rows, (const T *)G->u, (T *)G->u, G->sc, -1, 0.0, G->partial);
    k_l_norm<<<1, LB, 0, st>>>(G->partial, G->nb_rows, G->sc, M_BETA);
    k_l_scale<T><<<G->nb_rows, LB, 0, st>>>(G->n_rows, (T *)G->u, G->sc, M_BETA);
    // alpha_1 v_1 = K^T u_1
    int rc = gn_transpose<T>(G, G->u, G->v, -1, G->partial, st);
    if (rc) return rc;
    k_l_norm<<<1, LB, 0, st>>>(G->partial, G->nb_model, G->sc, M_ALPHA);
    k_l_scale<T><<<G->nb_model, LB, 0, st>>>(G->N, (T *)G->v, G->sc, M_ALPHA);
    k_l_copy<T><<<G->nb_model, LB, 0, st>>>(G->N, (const T *)G->v, (T *)G->h);
    k_l_zero<T><<<G->nb_model, LB, 0, st>>>(G->N, (T *)G->hbar);
    k_l_zero<T><<<G->nb_model, LB, 0, st>>>(G->N, (T *)G->x);
    k_m_start<<<1, 1, 0, st>>>(G->sc);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

template <typename T>
int lsmr_iteration(eik_gn *G, cudaStream_t st)
{
    // beta u = K v - alpha u
    int rc = gn_forward<T>(G, G->v, G->u, M_ALPHA, G->partial, st);
    if (rc) return rc;
    k_l_norm<<<1, LB, 0, st>>>(G->partial, G->nb_rows, G->sc, M_BETA);
    k_l_scale<T><<<G->nb_rows, LB, 0, st>>>(G->n_rows, (T *)G->u, G->sc, M_BETA);
    // alpha v = K^T u - beta v
    rc = gn_transpose<T>(G, G->u, G->v, M_BETA, G->partial, st);
    if (rc) return rc;
    k_l_norm<<<1, LB, 0, st>>>(G->partial, G->nb_model, G->sc, M_ALPHA);
    k_l_scale<T><<<G->nb_model, LB, 0, st>>>(G->N, (T *)G->v, G->sc, M_ALPHA);
    // rotations, then h, hbar, x and |x|
    k_m_step<<<1, 1, 0, st>>>(G->sc);
    k_m_update<T><<<G->nb_model, LB, 0, st>>>(G->N, (T *)G->x, (T *)G->h, (T *)G->hbar, (const T *)G->v, G->sc,
                                              G->partial);
    k_l_norm<<<1, LB, 0, st>>>(G->partial, G->nb_model, G->sc, M_NORMX);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

}  // namespace

// b = [-W_d r; 0; 0] (Eq. augmented-ls): -(w r) in FP64, then rounded to the vector type
template <typename T>
__global__ void k_gn_rhs(long long nd, long long n_rows, const double *__restrict__ wd, const double *__restrict__ r,
                         T *__restrict__ b)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    b[i] = i < nd ? (T)(-(wd[i] * r[i])) : T(0);
}

extern "C" {

void gn_free(eik_gn *G)
{
    if (!G) return;
    cudaDeviceSynchronize();
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    void *ptrs[] = {G->wd, G->sdiag, G->u, G->v, G->h, G->hbar, G->x, G->jp, G->yw, G->g, G->sc, G->partial,
                    G->pn, G->gc};
    for (void *p : ptrs) if (p) cudaFree(p);
    delete G;
}

static int gn_make(eik_tangent *t, const double *wd, const double *vk, double lambda, double gamma, int dtype,
                   int cells, eik_gn **out)
{
    try {
        if (!out) { set_error("out is NULL"); return EIK_ERR_INVALID; }
        *out = nullptr;
        if (!t || !wd || !vk || (dtype != EIK_F32 && dtype != EIK_F64) || !(lambda >= 0.0) || !(gamma >= 0.0)) {
            set_error("bad gn_create arguments");
            return EIK_ERR_INVALID;
        }
        Tangent *T = t->impl;
        if (T->n_rec == 0) { set_error("tangent has no receivers"); return EIK_ERR_INVALID; }
        eik_gn *G = new eik_gn();
        G->t = t;
        G->dtype = dtype;
        G->cells = cells;
        GridDesc mg = T->grid;       // the grid R differences on: nodes, or cells (extents n_d - 1)
        if (cells) {
            long long nc = 1;
            for (int d = 0; d < mg.ndim; ++d) { mg.n[d] -= 1; nc *= mg.n[d]; }
            mg.N = nc;
        }
        G->N = cells ? mg.N : T->N;
        G->nd = (long long)T->S * T->n_rec;
        G->R = make_rough(mg);
        G->nR = G->R.r0[G->R.nd];
        G->n_rows = G->nd + G->nR + G->N;
        G->lam = lambda;
        G->gamma = gamma;
        G->nb_rows = nblocks(G->n_rows);
        G->nb_model = nblocks(G->N);
        const size_t es = dtype == EIK_F32 ? 4 : 8;
        cudaError_t e = cudaMalloc((void **)&G->wd, G->nd * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void **)&G->sdiag, G->N * sizeof(double));
        void **model[] = {&G->v, &G->h, &G->hbar, &G->x};
        for (void **p : model) if (e == cudaSuccess) e = cudaMalloc(p, G->N * es);
        if (e == cudaSuccess) e = cudaMalloc(&G->g, T->N * es);
        if (cells && e == cudaSuccess) e = cudaMalloc(&G->pn, T->N * es);
        if (cells && e == cudaSuccess) e = cudaMalloc(&G->gc, G->N * es);
        if (e == cudaSuccess) e = cudaMalloc(&G->u, G->n_rows * es);
        if (e == cudaSuccess) e = cudaMalloc(&G->jp, G->nd * es);
        if (e == cudaSuccess) e = cudaMalloc(&G->yw, G->nd * es);
        if (e == cudaSuccess) e = cudaMalloc((void **)&G->sc, M_NSCAL * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void **)&G->partial, LMAXB * sizeof(double));
        if (e == cudaSuccess) e = cudaMemset(G->sc, 0, M_NSCAL * sizeof(double));
        if (e == cudaSuccess) e = cudaMemcpy(G->wd, wd, G->nd * sizeof(double), cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) {
            k_gn_sdiag<<<G->nb_model, LB>>>(G->N, gamma, vk, G->sdiag);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            int rc = cuda_fail(e, "gn_create", __FILE__, __LINE__);
            gn_free(G);
            return rc;
        }
        *out = G;
        return EIK_OK;
    } catch (...) {
        set_error("gn_create failed");
        return EIK_ERR_OOM;
    }
}

int gn_create(eik_tangent *t, const double *wd, const double *vk, double lambda, double gamma, int dtype, eik_gn **out)
{
    return gn_make(t, wd, vk, lambda, gamma, dtype, 0, out);
}

int gn_create_cells(eik_tangent *t, const double *wd, const double *v_cells, double lambda, double gamma, int dtype,
                    eik_gn **out)
{
    return gn_make(t, wd, v_cells, lambda, gamma, dtype, 1, out);
}

int gn_dims(const eik_gn *G, int64_t *n_rows, int64_t *n_data, int64_t *n_rough)
{
    if (!G) { set_error("gn is NULL"); return EIK_ERR_INVALID; }
    if (n_rows) *n_rows = G->n_rows;
    if (n_data) *n_data = G->nd;
    if (n_rough) *n_rough = G->nR;
    return EIK_OK;
}

int gn_apply(eik_gn *G, const void *p, void *out, eik_stream stream)
{
    if (!G || !p || !out) { set_error("bad gn_apply arguments"); return EIK_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    return G->dtype == EIK_F32 ? gn_forward<float>(G, p, out, -1, nullptr, st)
                               : gn_forward<double>(G, p, out, -1, nullptr, st);
}

int gn_apply_T(eik_gn *G, const void *y, void *out, eik_stream stream)
{
    if (!G || !y || !out) { set_error("bad gn_apply_T arguments"); return EIK_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    return G->dtype == EIK_F32 ? gn_transpose<float>(G, y, out, -1, nullptr, st)
                               : gn_transpose<double>(G, y, out, -1, nullptr, st);
}

int gn_rhs(eik_gn *G, const double *r, void *b, eik_stream stream)
{
    if (!G || !r || !b) { set_error("bad gn_rhs arguments"); return EIK_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((G->n_rows + 255) / 256);
    if (G->dtype == EIK_F32) k_gn_rhs<float><<<blocks, 256, 0, st>>>(G->nd, G->n_rows, G->wd, r, (float *)b);
    else k_gn_rhs<double><<<blocks, 256, 0, st>>>(G->nd, G->n_rows, G->wd, r, (double *)b);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

int gn_lsmr_start(eik_gn *G, const void *b, eik_stream stream)
{
    if (!G || !b) { set_error("bad gn_lsmr_start arguments"); return EIK_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    G->iters = 0;
    return G->dtype == EIK_F32 ? lsmr_begin<float>(G, b, st) : lsmr_begin<double>(G, b, st);
}

int gn_lsmr_iterate(eik_gn *G, int iters, int use_graph, eik_stream stream)
{
    eik::NvtxRange range("LSMR iterations");
    if (!G || iters < 0) { set_error("bad gn_lsmr_iterate arguments"); return EIK_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    if (use_graph && !G->exec) {
        // the traversal workspaces exist after gn_lsmr_start, so nothing allocates while capturing
        if (st == nullptr) { set_error("graph capture needs a non-default stream"); return EIK_ERR_INVALID; }
        EIK_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = G->dtype == EIK_F32 ? lsmr_iteration<float>(G, st) : lsmr_iteration<double>(G, st);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        G->graph = g;
        EIK_CHECK(cudaGraphInstantiate(&G->exec, g, 0));
    }
    for (int k = 0; k < iters; ++k) {
        if (use_graph) EIK_CHECK(cudaGraphLaunch(G->exec, st));
        else {
            int rc = G->dtype == EIK_F32 ? lsmr_iteration<float>(G, st) : lsmr_iteration<double>(G, st);
            if (rc) return rc;
        }
        ++G->iters;
    }
    return EIK_OK;
}

int gn_lsmr_solution(eik_gn *G, void *x, double *scalars, eik_stream stream)
{
    if (!G) { set_error("bad gn_lsmr_solution arguments"); return EIK_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = G->dtype == EIK_F32 ? 4 : 8;
    if (x) EIK_CHECK(cudaMemcpyAsync(x, G->x, G->N * es, cudaMemcpyDeviceToDevice, st));
    if (scalars) {
        double h[M_NSCAL];
        EIK_CHECK(cudaMemcpyAsync(h, G->sc, sizeof(h), cudaMemcpyDeviceToHost, st));
        EIK_CHECK(cudaStreamSynchronize(st));
        scalars[0] = h[M_NORMR];
        scalars[1] = fabs(h[M_ZETABAR]);
        scalars[2] = sqrt(h[M_NORMA2]);
        scalars[3] = h[M_NORMX];
        scalars[4] = h[M_NORMB];
        scalars[5] = (double)G->iters;
    }
    return EIK_OK;
}

}  // extern "C"
