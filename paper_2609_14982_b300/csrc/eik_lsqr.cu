// LSQR (Paige and Saunders, 1982) on the frozen Jacobian J of a tangent, with every
// vector operation and every scalar on the device so that one iteration can be
// captured in a CUDA graph and replayed (the inner Krylov solve of Sec. 4.5 uses LSMR on
// an augmented operator; the bare-J LSQR here is the Krylov loop of the benchmark
// configuration).  Model: slowness-type vector x [N] (one right-hand side), data
// [S][n_rec].  Norms are deterministic: per-block partial sums in a fixed order, then one
// block adds the partials in order (FP64).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "eik_internal.h"
#include "eik_krylov.h"

namespace eik {

// scalar slots
enum { L_ALPHA = 0, L_BETA, L_RHOBAR, L_PHIBAR, L_PHI, L_RHO, L_THETA, L_C, L_S, L_NSCAL = 16 };

// start: phibar = beta, rhobar = alpha
__global__ void k_l_start(double *sc)
{
    sc[L_PHIBAR] = sc[L_BETA];
    sc[L_RHOBAR] = sc[L_ALPHA];
}

// plane rotation of one LSQR step
__global__ void k_l_rot(double *sc)
{
    double rhobar = sc[L_RHOBAR], beta = sc[L_BETA], alpha = sc[L_ALPHA], phibar = sc[L_PHIBAR];
    double rho = sqrt(rhobar * rhobar + beta * beta);
    double c = rho > 0.0 ? rhobar / rho : 1.0, s = rho > 0.0 ? beta / rho : 0.0;
    sc[L_RHO] = rho;
    sc[L_C] = c;
    sc[L_S] = s;
    sc[L_THETA] = s * alpha;
    sc[L_RHOBAR] = -c * alpha;
    sc[L_PHI] = c * phibar;
    sc[L_PHIBAR] = s * phibar;
}

// x += (phi/rho) w ;  w = v - (theta/rho) w
template <typename T>
__global__ void k_l_xw(long long n, T *x, T *w, const T *v, const double *sc)
{
    double rho = sc[L_RHO];
    double f = rho > 0.0 ? sc[L_PHI] / rho : 0.0, g = rho > 0.0 ? sc[L_THETA] / rho : 0.0;
    for (long long i = blockIdx.x * (long long)LB + threadIdx.x; i < n; i += (long long)gridDim.x * LB) {
        double wi = (double)w[i];
        x[i] = (T)((double)x[i] + f * wi);
        w[i] = (T)((double)v[i] - g * wi);
    }
}

}  // namespace eik

using namespace eik;

struct eik_tangent { Tangent *impl; };

struct eik_lsqr {
    eik_tangent *t = nullptr;
    int dtype = EIK_F64;
    long long n_model = 0, n_data = 0;
    void *u = nullptr, *v = nullptr, *w = nullptr, *x = nullptr, *Av = nullptr, *Atu = nullptr;
    double *sc = nullptr, *partial = nullptr;
    int nb_model = 0, nb_data = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int iters = 0;
};

static int lsqr_fwd(eik_lsqr *L, cudaStream_t st)
{
    return traverse(L->t->impl, false, MODE_J, L->v, 1, 1, nullptr, L->Av, 0, L->dtype, st);
}

static int lsqr_bwd(eik_lsqr *L, cudaStream_t st)
{
    return traverse(L->t->impl, true, MODE_J, L->u, 0, 1, nullptr, L->Atu, 1, L->dtype, st);
}

template <typename T>
static int lsqr_iteration(eik_lsqr *L, cudaStream_t st)
{
    // u = J v - alpha u ; beta = |u| ; u /= beta
    int rc = lsqr_fwd(L, st);
    if (rc) return rc;
    k_l_axpby_sq<T><<<L->nb_data, LB, 0, st>>>(L->n_data, (const T *)L->Av, (T *)L->u, L->sc, L_ALPHA, 1.0, L->partial);
    k_l_norm<<<1, LB, 0, st>>>(L->partial, L->nb_data, L->sc, L_BETA);
    k_l_scale<T><<<L->nb_data, LB, 0, st>>>(L->n_data, (T *)L->u, L->sc, L_BETA);
    // v = J^T u - beta v ; alpha = |v| ; v /= alpha
    rc = lsqr_bwd(L, st);
    if (rc) return rc;
    k_l_axpby_sq<T><<<L->nb_model, LB, 0, st>>>(L->n_model, (const T *)L->Atu, (T *)L->v, L->sc, L_BETA, 1.0, L->partial);
    k_l_norm<<<1, LB, 0, st>>>(L->partial, L->nb_model, L->sc, L_ALPHA);
    k_l_scale<T><<<L->nb_model, LB, 0, st>>>(L->n_model, (T *)L->v, L->sc, L_ALPHA);
    k_l_rot<<<1, 1, 0, st>>>(L->sc);
    k_l_xw<T><<<L->nb_model, LB, 0, st>>>(L->n_model, (T *)L->x, (T *)L->w, (const T *)L->v, L->sc);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

template <typename T>
static int lsqr_begin(eik_lsqr *L, const void *b, cudaStream_t st)
{
    const size_t es = sizeof(T);
    EIK_CHECK(cudaMemcpyAsync(L->u, b, L->n_data * es, cudaMemcpyDeviceToDevice, st));
    k_l_axpby_sq<T><<<L->nb_data, LB, 0, st>>>(L->n_data, (const T *)L->u, (T *)L->u, L->sc, -1, 0.0, L->partial);
    k_l_norm<<<1, LB, 0, st>>>(L->partial, L->nb_data, L->sc, L_BETA);
    k_l_scale<T><<<L->nb_data, LB, 0, st>>>(L->n_data, (T *)L->u, L->sc, L_BETA);
    int rc = lsqr_bwd(L, st);
    if (rc) return rc;
    k_l_axpby_sq<T><<<L->nb_model, LB, 0, st>>>(L->n_model, (const T *)L->Atu, (T *)L->v, L->sc, -1, 0.0, L->partial);
    k_l_norm<<<1, LB, 0, st>>>(L->partial, L->nb_model, L->sc, L_ALPHA);
    k_l_scale<T><<<L->nb_model, LB, 0, st>>>(L->n_model, (T *)L->v, L->sc, L_ALPHA);
    k_l_copy<T><<<L->nb_model, LB, 0, st>>>(L->n_model, (const T *)L->v, (T *)L->w);
    k_l_zero<T><<<L->nb_model, LB, 0, st>>>(L->n_model, (T *)L->x);
    k_l_start<<<1, 1, 0, st>>>(L->sc);
    EIK_CHECK_LAUNCH();
    return EIK_OK;
}

extern "C" {

int lsqr_create(eik_tangent *t, int dtype, eik_lsqr **out)
{
    try {
        if (!t || !out || (dtype != EIK_F32 && dtype != EIK_F64)) { set_error("bad lsqr_create arguments"); return EIK_ERR_INVALID; }
        Tangent *T = t->impl;
        if (T->n_rec == 0) { set_error("tangent has no receivers"); return EIK_ERR_INVALID; }
        eik_lsqr *L = new eik_lsqr();
        L->t = t;
        L->dtype = dtype;
        L->n_model = T->N;
        L->n_data = (long long)T->S * T->n_rec;
        const size_t es = dtype == EIK_F32 ? 4 : 8;
        auto nb = [](long long n) { long long b = (n + LB - 1) / LB; return (int)(b < LMAXB ? (b < 1 ? 1 : b) : LMAXB); };
        L->nb_model = nb(L->n_model);
        L->nb_data = nb(L->n_data);
        cudaError_t e = cudaSuccess;
        void **bufs[] = {&L->v, &L->w, &L->x, &L->Atu};
        for (void **p : bufs) if (e == cudaSuccess) e = cudaMalloc(p, L->n_model * es);
        if (e == cudaSuccess) e = cudaMalloc(&L->u, L->n_data * es);
        if (e == cudaSuccess) e = cudaMalloc(&L->Av, L->n_data * es);
        if (e == cudaSuccess) e = cudaMalloc((void **)&L->sc, L_NSCAL * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void **)&L->partial, LMAXB * sizeof(double));
        if (e == cudaSuccess) e = cudaMemset(L->sc, 0, L_NSCAL * sizeof(double));
        if (e != cudaSuccess) {
            int rc = cuda_fail(e, "lsqr_create", __FILE__, __LINE__);
            lsqr_free(L);
            return rc;
        }
        *out = L;
        return EIK_OK;
    } catch (...) {
        set_error("lsqr_create failed");
        return EIK_ERR_OOM;
    }
}

int lsqr_start(eik_lsqr *L, const void *b, eik_stream stream)
{
    if (!L || !b) { set_error("bad lsqr_start arguments"); return EIK_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    L->iters = 0;
    return L->dtype == EIK_F32 ? lsqr_begin<float>(L, b, st) : lsqr_begin<double>(L, b, st);
}

int lsqr_iterate(eik_lsqr *L, int iters, int use_graph, eik_stream stream)
{
    eik::NvtxRange range("LSQR iterations");
    if (!L || iters < 0) { set_error("bad lsqr_iterate arguments"); return EIK_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    if (use_graph && !L->exec) {
        // the traversal workspaces exist after lsqr_start, so nothing allocates while capturing
        if (st == nullptr) { set_error("graph capture needs a non-default stream"); return EIK_ERR_INVALID; }
        EIK_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = L->dtype == EIK_F32 ? lsqr_iteration<float>(L, st) : lsqr_iteration<double>(L, st);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        L->graph = g;
        EIK_CHECK(cudaGraphInstantiate(&L->exec, g, 0));
    }
    for (int k = 0; k < iters; ++k) {
        if (use_graph) EIK_CHECK(cudaGraphLaunch(L->exec, st));
        else {
            int rc = L->dtype == EIK_F32 ? lsqr_iteration<float>(L, st) : lsqr_iteration<double>(L, st);
            if (rc) return rc;
        }
        ++L->iters;
    }
    return EIK_OK;
}

int lsqr_solution(eik_lsqr *L, void *x, double *scalars, eik_stream stream)
{
    if (!L) { set_error("bad lsqr_solution arguments"); return EIK_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = L->dtype == EIK_F32 ? 4 : 8;
    if (x) EIK_CHECK(cudaMemcpyAsync(x, L->x, L->n_model * es, cudaMemcpyDeviceToDevice, st));
    if (scalars) {
        EIK_CHECK(cudaMemcpyAsync(scalars, L->sc, 9 * sizeof(double), cudaMemcpyDeviceToHost, st));
        EIK_CHECK(cudaStreamSynchronize(st));
    }
    return EIK_OK;
}

void lsqr_free(eik_lsqr *L)
{
    if (!L) return;
    cudaDeviceSynchronize();
    if (L->exec) cudaGraphExecDestroy(L->exec);
    if (L->graph) cudaGraphDestroy(L->graph);
    void *ptrs[] = {L->u, L->v, L->w, L->x, L->Av, L->Atu, L->sc, L->partial};
    for (void *p : ptrs) if (p) cudaFree(p);
    delete L;
}

}  // extern "C"
