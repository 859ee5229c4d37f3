// Device vector kernels shared by the Krylov solvers (LSQR on J, LSMR on the augmented
// Gauss-Newton operator).  Scalars live in a device array so that an iteration can be
// captured in a CUDA graph.  Norms are deterministic: per-block partial sums in a fixed
// order, then one block adds the partials in order (FP64).
#pragma once
#include <cuda_runtime.h>

#include <cmath>

namespace eik {

constexpr int LB = 256;          // threads per block of the vector kernels
constexpr int LMAXB = 1024;      // partial sums (blocks of the reductions)

template <typename T>
__global__ void k_l_axpby_sq(long long n, const T *__restrict__ a, T *__restrict__ u, const double *sc, int coef_slot,
                             double sign, double *partial)
{
    // u = a - sign * sc[coef] * u ;  partial[block] = sum u^2 over the block's stride
    __shared__ double red[LB];
    // coef_slot < 0: u = a (u is not read, so it may hold anything, e.g. fresh memory)
    const bool axpby = coef_slot >= 0;
    double coef = axpby ? sign * sc[coef_slot] : 0.0;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)LB + threadIdx.x; i < n; i += (long long)gridDim.x * LB) {
        double v = axpby ? (double)a[i] - coef * (double)u[i] : (double)a[i];
        T tv = (T)v;
        u[i] = tv;
        acc += (double)tv * (double)tv;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = LB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

static __global__ void k_l_norm(const double *partial, int nb, double *sc, int slot)
{
    __shared__ double red[LB];
    double acc = 0.0;
    // fixed order: thread t sums partials t, t+LB, ...
    for (int b = threadIdx.x; b < nb; b += LB) acc += partial[b];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = LB / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) sc[slot] = sqrt(red[0]);
}

template <typename T>
__global__ void k_l_scale(long long n, T *u, const double *sc, int slot)
{
    double s = sc[slot];
    double inv = s > 0.0 ? 1.0 / s : 0.0;
    for (long long i = blockIdx.x * (long long)LB + threadIdx.x; i < n; i += (long long)gridDim.x * LB)
        u[i] = (T)((double)u[i] * inv);
}

template <typename T>
__global__ void k_l_copy(long long n, const T *a, T *b)
{
    for (long long i = blockIdx.x * (long long)LB + threadIdx.x; i < n; i += (long long)gridDim.x * LB) b[i] = a[i];
}

template <typename T>
__global__ void k_l_zero(long long n, T *b)
{
    for (long long i = blockIdx.x * (long long)LB + threadIdx.x; i < n; i += (long long)gridDim.x * LB) b[i] = T(0);
}

}  // namespace eik
