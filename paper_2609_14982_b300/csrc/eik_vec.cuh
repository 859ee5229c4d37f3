// Vector loads and stores of right-hand-side rows shared by the traversal and sweeping
// kernels (device code only; not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstring>

namespace eik {

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

}  // namespace eik
