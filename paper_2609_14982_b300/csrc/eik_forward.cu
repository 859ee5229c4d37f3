// First-arrival state T = T0 tau for point sources (Sec. 2.1-2.2): the paper takes its
// nonlinear state from a cited factored topography-dependent solver without giving the
// scheme; this file solves the factored full-metric equation
//     H(tau, grad_xi tau) = sqrt(P^T G P) = s,   P = tau g0 + T0 grad_xi tau,
// with T0 = s_src |x - x_src|, g0 = J^T grad_x T0, by first-order Lax-Friedrichs
// sweeping (Kao, Osher and Qian, 2004): Gauss-Seidel over the 2^ndim logical orderings,
// each ordering run hyperplane by hyperplane (identical to the lexicographic sweep).
// Node update (interior, tau_+/- the neighbours along axis d, h_d the spacing):
//     p_d   = (tau_+ - tau_-) / (2 h_d),   P_b = tau_i g0_b + T0 p_b,
//     H     = sqrt(sum_a P_a (sum_b G_ab P_b)),   alpha_d = T0 sqrt(G_dd),
//     tau_i = ((s_i - H) + sum_d alpha_d (tau_+ + tau_-) / (2 h_d)) / (sum_d alpha_d / h_d).
// After every ordering each boundary node takes the value of its nearest interior node
// along the inward diagonal (one step inward along every boundary axis), which keeps
// the iteration monotone.  Nodes within eik_src_radius * max(h) of the source keep
// tau = 1.  Start: tau = 1.  Stop, per source: the first cycle whose largest |change|
// for that source is below eik_tol (that source then stops iterating).
// Compiled with -fmad=false so that every step is a separately rounded IEEE operation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "eik_internal.h"

namespace eik {

__global__ void k_metric(GridDesc g, const double *__restrict__ xyz, double *__restrict__ G, double *__restrict__ Jout);

// The per-(source, node) arrays of the LF solve (T0, g0, alpha, tau, fixed) are stored
// node-major, v = i * S + a: the threads of a hyperplane launch take the sources of a
// node as their fastest index, so their loads of a node's (and its neighbours') values
// are contiguous across the warp.
constexpr int DSLOTS = 1024;   // convergence maxima per source, spread over this many words

// per (source, node): T0, g0 = J^T grad_x T0, alpha_d, fixed flag
__global__ void k_eik_prep(GridDesc g, int S, const double *__restrict__ xyz, const double *__restrict__ Jm,
                           const double *__restrict__ G, const double *__restrict__ s, const int *__restrict__ src,
                           double radius, double *T0, double *g0, double *alpha, unsigned char *fixed, double *tau)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= g.N * S) return;
    const int nd = g.ndim;
    long long i = v / S, a = v - i * S;
    long long k = src[a];
    double ss = s[k];
    double d[3], r2 = 0.0;
    for (int c = 0; c < nd; ++c) { d[c] = xyz[i * nd + c] - xyz[k * nd + c]; r2 = r2 + d[c] * d[c]; }
    double r = sqrt(r2);
    T0[v] = ss * r;
    double gx[3];
    for (int c = 0; c < nd; ++c) gx[c] = r > 0.0 ? ss * d[c] / r : 0.0;
    for (int b = 0; b < nd; ++b) {
        double acc = 0.0;
        for (int c = 0; c < nd; ++c) acc = acc + Jm[i * nd * nd + c * nd + b] * gx[c];
        g0[v * nd + b] = acc;
    }
    for (int b = 0; b < nd; ++b) alpha[v * nd + b] = T0[v] * sqrt(G[i * nd * nd + b * nd + b]);
    fixed[v] = r <= radius ? 1 : 0;
    tau[v] = 1.0;
}

// the same for point sources: position xs [S][3], slowness ss [S] and fixed radius rad [S]
// per source (the point-source reading: every corner of the source cell stays fixed)
__global__ void k_eik_prep_pt(GridDesc g, int S, const double *__restrict__ xyz, const double *__restrict__ Jm,
                              const double *__restrict__ G, const double *__restrict__ xs, const double *__restrict__ ss,
                              const double *__restrict__ rad, double *T0, double *g0, double *alpha,
                              unsigned char *fixed, double *tau)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= g.N * S) return;
    const int nd = g.ndim;
    long long i = v / S, a = v - i * S;
    const double sv = ss[a];
    double d[3], r2 = 0.0;
    for (int c = 0; c < nd; ++c) { d[c] = xyz[i * nd + c] - xs[a * 3 + c]; r2 = r2 + d[c] * d[c]; }
    double r = sqrt(r2);
    T0[v] = sv * r;
    double gx[3];
    for (int c = 0; c < nd; ++c) gx[c] = r > 0.0 ? sv * d[c] / r : 0.0;
    for (int b = 0; b < nd; ++b) {
        double acc = 0.0;
        for (int c = 0; c < nd; ++c) acc = acc + Jm[i * nd * nd + c * nd + b] * gx[c];
        g0[v * nd + b] = acc;
    }
    for (int b = 0; b < nd; ++b) alpha[v * nd + b] = T0[v] * sqrt(G[i * nd * nd + b * nd + b]);
    fixed[v] = r <= rad[a] ? 1 : 0;
    tau[v] = 1.0;
}

// fixed radius per point source: max(radius, largest corner distance); FP64 threshold
__global__ void k_point_radius(int S, const double *__restrict__ r, const double *__restrict__ ss, double radius,
                               double dist64, double *__restrict__ rad, double *__restrict__ t0_fp64)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= S) return;
    double m = radius;
    for (int q = 0; q < 8; ++q) m = r[a * 8 + q] > m ? r[a * 8 + q] : m;
    rad[a] = m;
    t0_fp64[a] = ss[a] * dist64;
}

// warm start: tau = T_init / T0 at every node that is not fixed (T_init [S][N], source-major)
__global__ void k_tau_from_T(long long N, int S, const double *__restrict__ T_init, const double *__restrict__ T0,
                             const unsigned char *__restrict__ fixed, double *__restrict__ tau)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= N * S) return;
    const long long i = v / S, a = v - i * S;
    if (fixed[v] || !(T0[v] > 0.0)) return;
    const double t = T_init[a * N + i] / T0[v];
    if (t > 0.0 && t < 1e30) tau[v] = t;     // keep tau = 1 where the given value is unusable
}

struct LFParams {
    GridDesc g;
    int S, order, h, lo0, hi0;
    int fp32;                  // update nodes with T0 > t0_fp64 in FP32 arithmetic
    const double *t0_fp64;     // [S] threshold on T0 per source (s_src * radius)
    const double *G, *s, *T0, *g0, *alpha;
    const unsigned char *fixed;
    const unsigned char *active;   // [S] sources still iterating
    double *tau;
    unsigned long long *dmax;   // [S][DSLOTS] bit patterns of max |d tau| (non-negative doubles)
};

__device__ __forceinline__ double lf_update(const LFParams &P, long long a, long long i, const int *c)
{
    const GridDesc &g = P.g;
    const int nd = g.ndim;
    const long long S = P.S, v = i * S + a;
    const double *tau = P.tau + a;   // node j of source a at tau[j * S]
    const double T0 = P.T0[v];
    const double ti = tau[i * S];
    double p[3], Pv[3];
    for (int d = 0; d < nd; ++d) p[d] = (tau[(i + g.st[d]) * S] - tau[(i - g.st[d]) * S]) / (2.0 * g.dxi[d]);
    for (int b = 0; b < nd; ++b) Pv[b] = ti * P.g0[v * nd + b] + T0 * p[b];
    double H2 = 0.0;
    for (int x = 0; x < nd; ++x) {
        double row = 0.0;
        for (int b = 0; b < nd; ++b) row = row + P.G[i * nd * nd + x * nd + b] * Pv[b];
        H2 = H2 + Pv[x] * row;
    }
    double H = sqrt(H2);
    double num = P.s[i] - H, den = 0.0;
    for (int d = 0; d < nd; ++d) {
        double al = P.alpha[v * nd + d];
        num = num + al * (tau[(i + g.st[d]) * S] + tau[(i - g.st[d]) * S]) / (2.0 * g.dxi[d]);
        den = den + al / g.dxi[d];
    }
    (void)c;
    return num / den;
}

// the same update in FP32 arithmetic (inputs rounded to FP32, result stored as FP64)
__device__ __forceinline__ double lf_update_f32(const LFParams &P, long long a, long long i)
{
    const GridDesc &g = P.g;
    const int nd = g.ndim;
    const long long S = P.S, v = i * S + a;
    const double *tau = P.tau + a;
    const float T0 = (float)P.T0[v];
    const float ti = (float)tau[i * S];
    float p[3], Pv[3];
    for (int d = 0; d < nd; ++d)
        p[d] = ((float)tau[(i + g.st[d]) * S] - (float)tau[(i - g.st[d]) * S]) / (2.0f * (float)g.dxi[d]);
    for (int b = 0; b < nd; ++b) Pv[b] = ti * (float)P.g0[v * nd + b] + T0 * p[b];
    float H2 = 0.0f;
    for (int x = 0; x < nd; ++x) {
        float row = 0.0f;
        for (int b = 0; b < nd; ++b) row = row + (float)P.G[i * nd * nd + x * nd + b] * Pv[b];
        H2 = H2 + Pv[x] * row;
    }
    float num = (float)P.s[i] - sqrtf(H2), den = 0.0f;
    for (int d = 0; d < nd; ++d) {
        const float al = (float)P.alpha[v * nd + d];
        num = num + al * ((float)tau[(i + g.st[d]) * S] + (float)tau[(i - g.st[d]) * S]) / (2.0f * (float)g.dxi[d]);
        den = den + al / (float)g.dxi[d];
    }
    return (double)(num / den);
}

// max |d tau| of the warp's lanes into source key's word of this block's slot: one atomic
// per warp when all lanes work for the same source, else one per lane, spread over
// DSLOTS words per source.  Every lane of the warp must call it (lanes without an update
// pass key = -1).  Same-address atomics serialise in L2; one word per source made them
// the cost of a hyperplane launch.
__device__ __forceinline__ void warp_max_into(unsigned long long *dmax, int key, double dd)
{
    dmax += blockIdx.x & (DSLOTS - 1);
    const unsigned full = 0xffffffffu;
    unsigned long long bits = key >= 0 ? (unsigned long long)__double_as_longlong(dd) : 0ull;
    const int k0 = __shfl_sync(full, key, 0);
    if (__all_sync(full, key == k0 || key < 0) && k0 >= 0) {
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(full, bits, o);
            bits = other > bits ? other : bits;   // non-negative doubles order like their bits
        }
        if ((threadIdx.x & 31) == 0) atomicMax(dmax + (long long)k0 * DSLOTS, bits);
    } else if (key >= 0) {
        atomicMax(dmax + (long long)key * DSLOTS, bits);
    }
}

__global__ void k_lf_plane(LFParams P)
{
    const GridDesc &g = P.g;
    const int nd = g.ndim;
    // interior nodes only: coordinates 1..n-2 along every axis
    const int m0 = g.n[0] - 2, m1 = g.n[1] - 2, m2 = nd == 3 ? g.n[2] - 2 : 1;
    long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long span = (long long)(P.hi0 - P.lo0 + 1) * (nd == 3 ? m1 : 1);
    bool valid = tid < span * P.S;
    long long cell = valid ? tid / P.S : 0, a = tid - cell * P.S;   // sources fastest
    valid = valid && P.active[a];
    int c0 = 0, c1 = 0, c2 = 0;
    if (nd == 3) {
        c0 = P.lo0 + (int)(cell / m1);
        c1 = (int)(cell % m1);
        c2 = P.h - c0 - c1;
        valid = valid && c2 >= 0 && c2 < m2;
    } else {
        c0 = P.lo0 + (int)cell;
        c1 = P.h - c0;
        valid = valid && c1 >= 0 && c1 < m1;
    }
    long long v = 0;
    double dd = 0.0;
    if (valid) {
        const int i0 = 1 + ((P.order & 1) ? m0 - 1 - c0 : c0);
        const int i1 = 1 + ((P.order & 2) ? m1 - 1 - c1 : c1);
        const int i2 = nd == 3 ? 1 + ((P.order & 4) ? m2 - 1 - c2 : c2) : 0;
        const long long i = nd == 3 ? ((long long)i0 * g.n[1] + i1) * g.n[2] + i2 : (long long)i0 * g.n[1] + i1;
        v = i * P.S + a;
        valid = !P.fixed[v];
        if (valid) {
            int c[3] = {i0, i1, i2};
            const double nv = (P.fp32 && P.T0[v] > P.t0_fp64[a]) ? lf_update_f32(P, a, i) : lf_update(P, a, i, c);
            const double old = P.tau[v];
            P.tau[v] = nv;
            dd = fabs(nv - old);
        }
    }
    warp_max_into(P.dmax, valid ? (int)a : -1, dd);
}

// boundary nodes take the value of the nearest interior node along the inward diagonal
__global__ void k_lf_boundary(GridDesc g, int S, const unsigned char *__restrict__ fixed,
                              const unsigned char *__restrict__ active, double *tau, unsigned long long *dmax)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    bool valid = v < g.N * S && !fixed[v];
    const long long i = valid ? v / S : 0, a = v - i * S;
    valid = valid && active[a];
    double dd = 0.0;
    if (valid) {
        int c[3];
        if (g.ndim == 3) { c[2] = (int)(i % g.n[2]); c[1] = (int)((i / g.n[2]) % g.n[1]); c[0] = (int)(i / g.st[0]); }
        else { c[1] = (int)(i % g.n[1]); c[0] = (int)(i / g.n[1]); c[2] = 0; }
        long long step = 0;
        for (int d = 0; d < g.ndim; ++d) {
            if (c[d] == 0) step += g.st[d];
            else if (c[d] == g.n[d] - 1) step -= g.st[d];
        }
        valid = step != 0;
        if (valid) {
            const double nv = tau[(i + step) * S + a];
            dd = fabs(nv - tau[v]);
            tau[v] = nv;
        }
    }
    warp_max_into(dmax, valid ? (int)a : -1, dd);
}

// T0 beyond which a node of source a is far enough from it for FP32 arithmetic
__global__ void k_t0_threshold(int S, const double *__restrict__ s, const int *__restrict__ src, double dist, double *out)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < S) out[a] = s[src[a]] * dist;
}

// T [S][N] (source-major, the caller's layout) from the node-major T0 and tau
__global__ void k_eik_out(long long N, int S, const double *T0, const double *tau, double *T)
{
    const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (o >= N * S) return;
    const long long a = o / N, i = o - a * N, v = i * S + a;
    T[o] = T0[v] * tau[v];
}

// max over the DSLOTS words of each source into its first word
__global__ void k_dmax_fold(unsigned long long *dmax)
{
    __shared__ unsigned long long red[256];
    unsigned long long *w = dmax + (long long)blockIdx.x * DSLOTS;
    unsigned long long m = 0;
    for (int k = threadIdx.x; k < DSLOTS; k += blockDim.x) m = w[k] > m ? w[k] : m;
    red[threadIdx.x] = m;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h && red[threadIdx.x + h] > red[threadIdx.x]) red[threadIdx.x] = red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) w[0] = red[0];
}

// One LF cycle: the 2^ndim orderings, each a sequence of hyperplane launches (a plane's
// nodes only read the previous plane's values: Gauss-Seidel order) and the boundary copy.
static void lf_cycle_launch(LFParams P, long long SN, int m0, int m1, int hmax_i, int nord, cudaStream_t st)
{
    const int nd = P.g.ndim;
    cudaMemsetAsync(P.dmax, 0, (size_t)P.S * DSLOTS * sizeof(unsigned long long), st);
    for (int o = 0; o < nord; ++o) {
        P.order = o;
        for (int h = 0; h <= hmax_i; ++h) {
            P.h = h;
            const int rest = hmax_i - (m0 - 1);
            P.lo0 = std::max(0, h - rest);
            P.hi0 = std::min(m0 - 1, h);
            const long long span = (long long)(P.hi0 - P.lo0 + 1) * (nd == 3 ? m1 : 1) * P.S;
            k_lf_plane<<<(unsigned)((span + 255) / 256), 256, 0, st>>>(P);
        }
        k_lf_boundary<<<(unsigned)((SN + 255) / 256), 256, 0, st>>>(P.g, P.S, P.fixed, P.active, P.tau, P.dmax);
    }
    k_dmax_fold<<<P.S, 256, 0, st>>>(P.dmax);
}

// Cycles until every source's largest change over a cycle is below tol (each source
// stops iterating at its own first such cycle).  With use_graph the thousands of
// launches of one cycle are captured once (on a private stream) and replayed per cycle.
static cudaError_t lf_cycles(LFParams P, int S, long long SN, int m0, int m1, int hmax_i, int nord, double tol,
                             int max_cycles, bool use_graph, int *used, cudaStream_t st)
{
    std::vector<unsigned char> h_active(S, 1);
    std::vector<unsigned long long> h_dmax(S);
    cudaError_t e = cudaMemcpyAsync((void *)P.active, h_active.data(), S, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
    };
    if (use_graph) {
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            lf_cycle_launch(P, SN, m0, m1, hmax_i, nord, cap);
            e = cudaStreamEndCapture(cap, &graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) { cleanup(); return e; }
    }
    int left = S;
    *used = -1;
    for (int cyc = 1; cyc <= max_cycles; ++cyc) {
        if (use_graph) e = cudaGraphLaunch(exec, st);
        else {
            lf_cycle_launch(P, SN, m0, m1, hmax_i, nord, st);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(h_dmax.data(), sizeof(unsigned long long), P.dmax, DSLOTS * sizeof(unsigned long long),
                                  sizeof(unsigned long long), S, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { cleanup(); return e; }
        bool changed = false;
        for (int a = 0; a < S; ++a) {
            if (!h_active[a]) continue;
            double dm;
            std::memcpy(&dm, &h_dmax[a], sizeof dm);
            if (dm < tol) { h_active[a] = 0; --left; changed = true; }
        }
        if (left == 0) { *used = cyc; break; }
        if (changed) {
            e = cudaMemcpyAsync((void *)P.active, h_active.data(), S, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) { cleanup(); return e; }
        }
    }
    cleanup();
    return cudaSuccess;
}

}  // namespace eik

using namespace eik;

// node sources (src_node) or point sources (src_f: host [S][ndim] fractional logical
// coordinates)
static int forward_impl(const eik_grid *gin, const double *s, int S, const int *src_node, const double *src_f,
                        double *T, const eik_opts *opts_in, int *cycles, eik_stream stream,
                        const double *T_init = nullptr)
{
    NvtxRange range(src_f ? "eik_forward_points" : (T_init ? "eik_forward_warm" : "eik_forward"));
    try {
        if (!gin || (gin->ndim != 2 && gin->ndim != 3) || !gin->xyz || !s || !T || (!src_node && !src_f) || S <= 0) {
            set_error("bad eik_forward arguments");
            return EIK_ERR_INVALID;
        }
        eik_opts def;
        eik_opts_default(&def);
        const eik_opts *opts = opts_in ? opts_in : &def;
        GridDesc g = make_grid_desc(gin);
        for (int d = 0; d < g.ndim; ++d)
            if (g.n[d] < 3) { set_error("grid needs >= 3 nodes per axis"); return EIK_ERR_INVALID; }
        if (src_node)
            for (int a = 0; a < S; ++a)
                if (src_node[a] < 0 || src_node[a] >= g.N) { set_error("source node out of range"); return EIK_ERR_INVALID; }
        cudaStream_t st = (cudaStream_t)stream;
        const int nd = g.ndim;
        const long long N = g.N, SN = N * S;
        double *G = nullptr, *Jm = nullptr, *T0 = nullptr, *g0 = nullptr, *alpha = nullptr, *tau = nullptr;
        unsigned char *fixed = nullptr, *active = nullptr;
        int *src_d = nullptr;
        unsigned long long *dmax = nullptr;
        double *t0_fp64 = nullptr, *rad = nullptr;
        PointData pd;
        auto release = [&]() {
            cudaFree(G); cudaFree(Jm); cudaFree(T0); cudaFree(g0); cudaFree(alpha); cudaFree(tau);
            cudaFree(fixed); cudaFree(active); cudaFree(src_d); cudaFree(dmax); cudaFree(t0_fp64); cudaFree(rad);
            free_point_data(pd);
        };
        if (src_f) {
            int rc = point_sources(g, gin->xyz, s, S, src_f, pd, st);
            if (rc) { release(); return rc; }
        }
#define TRY(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { int rc_ = cuda_fail(e_, #call, __FILE__, __LINE__); release(); return rc_; } } while (0)
        TRY(cudaMalloc(&G, N * nd * nd * sizeof(double)));
        TRY(cudaMalloc(&Jm, N * nd * nd * sizeof(double)));
        TRY(cudaMalloc(&T0, SN * sizeof(double)));
        TRY(cudaMalloc(&g0, SN * nd * sizeof(double)));
        TRY(cudaMalloc(&alpha, SN * nd * sizeof(double)));
        TRY(cudaMalloc(&tau, SN * sizeof(double)));
        TRY(cudaMalloc(&fixed, SN));
        TRY(cudaMalloc(&src_d, S * sizeof(int)));
        TRY(cudaMalloc(&dmax, (size_t)S * DSLOTS * sizeof(unsigned long long)));
        TRY(cudaMalloc(&active, S));
        TRY(cudaMalloc(&t0_fp64, S * sizeof(double)));
        double hmax = 0.0;
        for (int d = 0; d < nd; ++d) hmax = std::max(hmax, g.dxi[d]);
        k_metric<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(g, gin->xyz, G, Jm);
        if (src_f) {
            TRY(cudaMalloc(&rad, S * sizeof(double)));
            k_point_radius<<<(S + 127) / 128, 128, 0, st>>>(S, pd.r, pd.ss, opts->eik_src_radius * hmax,
                                                            opts->eik_fp64_radius * hmax, rad, t0_fp64);
            k_eik_prep_pt<<<(unsigned)((SN + 255) / 256), 256, 0, st>>>(g, S, gin->xyz, Jm, G, pd.xs, pd.ss, rad, T0,
                                                                         g0, alpha, fixed, tau);
        } else {
            TRY(cudaMemcpyAsync(src_d, src_node, S * sizeof(int), cudaMemcpyHostToDevice, st));
            k_eik_prep<<<(unsigned)((SN + 255) / 256), 256, 0, st>>>(g, S, gin->xyz, Jm, G, s, src_d,
                                                                      opts->eik_src_radius * hmax, T0, g0, alpha, fixed, tau);
            k_t0_threshold<<<(S + 127) / 128, 128, 0, st>>>(S, s, src_d, opts->eik_fp64_radius * hmax, t0_fp64);
        }
        TRY(cudaGetLastError());
        if (T_init) {
            k_tau_from_T<<<(unsigned)((SN + 255) / 256), 256, 0, st>>>(N, S, T_init, T0, fixed, tau);
            TRY(cudaGetLastError());
        }
        LFParams P{};
        P.g = g; P.S = S; P.G = G; P.s = s; P.T0 = T0; P.g0 = g0; P.alpha = alpha; P.fixed = fixed; P.tau = tau;
        P.dmax = dmax; P.active = active;
        P.fp32 = opts->eik_fp32 ? 1 : 0; P.t0_fp64 = t0_fp64;
        const double tol = opts->eik_fp32 ? std::max(opts->eik_tol, 1e-6) : opts->eik_tol;
        const int m0 = g.n[0] - 2, m1 = g.n[1] - 2, m2 = nd == 3 ? g.n[2] - 2 : 1;
        const int hmax_i = (m0 - 1) + (m1 - 1) + (nd == 3 ? m2 - 1 : 0);
        const int nord = 1 << nd;
        // each source stops at the first cycle whose largest change is below eik_tol
        int used = -1;
        TRY(lf_cycles(P, S, SN, m0, m1, hmax_i, nord, tol, opts->eik_max_cycles, true, &used, st));
        k_eik_out<<<(unsigned)((SN + 255) / 256), 256, 0, st>>>(N, S, T0, tau, T);
        TRY(cudaGetLastError());
        TRY(cudaStreamSynchronize(st));
#undef TRY
        release();
        if (cycles) *cycles = used < 0 ? opts->eik_max_cycles : used;
        if (used < 0) { set_error("eik_forward did not converge in %d cycles", opts->eik_max_cycles); return EIK_ERR_NOT_CONVERGED; }
        return EIK_OK;
    } catch (...) {
        set_error("eik_forward failed");
        return EIK_ERR_INVALID;
    }
}

extern "C" int eik_forward(const eik_grid *gin, const double *s, int S, const int *src_node, double *T,
                           const eik_opts *opts_in, int *cycles, eik_stream stream)
{
    if (!src_node) { set_error("bad eik_forward arguments"); return EIK_ERR_INVALID; }
    return forward_impl(gin, s, S, src_node, nullptr, T, opts_in, cycles, stream);
}

extern "C" int eik_forward_warm(const eik_grid *gin, const double *s, int S, const int *src_node,
                                const double *T_init, double *T, const eik_opts *opts_in, int *cycles, eik_stream stream)
{
    if (!src_node || !T_init) { set_error("bad eik_forward_warm arguments"); return EIK_ERR_INVALID; }
    return forward_impl(gin, s, S, src_node, nullptr, T, opts_in, cycles, stream, T_init);
}

extern "C" int eik_forward_points(const eik_grid *gin, const double *s, int S, const double *src_f, double *T,
                                  const eik_opts *opts_in, int *cycles, eik_stream stream)
{
    if (!src_f) { set_error("bad eik_forward_points arguments"); return EIK_ERR_INVALID; }
    return forward_impl(gin, s, S, nullptr, src_f, T, opts_in, cycles, stream);
}

// ---------------------------------------------------------------------------------
// eik_forward_noalloc: the same state solve for callers that must not allocate device
// memory.  Its scratch lives in one file-scope device array of fixed size instead of
// cudaMalloc'd buffers.  Host code may not pass the array's name to a kernel (on the
// host it is only a stand-in symbol); the device address is looked up once per device
// with cudaGetSymbolAddress, with that device current, on the first call there.
// ---------------------------------------------------------------------------------
#include <mutex>

#define EIK_NOALLOC_SCRATCH_BYTES (64ull << 20)

static __device__ __align__(256) unsigned char g_eik_noalloc_scratch[EIK_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// bytes of scratch one call needs (same buffers eik_forward allocates)
size_t noalloc_bytes(int nd, long long N, int S)
{
    const long long SN = N * S;
    size_t b = 0;
    b += align256((size_t)N * nd * nd * sizeof(double));     // G
    b += align256((size_t)N * nd * nd * sizeof(double));     // J
    b += align256((size_t)SN * sizeof(double));              // T0
    b += align256((size_t)SN * nd * sizeof(double));         // g0
    b += align256((size_t)SN * nd * sizeof(double));         // alpha
    b += align256((size_t)SN * sizeof(double));              // tau
    b += align256((size_t)SN);                               // fixed flags
    b += align256((size_t)S * sizeof(int));                  // source nodes
    b += align256((size_t)S * DSLOTS * sizeof(unsigned long long));   // max change per source
    b += align256((size_t)S);                                // active flags
    b += align256((size_t)S * sizeof(double));               // FP32 thresholds
    return b;
}

int scratch_for_current_device(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
    if (dev < 0 || dev >= kMaxDevices) { set_error("device index %d not supported", dev); return EIK_ERR_INVALID; }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_eik_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
    return EIK_OK;
}
}  // namespace

extern "C" size_t eik_forward_noalloc_capacity(void) { return (size_t)EIK_NOALLOC_SCRATCH_BYTES; }

extern "C" int eik_forward_noalloc(const eik_grid *gin, const double *s, int S, const int *src_node, double *T,
                                   const eik_opts *opts_in, int *cycles, eik_stream stream)
{
    try {
        if (!gin || (gin->ndim != 2 && gin->ndim != 3) || !gin->xyz || !s || !T || !src_node || S <= 0) {
            set_error("bad eik_forward_noalloc arguments");
            return EIK_ERR_INVALID;
        }
        eik_opts def;
        eik_opts_default(&def);
        const eik_opts *opts = opts_in ? opts_in : &def;
        GridDesc g = make_grid_desc(gin);
        for (int d = 0; d < g.ndim; ++d)
            if (g.n[d] < 3) { set_error("grid needs >= 3 nodes per axis"); return EIK_ERR_INVALID; }
        for (int a = 0; a < S; ++a)
            if (src_node[a] < 0 || src_node[a] >= g.N) { set_error("source node out of range"); return EIK_ERR_INVALID; }
        const int nd = g.ndim;
        const long long N = g.N, SN = N * S;
        const size_t need = noalloc_bytes(nd, N, S);
        if (need > EIK_NOALLOC_SCRATCH_BYTES) {
            set_error("eik_forward_noalloc needs %zu bytes of scratch for %d sources x %lld nodes; its fixed "
                      "scratch holds %zu bytes (use eik_forward)", need, S, N, (size_t)EIK_NOALLOC_SCRATCH_BYTES);
            return EIK_ERR_INVALID;
        }
        unsigned char *base = nullptr;
        int rc = scratch_for_current_device(&base);
        if (rc) return rc;
        size_t off = 0;
        auto carve = [&](size_t bytes) { unsigned char *p = base + off; off += align256(bytes); return p; };
        double *G = (double *)carve((size_t)N * nd * nd * sizeof(double));
        double *Jm = (double *)carve((size_t)N * nd * nd * sizeof(double));
        double *T0 = (double *)carve((size_t)SN * sizeof(double));
        double *g0 = (double *)carve((size_t)SN * nd * sizeof(double));
        double *alpha = (double *)carve((size_t)SN * nd * sizeof(double));
        double *tau = (double *)carve((size_t)SN * sizeof(double));
        unsigned char *fixed = carve((size_t)SN);
        int *src_d = (int *)carve((size_t)S * sizeof(int));
        unsigned long long *dmax = (unsigned long long *)carve((size_t)S * DSLOTS * sizeof(unsigned long long));
        unsigned char *active = carve((size_t)S);
        double *t0_fp64 = (double *)carve((size_t)S * sizeof(double));
        cudaStream_t st = (cudaStream_t)stream;
        // on a failure after work was queued, wait for that work before returning: the next
        // call reuses the same scratch array and must not race with leftovers of this one
#define TRY(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { cudaStreamSynchronize(st); cudaGetLastError(); \
                                                                      return cuda_fail(e_, #call, __FILE__, __LINE__); } } while (0)
        TRY(cudaMemcpyAsync(src_d, src_node, S * sizeof(int), cudaMemcpyHostToDevice, st));
        double hmax = 0.0;
        for (int d = 0; d < nd; ++d) hmax = std::max(hmax, g.dxi[d]);
        // every buffer is fully rewritten below (tau by the prep kernel, dmax per cycle),
        // so contents left by an earlier call do not matter
        k_metric<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(g, gin->xyz, G, Jm);
        k_eik_prep<<<(unsigned)((SN + 255) / 256), 256, 0, st>>>(g, S, gin->xyz, Jm, G, s, src_d,
                                                                  opts->eik_src_radius * hmax, T0, g0, alpha, fixed, tau);
        TRY(cudaGetLastError());
        LFParams P{};
        P.g = g; P.S = S; P.G = G; P.s = s; P.T0 = T0; P.g0 = g0; P.alpha = alpha; P.fixed = fixed; P.tau = tau;
        P.dmax = dmax; P.active = active;
        P.fp32 = opts->eik_fp32 ? 1 : 0; P.t0_fp64 = t0_fp64;
        k_t0_threshold<<<(S + 127) / 128, 128, 0, st>>>(S, s, src_d, opts->eik_fp64_radius * hmax, t0_fp64);
        const double tol = opts->eik_fp32 ? std::max(opts->eik_tol, 1e-6) : opts->eik_tol;
        const int m0 = g.n[0] - 2, m1 = g.n[1] - 2, m2 = nd == 3 ? g.n[2] - 2 : 1;
        const int hmax_i = (m0 - 1) + (m1 - 1) + (nd == 3 ? m2 - 1 : 0);
        const int nord = 1 << nd;
        // each source stops at the first cycle whose largest change is below eik_tol; direct
        // launches (a graph would be one more object to create)
        int used = -1;
        TRY(lf_cycles(P, S, SN, m0, m1, hmax_i, nord, tol, opts->eik_max_cycles, false, &used, st));
        k_eik_out<<<(unsigned)((SN + 255) / 256), 256, 0, st>>>(N, S, T0, tau, T);
        TRY(cudaGetLastError());
        TRY(cudaStreamSynchronize(st));
#undef TRY
        if (cycles) *cycles = used < 0 ? opts->eik_max_cycles : used;
        if (used < 0) { set_error("eik_forward_noalloc did not converge in %d cycles", opts->eik_max_cycles); return EIK_ERR_NOT_CONVERGED; }
        return EIK_OK;
    } catch (...) {
        set_error("eik_forward_noalloc failed");
        return EIK_ERR_INVALID;
    }
}
