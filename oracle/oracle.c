/*
 * CPU FP64 oracle for the frozen full-metric Eikonal tangent transport.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load or call this
 * file: only the tests, the smoke check and the benchmark's CPU-baseline leg do.
 * It shares no code, header or table with the CUDA library.
 *
 * Plain, slow, single-threaded C; every function follows one passage of the paper
 * (arxiv 2609.14982) and is written for a reader checking it against the text.
 * Build with -O2 -ffp-contract=off so that no multiply-add is fused: the upwind
 * decision (sign of a_f) must come out of the exact operation sequence stated here.
 *
 * Conventions: logical dims 3-D (xi, eta, zeta) or 2-D (xi, zeta); node (i,j,k) has
 * linear index (i*n1 + j)*n2 + k (2-D: i*n1 + k); xyz is [N][ndim].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* grid helpers                                                              */
/* ------------------------------------------------------------------------ */
static void strides(int ndim, const int *n, long *st)
{
    if (ndim == 3) { st[2] = 1; st[1] = n[2]; st[0] = (long)n[1] * n[2]; }
    else           { st[1] = 1; st[0] = n[1]; }
}

static void coords(int ndim, const int *n, long i, int *idx)
{
    if (ndim == 3) { idx[2] = (int)(i % n[2]); idx[1] = (int)((i / n[2]) % n[1]); idx[0] = (int)(i / ((long)n[1] * n[2])); }
    else           { idx[1] = (int)(i % n[1]); idx[0] = (int)(i / n[1]); }
}

/* d f / d xi_b at a node, for a field with `ncomp` interleaved components.
 * Interior: central (f+ - f-)/(2h).  Edges: second-order one-sided
 * (-3 f0 + 4 f1 - f2)/(2h) and (3 fn - 4 f(n-1) + f(n-2))/(2h).
 * (Sec. 2.2: J = dx/dxi is formed from the node coordinates; the same stencil is
 * used for the nodal logical gradient of T.) */
static double fd1(const double *f, int ncomp, int comp, long i, int idxb, int nb, long stb, double h)
{
    double t;
    if (idxb == 0) {
        double f0 = f[i * ncomp + comp], f1 = f[(i + stb) * ncomp + comp], f2 = f[(i + 2 * stb) * ncomp + comp];
        t = (-3.0 * f0 + 4.0 * f1) - f2;
    } else if (idxb == nb - 1) {
        double f0 = f[i * ncomp + comp], f1 = f[(i - stb) * ncomp + comp], f2 = f[(i - 2 * stb) * ncomp + comp];
        t = (3.0 * f0 - 4.0 * f1) + f2;
    } else {
        t = f[(i + stb) * ncomp + comp] - f[(i - stb) * ncomp + comp];
    }
    return t / (2.0 * h);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2, Eq. (metric-eikonal): J_ab = dx_a/dxi_b, G = J^{-1} J^{-T}       */
/* ------------------------------------------------------------------------ */
int or_metric(int ndim, const int *n, const double *dxi, const double *xyz,
              double *Jout /* [N][ndim][ndim] */, double *G /* [N][ndim][ndim] */, double *detJ /* [N] */)
{
    long st[3], N = 1;
    int idx[3];
    for (int d = 0; d < ndim; ++d) { N *= n[d]; if (n[d] < 3) return -1; }
    strides(ndim, n, st);
    for (long i = 0; i < N; ++i) {
        double J[3][3], K[3][3];
        coords(ndim, n, i, idx);
        for (int a = 0; a < ndim; ++a)
            for (int b = 0; b < ndim; ++b)
                J[a][b] = fd1(xyz, ndim, a, i, idx[b], n[b], st[b], dxi[b]);
        double det;
        if (ndim == 3) {
            /* K = adj(J)/det(J), adj = transposed cofactor matrix */
            double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
            double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
            double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
            double c10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
            double c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
            double c12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
            double c20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
            double c21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
            double c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            det = (J[0][0] * c00 + J[0][1] * c01) + J[0][2] * c02;
            K[0][0] = c00 / det; K[1][0] = c01 / det; K[2][0] = c02 / det;
            K[0][1] = c10 / det; K[1][1] = c11 / det; K[2][1] = c12 / det;
            K[0][2] = c20 / det; K[1][2] = c21 / det; K[2][2] = c22 / det;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    G[i * 9 + a * 3 + b] = (K[a][0] * K[b][0] + K[a][1] * K[b][1]) + K[a][2] * K[b][2];
        } else {
            det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            K[0][0] = J[1][1] / det; K[0][1] = -J[0][1] / det;
            K[1][0] = -J[1][0] / det; K[1][1] = J[0][0] / det;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    G[i * 4 + a * 2 + b] = K[a][0] * K[b][0] + K[a][1] * K[b][1];
        }
        if (Jout) for (int a = 0; a < ndim; ++a) for (int b = 0; b < ndim; ++b) Jout[i * ndim * ndim + a * ndim + b] = J[a][b];
        if (detJ) detJ[i] = det;
    }
    return 0;
}

/* nodal logical gradient of a scalar field, same stencil as the metric */
int or_grad(int ndim, const int *n, const double *dxi, const double *f, double *g /* [N][ndim] */)
{
    long st[3], N = 1;
    int idx[3];
    for (int d = 0; d < ndim; ++d) { N *= n[d]; if (n[d] < 3) return -1; }
    strides(ndim, n, st);
    for (long i = 0; i < N; ++i) {
        coords(ndim, n, i, idx);
        for (int b = 0; b < ndim; ++b) g[i * ndim + b] = fd1(f, 1, 0, i, idx[b], n[b], st[b], dxi[b]);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1-3.2, Eqs. (discrete-row), (transport-system): face-based upwind  */
/* rows A = I - W in gather form, and the calibration c^(s) = (A T)_i / s_i.  */
/*                                                                            */
/* For node i, direction d and side sg in {-1, +1} with neighbour j = i+sg e_d:*/
/*   G_f = (G_i + G_j)/2,                                                     */
/*   g_f = (gradT_i + gradT_j)/2 with component d replaced by the compact     */
/*         difference across the face, (T_i - T_j)/h_d (sg=-1) or             */
/*         (T_j - T_i)/h_d (sg=+1),                                           */
/*   a_f = sum_b G_f[d][b] g_f[b]  (b ascending),                             */
/*   c_ij = max(0, -sg a_f)/h_d: j is upstream iff c_ij > 0.                   */
/* Faces are visited d ascending, sg = -1 then +1.  d_i = sum c_ij (in that   */
/* order), w_ij = c_ij/d_i.  The source node is a seed row (identity, q = 0); */
/* a non-seed row with no upstream face is an identity row.                   */
/* row_type: 0 interior, 1 seed, 2 identity (no upstream).                    */
/* Returns nnz, or -1 on bad input.                                           */
/* ------------------------------------------------------------------------ */
static int in_list(long i, const long *list, int n)
{
    for (int k = 0; k < n; ++k)
        if (list[k] == i) return 1;
    return 0;
}

/* The same rows with a set of seed rows (an on-grid source: its node; an off-grid point */
/* source: the corners of its cell).                                                     */
long or_assemble_seeds(int ndim, const int *n, const double *dxi, const double *G, const double *gradT,
                       const double *T, const double *s, const long *seeds, int nseeds,
                       long *row_ptr, int *col, double *cw, double *w, double *cs, int *row_type);

long or_assemble(int ndim, const int *n, const double *dxi, const double *G, const double *gradT,
                 const double *T, const double *s, long src,
                 long *row_ptr /* [N+1] */, int *col /* [2 ndim N] */, double *cw /* c_ij */,
                 double *w, double *cs /* [N] */, int *row_type /* [N] */)
{
    return or_assemble_seeds(ndim, n, dxi, G, gradT, T, s, &src, 1, row_ptr, col, cw, w, cs, row_type);
}

long or_assemble_seeds(int ndim, const int *n, const double *dxi, const double *G, const double *gradT,
                       const double *T, const double *s, const long *seeds, int nseeds,
                       long *row_ptr, int *col, double *cw, double *w, double *cs, int *row_type)
{
    long st[3], N = 1, nnz = 0;
    int idx[3];
    const int nd2 = ndim * ndim;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    strides(ndim, n, st);
    for (long i = 0; i < N; ++i) {
        row_ptr[i] = nnz;
        coords(ndim, n, i, idx);
        if (in_list(i, seeds, nseeds)) { row_type[i] = 1; cs[i] = 0.0; continue; }
        long start = nnz;
        for (int d = 0; d < ndim; ++d) {
            for (int sg = -1; sg <= 1; sg += 2) {
                int nb = idx[d] + sg;
                if (nb < 0 || nb >= n[d]) continue;
                long j = i + sg * st[d];
                double gf[3], af = 0.0;
                for (int b = 0; b < ndim; ++b) gf[b] = (gradT[i * ndim + b] + gradT[j * ndim + b]) * 0.5;
                gf[d] = (sg < 0) ? (T[i] - T[j]) / dxi[d] : (T[j] - T[i]) / dxi[d];
                for (int b = 0; b < ndim; ++b) {
                    double Gf = (G[i * nd2 + d * ndim + b] + G[j * nd2 + d * ndim + b]) * 0.5;
                    af = af + Gf * gf[b];
                }
                double v = (sg < 0) ? af : -af;
                if (v > 0.0) {
                    col[nnz] = (int)j;
                    cw[nnz] = v / dxi[d];
                    ++nnz;
                }
            }
        }
        if (nnz == start) {  /* no upstream face: identity row */
            row_type[i] = 2;
            cs[i] = T[i] / s[i];
            continue;
        }
        double di = 0.0;
        for (long e = start; e < nnz; ++e) di = di + cw[e];
        double acc = 0.0;
        for (long e = start; e < nnz; ++e) {
            w[e] = cw[e] / di;
            acc = acc + w[e] * T[col[e]];
        }
        row_type[i] = 0;
        cs[i] = (T[i] - acc) / s[i];   /* Sec. 3.2: l = A T, c_i = l_i / s_i */
    }
    row_ptr[N] = nnz;
    return nnz;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1: strongly connected components (Tarjan, ref50), iterative.        */
/* Graph: edge j -> i for every j in U(i).  Tarjan is run on the reversed     */
/* edges i -> j, which has the same components.  label[v] = smallest node     */
/* index in v's component.  Returns the number of components.                 */
/* ------------------------------------------------------------------------ */
long or_scc(long N, const long *row_ptr, const int *col, int *label)
{
    long *index = malloc(N * sizeof(long)), *low = malloc(N * sizeof(long));
    char *onstack = calloc(N, 1);
    int *stack = malloc(N * sizeof(int)), *cstack = malloc(N * sizeof(int));
    long *estack = malloc(N * sizeof(long));
    long counter = 0, ncomp = 0;
    long sp = 0, csp = 0;
    for (long v = 0; v < N; ++v) index[v] = -1;
    for (long root = 0; root < N; ++root) {
        if (index[root] >= 0) continue;
        /* call stack of (node, next edge) */
        cstack[csp] = (int)root; estack[csp] = row_ptr[root]; ++csp;
        index[root] = low[root] = counter++;
        stack[sp++] = (int)root; onstack[root] = 1;
        while (csp > 0) {
            int v = cstack[csp - 1];
            long e = estack[csp - 1];
            if (e < row_ptr[v + 1]) {
                estack[csp - 1] = e + 1;
                int u = col[e];
                if (index[u] < 0) {
                    index[u] = low[u] = counter++;
                    stack[sp++] = u; onstack[u] = 1;
                    cstack[csp] = u; estack[csp] = row_ptr[u]; ++csp;
                } else if (onstack[u] && index[u] < low[v]) {
                    low[v] = index[u];
                }
            } else {
                --csp;
                if (low[v] == index[v]) {
                    /* pop the component, label by its minimum node */
                    long top = sp;
                    int mn = v;
                    long k = sp - 1;
                    while (1) { int u = stack[k]; if (u < mn) mn = u; if (u == v) break; --k; }
                    for (long t = k; t < top; ++t) { label[stack[t]] = mn; onstack[stack[t]] = 0; }
                    sp = k;
                    ++ncomp;
                }
                if (csp > 0) {
                    int p = cstack[csp - 1];
                    if (low[v] < low[p]) low[p] = low[v];
                }
            }
        }
    }
    free(index); free(low); free(onstack); free(stack); free(cstack); free(estack);
    return ncomp;
}

/* ------------------------------------------------------------------------ */
/* Canonical condensation order (Sec. 4.1, Eq. block-form; the paper fixes no  */
/* particular topological order): level(C) = 0 without a predecessor component */
/* else 1 + max level of its predecessor components (longest path, Kahn on    */
/* the condensation DAG).  Components are ordered by (level, smallest node),  */
/* nodes inside a component ascending.                                        */
/* Outputs: level[v] (level of v's component), perm[N] (position -> node),   */
/* comp_ptr[ncomp+1] (component boundaries in perm), level_ptr[nlev+1].       */
/* Returns the number of levels, or -1 if the condensation is not acyclic.   */
/* ------------------------------------------------------------------------ */
/* canonical order key: (level, smallest node of the component, node), compared in that order */
typedef struct { long lev, comp, node; } order_key;

static int cmp_key(const void *a, const void *b)
{
    const order_key *x = a, *y = b;
    if (x->lev != y->lev) return (x->lev > y->lev) - (x->lev < y->lev);
    if (x->comp != y->comp) return (x->comp > y->comp) - (x->comp < y->comp);
    return (x->node > y->node) - (x->node < y->node);
}

long or_levels(long N, const long *row_ptr, const int *col, const int *label,
               int *level, int *perm, long *comp_ptr, long *level_ptr, long *ncomp_out)
{
    /* compact component ids by smallest node */
    long *cid = malloc(N * sizeof(long));
    long m = 0;
    for (long v = 0; v < N; ++v) cid[v] = -1;
    long *rep = malloc(N * sizeof(long));
    for (long v = 0; v < N; ++v) if (label[v] == v) { cid[v] = m; rep[m] = v; ++m; }
    for (long v = 0; v < N; ++v) cid[v] = cid[label[v]];
    /* condensation edges with multiplicity: indegree of each component */
    long *indeg = calloc(m, sizeof(long));
    long *outcnt = calloc(m + 1, sizeof(long));
    for (long i = 0; i < N; ++i)
        for (long e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            long cj = cid[col[e]], ci = cid[i];
            if (cj != ci) { indeg[ci]++; outcnt[cj + 1]++; }
        }
    for (long c = 0; c < m; ++c) outcnt[c + 1] += outcnt[c];
    long *succ = malloc((outcnt[m] + 1) * sizeof(long));
    long *fill = malloc((m + 1) * sizeof(long));
    memcpy(fill, outcnt, (m + 1) * sizeof(long));
    for (long i = 0; i < N; ++i)
        for (long e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            long cj = cid[col[e]], ci = cid[i];
            if (cj != ci) succ[fill[cj]++] = ci;
        }
    long *clev = calloc(m, sizeof(long));
    long *queue = malloc(m * sizeof(long));
    long qh = 0, qt = 0, nlev = 0;
    for (long c = 0; c < m; ++c) if (indeg[c] == 0) queue[qt++] = c;
    while (qh < qt) {
        long c = queue[qh++];
        if (clev[c] + 1 > nlev) nlev = clev[c] + 1;
        for (long e = outcnt[c]; e < outcnt[c + 1]; ++e) {
            long d = succ[e];
            if (clev[c] + 1 > clev[d]) clev[d] = clev[c] + 1;
            if (--indeg[d] == 0) queue[qt++] = d;
        }
    }
    long ok = (qt == m);
    if (ok) {
        /* sort nodes by (level, smallest node of component, node) */
        order_key *key = malloc(N * sizeof(order_key));
        for (long v = 0; v < N; ++v) {
            level[v] = (int)clev[cid[v]];
            key[v].lev = clev[cid[v]];
            key[v].comp = label[v];
            key[v].node = v;
        }
        qsort(key, N, sizeof(order_key), cmp_key);
        long nc = 0;
        for (long p = 0; p <= nlev; ++p) level_ptr[p] = -1;
        for (long p = 0; p < N; ++p) {
            int v = (int)key[p].node;
            perm[p] = v;
            if (p == 0 || label[perm[p - 1]] != label[v]) comp_ptr[nc++] = p;
            if (level_ptr[level[v]] < 0) level_ptr[level[v]] = p;
        }
        comp_ptr[nc] = N;
        level_ptr[nlev] = N;
        *ncomp_out = nc;
        free(key);
    }
    free(cid); free(rep); free(indeg); free(outcnt); free(succ); free(fill); free(clev); free(queue);
    return ok ? nlev : -1;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.3: dense LU with partial pivoting of one nontrivial block,          */
/* P_C A_C = L_C U_C.  A is k x k row-major, overwritten by L (unit, below)   */
/* and U; piv[r] = row swapped with r at step r (first max |a| on ties).      */
/* Returns 0, or r+1 if the pivot at step r is exactly zero.                  */
/* ------------------------------------------------------------------------ */
int or_lu(int k, double *A, int *piv)
{
    for (int r = 0; r < k; ++r) {
        int p = r;
        double best = fabs(A[r * k + r]);
        for (int t = r + 1; t < k; ++t)
            if (fabs(A[t * k + r]) > best) { best = fabs(A[t * k + r]); p = t; }
        piv[r] = p;
        if (best == 0.0) return r + 1;
        if (p != r)
            for (int c = 0; c < k; ++c) { double tmp = A[r * k + c]; A[r * k + c] = A[p * k + c]; A[p * k + c] = tmp; }
        for (int t = r + 1; t < k; ++t) {
            double l = A[t * k + r] / A[r * k + r];
            A[t * k + r] = l;
            for (int c = r + 1; c < k; ++c) A[t * k + c] = A[t * k + c] - l * A[r * k + c];
        }
    }
    return 0;
}

/* solve A x = b in place using the factors of or_lu */
void or_lu_solve(int k, const double *LU, const int *piv, double *b)
{
    for (int r = 0; r < k; ++r) if (piv[r] != r) { double t = b[r]; b[r] = b[piv[r]]; b[piv[r]] = t; }
    for (int r = 0; r < k; ++r) for (int c = 0; c < r; ++c) b[r] = b[r] - LU[r * k + c] * b[c];
    for (int r = k - 1; r >= 0; --r) {
        for (int c = r + 1; c < k; ++c) b[r] = b[r] - LU[r * k + c] * b[c];
        b[r] = b[r] / LU[r * k + r];
    }
}

/* solve A^T y = b in place: A^T = U^T L^T P, so U^T z = b, L^T u = z, y = P^T u */
void or_lu_solve_T(int k, const double *LU, const int *piv, double *b)
{
    for (int r = 0; r < k; ++r) {
        for (int c = 0; c < r; ++c) b[r] = b[r] - LU[c * k + r] * b[c];
        b[r] = b[r] / LU[r * k + r];
    }
    for (int r = k - 1; r >= 0; --r) for (int c = r + 1; c < k; ++c) b[r] = b[r] - LU[c * k + r] * b[c];
    for (int r = k - 1; r >= 0; --r) if (piv[r] != r) { double t = b[r]; b[r] = b[piv[r]]; b[piv[r]] = t; }
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1 Prop. 3 / Sec. 4.3: block traversal x = A^{-1} q over the         */
/* condensation order.  Singleton i: x_i = q_i + sum_j w_ij x_j.  Block C:    */
/* b = q_C + W_{C,ext} x_ext, solve A_C x_C = b with its stored factors.      */
/* lu_off[c] is the offset of component c's k*k factors in lu (-1 singleton), */
/* piv_off[c] likewise in piv.  pos[v] = position of v in perm.               */
/* ------------------------------------------------------------------------ */
void or_btf_solve(long N, const long *row_ptr, const int *col, const double *w,
                  const int *perm, long ncomp, const long *comp_ptr,
                  const long *lu_off, const double *lu, const int *piv, const long *piv_off,
                  const double *q, double *x, double *work)
{
    (void)N;
    for (long c = 0; c < ncomp; ++c) {
        long p0 = comp_ptr[c], p1 = comp_ptr[c + 1];
        int k = (int)(p1 - p0);
        if (k == 1) {
            int i = perm[p0];
            double acc = q[i];
            for (long e = row_ptr[i]; e < row_ptr[i + 1]; ++e) acc = acc + w[e] * x[col[e]];
            x[i] = acc;
        } else {
            int lo = perm[p0], hi = perm[p1 - 1];   /* nodes ascending inside the block */
            for (int a = 0; a < k; ++a) {
                int i = perm[p0 + a];
                double acc = q[i];
                for (long e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                    int j = col[e];
                    int inside = 0;
                    if (j >= lo && j <= hi) for (int t = 0; t < k; ++t) if (perm[p0 + t] == j) { inside = 1; break; }
                    if (!inside) acc = acc + w[e] * x[j];
                }
                work[a] = acc;
            }
            or_lu_solve(k, lu + lu_off[c], piv + piv_off[c], work);
            for (int a = 0; a < k; ++a) x[perm[p0 + a]] = work[a];
        }
    }
}

/* transpose traversal lam = A^{-T} r, components in reverse order; the     */
/* column form (cptr, crow, cwv) lists for each j the rows i with j in U(i).  */
void or_btf_solve_T(long N, const long *cptr, const int *crow, const double *cwv,
                    const int *perm, long ncomp, const long *comp_ptr,
                    const long *lu_off, const double *lu, const int *piv, const long *piv_off,
                    const double *r, double *lam, double *work)
{
    (void)N;
    for (long c = ncomp - 1; c >= 0; --c) {
        long p0 = comp_ptr[c], p1 = comp_ptr[c + 1];
        int k = (int)(p1 - p0);
        if (k == 1) {
            int j = perm[p0];
            double acc = r[j];
            for (long e = cptr[j]; e < cptr[j + 1]; ++e) acc = acc + cwv[e] * lam[crow[e]];
            lam[j] = acc;
        } else {
            int lo = perm[p0], hi = perm[p1 - 1];
            for (int a = 0; a < k; ++a) {
                int j = perm[p0 + a];
                double acc = r[j];
                for (long e = cptr[j]; e < cptr[j + 1]; ++e) {
                    int i = crow[e];
                    int inside = 0;
                    if (i >= lo && i <= hi) for (int t = 0; t < k; ++t) if (perm[p0 + t] == i) { inside = 1; break; }
                    if (!inside) acc = acc + cwv[e] * lam[i];
                }
                work[a] = acc;
            }
            or_lu_solve_T(k, lu + lu_off[c], piv + piv_off[c], work);
            for (int a = 0; a < k; ++a) lam[perm[p0 + a]] = work[a];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.6: directional sweeping = Gauss-Seidel over the 2^ndim logical      */
/* orderings, cycled until max|x_new - x_old| <= tol * max|x| over one full   */
/* cycle.  transpose != 0 sweeps A^T (column form).  Returns the number of    */
/* cycles, or -1 if max_cycles is reached.                                    */
/* ------------------------------------------------------------------------ */
long or_sweep(int ndim, const int *n, int transpose, const long *ptr, const int *idx, const double *wv,
              const double *b, double *x, double tol, long max_cycles)
{
    long N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    for (long i = 0; i < N; ++i) x[i] = 0.0;
    (void)transpose;
    int nord = 1 << ndim;
    for (long cyc = 1; cyc <= max_cycles; ++cyc) {
        double dmax = 0.0, xmax = 0.0;
        for (int o = 0; o < nord; ++o) {
            int a[3] = {0, 0, 0};
            int n2 = ndim == 3 ? n[2] : 1, n1 = n[1];
            for (int i0 = 0; i0 < n[0]; ++i0)
                for (int i1 = 0; i1 < n1; ++i1)
                    for (int i2 = 0; i2 < n2; ++i2) {
                        a[0] = (o & 1) ? n[0] - 1 - i0 : i0;
                        a[1] = (o & 2) ? n1 - 1 - i1 : i1;
                        a[2] = (o & 4) ? n2 - 1 - i2 : i2;
                        long v = ndim == 3 ? ((long)a[0] * n1 + a[1]) * n2 + a[2] : (long)a[0] * n1 + a[1];
                        double acc = b[v];
                        for (long e = ptr[v]; e < ptr[v + 1]; ++e) acc = acc + wv[e] * x[idx[e]];
                        double dx = fabs(acc - x[v]);
                        if (dx > dmax) dmax = dx;
                        x[v] = acc;
                    }
        }
        for (long i = 0; i < N; ++i) if (fabs(x[i]) > xmax) xmax = fabs(x[i]);
        if (dmax <= tol * xmax) return cyc;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.5, Prop. 2: Kahn elimination (repeatedly remove vertices with no    */
/* unresolved predecessor).  removed[v] = 1 for eliminated vertices.  Returns */
/* the size of the residual set R.                                            */
/* ------------------------------------------------------------------------ */
long or_kahn_residual(long N, const long *row_ptr, const int *col, char *removed)
{
    long *indeg = malloc(N * sizeof(long)), *optr = calloc(N + 1, sizeof(long));
    for (long i = 0; i < N; ++i) {
        indeg[i] = row_ptr[i + 1] - row_ptr[i];
        for (long e = row_ptr[i]; e < row_ptr[i + 1]; ++e) optr[col[e] + 1]++;
    }
    for (long v = 0; v < N; ++v) optr[v + 1] += optr[v];
    long *fill = malloc((N + 1) * sizeof(long)), *succ = malloc((optr[N] + 1) * sizeof(long));
    memcpy(fill, optr, (N + 1) * sizeof(long));
    for (long i = 0; i < N; ++i)
        for (long e = row_ptr[i]; e < row_ptr[i + 1]; ++e) succ[fill[col[e]]++] = i;
    long *queue = malloc(N * sizeof(long)), qh = 0, qt = 0;
    for (long v = 0; v < N; ++v) { removed[v] = 0; if (indeg[v] == 0) queue[qt++] = v; }
    while (qh < qt) {
        long v = queue[qh++];
        removed[v] = 1;
        for (long e = optr[v]; e < optr[v + 1]; ++e) if (--indeg[succ[e]] == 0) queue[qt++] = succ[e];
    }
    free(indeg); free(optr); free(fill); free(succ); free(queue);
    return N - qt;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1-2.2: first-arrival state of one point source.  The paper cites   */
/* its factored topography-dependent solver without giving it; the oracle    */
/* states one reading: the factored full-metric equation                     */
/*   sqrt(P^T G P) = s,  P = tau g0 + T0 grad_xi tau,  T = T0 tau,            */
/*   T0 = s_src |x - x_src|,  g0 = J^T grad_x T0,                             */
/* solved by Lax-Friedrichs Gauss-Seidel sweeping (Kao, Osher, Qian 2004).    */
/* For each of the 2^ndim orderings: every interior node not within `radius` */
/* of the source (those keep tau = 1) is updated lexicographically with      */
/* node-local viscosity alpha_d = T0 sqrt(G_dd):                              */
/*   p_d = (tau+ - tau-)/(2 h_d),  P_b = tau g0_b + T0 p_b,                   */
/*   H = sqrt(sum_a P_a sum_b G_ab P_b),                                      */
/*   tau = ((s - H) + sum_d alpha_d (tau+ + tau-)/(2 h_d)) / sum_d alpha_d/h_d */
/* then every boundary node takes the value of its nearest interior node     */
/* along the inward diagonal (one step inward along each boundary axis);    */
/* this keeps the iteration monotone.  Start tau = 1; stop when the largest  */
/* change over one cycle is below tol.  Writes T [N]; returns cycles or -1.  */
/* ------------------------------------------------------------------------ */
static long eik_lf_core(int ndim, const int *n, const double *dxi, const double *xyz, const double *s,
                        const double *xsrc, double ss, double radius, double tol, long max_cycles, double *T);

long or_eik_lf(int ndim, const int *n, const double *dxi, const double *xyz, const double *s, long src,
               double radius, double tol, long max_cycles, double *T)
{
    long N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    if (src < 0 || src >= N) return -2;
    return eik_lf_core(ndim, n, dxi, xyz, s, xyz + src * ndim, s[src], radius, tol, max_cycles, T);
}

/* The same solve for a source at a point x_src between nodes with slowness s_src there: */
/* T0 = s_src |x - x_src|, nodes within radius of x_src keep tau = 1.                    */
long or_eik_lf_point(int ndim, const int *n, const double *dxi, const double *xyz, const double *s,
                     const double *xsrc, double ssrc, double radius, double tol, long max_cycles, double *T)
{
    return eik_lf_core(ndim, n, dxi, xyz, s, xsrc, ssrc, radius, tol, max_cycles, T);
}

static long eik_lf_core(int ndim, const int *n, const double *dxi, const double *xyz, const double *s,
                        const double *xsrc, double ss, double radius, double tol, long max_cycles, double *T)
{
    long st[3], N = 1;
    int idx[3];
    const int nd2 = ndim * ndim;
    for (int d = 0; d < ndim; ++d) { N *= n[d]; if (n[d] < 3) return -2; }
    strides(ndim, n, st);
    double *Jm = malloc(N * nd2 * sizeof(double)), *G = malloc(N * nd2 * sizeof(double));
    double *T0 = malloc(N * sizeof(double)), *g0 = malloc(N * ndim * sizeof(double));
    double *alpha = malloc(N * ndim * sizeof(double)), *tau = malloc(N * sizeof(double));
    char *fixed = malloc(N);
    or_metric(ndim, n, dxi, xyz, Jm, G, NULL);
    for (long i = 0; i < N; ++i) {
        double dd[3], r2 = 0.0;
        for (int c = 0; c < ndim; ++c) { dd[c] = xyz[i * ndim + c] - xsrc[c]; r2 = r2 + dd[c] * dd[c]; }
        double r = sqrt(r2);
        T0[i] = ss * r;
        double gx[3];
        for (int c = 0; c < ndim; ++c) gx[c] = r > 0.0 ? ss * dd[c] / r : 0.0;
        for (int b = 0; b < ndim; ++b) {
            double acc = 0.0;
            for (int c = 0; c < ndim; ++c) acc = acc + Jm[i * nd2 + c * ndim + b] * gx[c];
            g0[i * ndim + b] = acc;
        }
        for (int b = 0; b < ndim; ++b) alpha[i * ndim + b] = T0[i] * sqrt(G[i * nd2 + b * ndim + b]);
        fixed[i] = r <= radius;
        tau[i] = 1.0;
    }
    long used = -1;
    int nord = 1 << ndim;
    int lo2 = ndim == 3 ? 1 : 0, hi2 = ndim == 3 ? n[2] - 1 : 1, n2 = ndim == 3 ? n[2] : 1;
    for (long cyc = 1; cyc <= max_cycles && used < 0; ++cyc) {
        double dmax = 0.0;
        for (int o = 0; o < nord; ++o) {
            for (int c0 = 1; c0 < n[0] - 1; ++c0)
                for (int c1 = 1; c1 < n[1] - 1; ++c1)
                    for (int c2 = lo2; c2 < hi2; ++c2) {
                        idx[0] = (o & 1) ? n[0] - 1 - c0 : c0;
                        idx[1] = (o & 2) ? n[1] - 1 - c1 : c1;
                        idx[2] = ndim == 3 ? ((o & 4) ? n2 - 1 - c2 : c2) : 0;
                        long i = ndim == 3 ? ((long)idx[0] * n[1] + idx[1]) * n2 + idx[2] : (long)idx[0] * n[1] + idx[1];
                        if (fixed[i]) continue;
                        double p[3], P[3];
                        for (int d = 0; d < ndim; ++d) p[d] = (tau[i + st[d]] - tau[i - st[d]]) / (2.0 * dxi[d]);
                        for (int b = 0; b < ndim; ++b) P[b] = tau[i] * g0[i * ndim + b] + T0[i] * p[b];
                        double H2 = 0.0;
                        for (int x = 0; x < ndim; ++x) {
                            double row = 0.0;
                            for (int b = 0; b < ndim; ++b) row = row + G[i * nd2 + x * ndim + b] * P[b];
                            H2 = H2 + P[x] * row;
                        }
                        double num = s[i] - sqrt(H2), den = 0.0;
                        for (int d = 0; d < ndim; ++d) {
                            num = num + alpha[i * ndim + d] * (tau[i + st[d]] + tau[i - st[d]]) / (2.0 * dxi[d]);
                            den = den + alpha[i * ndim + d] / dxi[d];
                        }
                        double nv = num / den;
                        if (fabs(nv - tau[i]) > dmax) dmax = fabs(nv - tau[i]);
                        tau[i] = nv;
                    }
            for (long i = 0; i < N; ++i) {
                if (fixed[i]) continue;
                coords(ndim, n, i, idx);
                long step = 0;
                for (int d = 0; d < ndim; ++d) {
                    if (idx[d] == 0) step += st[d];
                    else if (idx[d] == n[d] - 1) step -= st[d];
                }
                if (step == 0) continue;
                double nv = tau[i + step];
                if (fabs(nv - tau[i]) > dmax) dmax = fabs(nv - tau[i]);
                tau[i] = nv;
            }
        }
        if (dmax < tol) used = cyc;
    }
    for (long i = 0; i < N; ++i) T[i] = T0[i] * tau[i];
    free(Jm); free(G); free(T0); free(g0); free(alpha); free(tau); free(fixed);
    return used;
}
