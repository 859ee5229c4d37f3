// C-ABI entry points of libeik (declared in include/eik.h).
#include <cuda_runtime.h>

#include <cstring>
#include <exception>
#include <new>

#include "eik_internal.h"

namespace eik { const char *last_error(); }

using eik::Tangent;

#define EIK_GUARD(...)                                                      \
    try { __VA_ARGS__ }                                                          \
    catch (const std::bad_alloc &) { eik::set_error("host out of memory"); return EIK_ERR_OOM; } \
    catch (const std::exception &e) { eik::set_error("%s", e.what()); return EIK_ERR_INVALID; } \
    catch (...) { eik::set_error("unknown failure"); return EIK_ERR_INVALID; }

struct eik_tangent { Tangent *impl; };

extern "C" {

void eik_opts_default(eik_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->model = EIK_MODEL_SLOWNESS;
    o->lu_pivot_tol = 1e-13;
    o->schedule = EIK_SCHED_PERSISTENT;
    o->threads = 256;
    o->chunk = 0;
    o->ctas_per_sm = 0;
    o->wait_timeout_s = 2.0;
    o->eik_tol = 1e-12;
    o->eik_max_cycles = 2000;
    o->eik_src_radius = 1.0;
    o->sweep_tol = 1e-12;
    o->sweep_max_cycles = 10000;
    o->rhs_chunk = 0;
    o->eik_fp32 = 0;
    o->eik_fp64_radius = 8.0;
    o->item_deps = 1;
    o->block_lu_min = 0;
}

const char *eik_last_error(void) { return eik::last_error(); }

const char *eik_version(void) { return "libeik 0.1 sm_103a"; }

static int check_grid(const eik_grid *g)
{
    if (!g || (g->ndim != 2 && g->ndim != 3) || !g->xyz) { eik::set_error("bad grid"); return EIK_ERR_INVALID; }
    for (int d = 0; d < g->ndim; ++d)
        if (g->n[d] < 3 || !(g->dxi[d] > 0)) { eik::set_error("grid needs >= 3 nodes and positive spacing per axis"); return EIK_ERR_INVALID; }
    return EIK_OK;
}

int tangent_build(const eik_grid *g, const double *T, const double *s, int S, const int *src_node,
                  const int *rec_node, int n_rec, const eik_opts *opts, eik_tangent **out, eik_stream stream)
{
    EIK_GUARD({
        if (!out) { eik::set_error("out is NULL"); return EIK_ERR_INVALID; }
        *out = nullptr;
        int rc = check_grid(g);
        if (rc) return rc;
        if (S <= 0 || !T || !s || !src_node || n_rec < 0 || (n_rec > 0 && !rec_node)) {
            eik::set_error("bad tangent_build arguments");
            return EIK_ERR_INVALID;
        }
        eik_opts def;
        eik_opts_default(&def);
        Tangent *t = nullptr;
        rc = eik::build_tangent(g, T, s, S, src_node, rec_node, n_rec, opts ? opts : &def, &t, (cudaStream_t)stream);
        if (rc) return rc;
        *out = new eik_tangent{t};
        return EIK_OK;
    })
}

int tangent_build_points(const eik_grid *g, const double *T, const double *s, int S, const double *src_f,
                         const int *rec_node, int n_rec, const eik_opts *opts, eik_tangent **out, eik_stream stream)
{
    EIK_GUARD({
        if (!out) { eik::set_error("out is NULL"); return EIK_ERR_INVALID; }
        *out = nullptr;
        int rc = check_grid(g);
        if (rc) return rc;
        if (S <= 0 || !T || !s || !src_f || n_rec < 0 || (n_rec > 0 && !rec_node)) {
            eik::set_error("bad tangent_build_points arguments");
            return EIK_ERR_INVALID;
        }
        eik_opts def;
        eik_opts_default(&def);
        Tangent *t = nullptr;
        rc = eik::build_tangent(g, T, s, S, nullptr, rec_node, n_rec, opts ? opts : &def, &t, (cudaStream_t)stream,
                                src_f);
        if (rc) return rc;
        *out = new eik_tangent{t};
        return EIK_OK;
    })
}

int tangent_apply(eik_tangent *t, const void *p, int shared_model, int R, void *dT_full, void *d_rec, int dtype,
                  eik_stream stream)
{
    EIK_GUARD({
        if (!t) { eik::set_error("tangent is NULL"); return EIK_ERR_INVALID; }
        if (d_rec && t->impl->n_rec == 0) { eik::set_error("tangent has no receivers"); return EIK_ERR_INVALID; }
        return eik::traverse(t->impl, false, eik::MODE_J, p, shared_model, R, dT_full, d_rec, 0, dtype,
                             (cudaStream_t)stream);
    })
}

int tangent_apply_T(eik_tangent *t, const void *y, int R, int sum_sources, void *g, void *lam_full, int dtype,
                    eik_stream stream)
{
    EIK_GUARD({
        if (!t) { eik::set_error("tangent is NULL"); return EIK_ERR_INVALID; }
        if (t->impl->n_rec == 0) { eik::set_error("tangent has no receivers"); return EIK_ERR_INVALID; }
        if (sum_sources < 0 || sum_sources > 2) { eik::set_error("sum_sources must be 0, 1 or 2"); return EIK_ERR_INVALID; }
        return eik::traverse(t->impl, true, eik::MODE_J, y, 0, R, lam_full, g, sum_sources, dtype,
                             (cudaStream_t)stream);
    })
}

static int batch_entry(eik_tangent *const *t, int ntan, bool tr, const void *const *in, const int *R,
                       void *const *out, int dtype, eik_stream stream)
{
    EIK_GUARD({
        if (!t || !in || !R || !out || ntan < 1 || ntan > 4) { eik::set_error("bad batch arguments"); return EIK_ERR_INVALID; }
        Tangent *ts[4];
        for (int k = 0; k < ntan; ++k) {
            if (!t[k]) { eik::set_error("batch: tangent %d is NULL", k); return EIK_ERR_INVALID; }
            ts[k] = t[k]->impl;
        }
        return eik::traverse_batch(ts, ntan, tr, in, R, out, dtype, (cudaStream_t)stream);
    })
}

int tangent_apply_batch(eik_tangent *const *t, int ntan, const void *const *p, const int *R, void *const *d_rec,
                        int dtype, eik_stream stream)
{
    return batch_entry(t, ntan, false, p, R, d_rec, dtype, stream);
}

int tangent_apply_T_batch(eik_tangent *const *t, int ntan, const void *const *y, const int *R, void *const *g,
                          int dtype, eik_stream stream)
{
    return batch_entry(t, ntan, true, y, R, g, dtype, stream);
}

int tangent_set_receivers(eik_tangent *t, int n_rec, const double *f)
{
    EIK_GUARD({
        if (!t || n_rec < 0 || (n_rec > 0 && !f)) { eik::set_error("bad tangent_set_receivers arguments"); return EIK_ERR_INVALID; }
        EIK_CHECK(cudaDeviceSynchronize());
        return eik::set_receivers_interp(t->impl, n_rec, f);
    })
}

int tangent_apply_interp(eik_tangent *t, const void *ds, int shared_model, int R, void *d_rec, int dtype,
                         eik_stream stream)
{
    EIK_GUARD({
        if (!t || !ds || !d_rec || R <= 0) { eik::set_error("bad tangent_apply_interp arguments"); return EIK_ERR_INVALID; }
        return eik::apply_interp_entry(t->impl, ds, shared_model, R, d_rec, dtype, (cudaStream_t)stream);
    })
}

int tangent_apply_interp_T(eik_tangent *t, const void *y, int R, void *g, int dtype, eik_stream stream)
{
    EIK_GUARD({
        if (!t || !y || !g || R <= 0) { eik::set_error("bad tangent_apply_interp_T arguments"); return EIK_ERR_INVALID; }
        return eik::apply_interp_T_entry(t->impl, y, R, g, dtype, (cudaStream_t)stream);
    })
}

int tangent_solve(eik_tangent *t, const void *q, int R, void *x, int dtype, eik_stream stream)
{
    EIK_GUARD({
        if (!t || !x) { eik::set_error("tangent or output is NULL"); return EIK_ERR_INVALID; }
        return eik::traverse(t->impl, false, eik::MODE_RAW, q, 0, R, x, nullptr, 0, dtype, (cudaStream_t)stream);
    })
}

int tangent_solve_T(eik_tangent *t, const void *r, int R, void *x, int dtype, eik_stream stream)
{
    EIK_GUARD({
        if (!t || !x) { eik::set_error("tangent or output is NULL"); return EIK_ERR_INVALID; }
        return eik::traverse(t->impl, true, eik::MODE_RAW, r, 0, R, x, nullptr, 0, dtype, (cudaStream_t)stream);
    })
}

int tangent_sample(const eik_tangent *tt, const double *field, double *out, eik_stream stream)
{
    EIK_GUARD({
        if (!tt || !field || !out) { eik::set_error("bad tangent_sample arguments"); return EIK_ERR_INVALID; }
        Tangent *t = tt->impl;
        long long n = (long long)t->S * t->n_rec;
        if (n == 0) return EIK_OK;
        eik::launch_sample(t->N, t->S, t->n_rec, t->rec_nat, field, out, (cudaStream_t)stream);
        EIK_CHECK_LAUNCH();
        return EIK_OK;
    })
}

int tangent_stats(const eik_tangent *t, int source, eik_stats *out)
{
    if (!t || !out || source < 0 || source >= t->impl->S) { eik::set_error("bad tangent_stats arguments"); return EIK_ERR_INVALID; }
    *out = t->impl->stats[source];
    return EIK_OK;
}

int tangent_dims(const eik_tangent *t, int *S, int64_t *N, int *n_rec)
{
    if (!t) { eik::set_error("tangent is NULL"); return EIK_ERR_INVALID; }
    if (S) *S = t->impl->S;
    if (N) *N = t->impl->N;
    if (n_rec) *n_rec = t->impl->n_rec;
    return EIK_OK;
}

int tangent_export(const eik_tangent *tt, int source, int *label, int *level, int *perm, int64_t *level_ptr,
                   int64_t *row_ptr, int *col, double *w, double *cs)
{
    EIK_GUARD({
        if (!tt || source < 0 || source >= tt->impl->S) { eik::set_error("bad tangent_export arguments"); return EIK_ERR_INVALID; }
        Tangent *t = tt->impl;
        const long long N = t->N, off = (long long)source * N;
        const int slots = 2 * t->grid.ndim;
        EIK_CHECK(cudaDeviceSynchronize());
        if (label) EIK_CHECK(cudaMemcpy(label, t->label + off, N * sizeof(int), cudaMemcpyDeviceToHost));
        if (level) EIK_CHECK(cudaMemcpy(level, t->level + off, N * sizeof(int), cudaMemcpyDeviceToHost));
        if (perm) {
            EIK_CHECK(cudaMemcpy(perm, t->perm + off, N * sizeof(int), cudaMemcpyDeviceToHost));
            for (long long p = 0; p < N; ++p) if (perm[p] < 0) perm[p] = ~perm[p];
        }
        if (level_ptr) {
            for (int L = 0; L <= t->nlev[source]; ++L)
                level_ptr[L] = t->level_ptr[(size_t)source * (t->maxL + 1) + L];
        }
        if (row_ptr || col || w) {
            std::vector<int> cnt(N), nn((size_t)N * slots);
            std::vector<double> nw((size_t)N * slots);
            EIK_CHECK(cudaMemcpy(cnt.data(), t->nrow_cnt + off, N * sizeof(int), cudaMemcpyDeviceToHost));
            EIK_CHECK(cudaMemcpy(nn.data(), t->nrow_node + off * slots, (size_t)N * slots * sizeof(int), cudaMemcpyDeviceToHost));
            EIK_CHECK(cudaMemcpy(nw.data(), t->nrow_w + off * slots, (size_t)N * slots * sizeof(double), cudaMemcpyDeviceToHost));
            long long e = 0;
            for (long long i = 0; i < N; ++i) {
                if (row_ptr) row_ptr[i] = e;
                for (int k = 0; k < cnt[i]; ++k, ++e) {
                    if (col) col[e] = nn[(size_t)i * slots + k];
                    if (w) w[e] = nw[(size_t)i * slots + k];
                }
            }
            if (row_ptr) row_ptr[N] = e;
        }
        if (cs) EIK_CHECK(cudaMemcpy(cs, t->cs_nat + off, N * sizeof(double), cudaMemcpyDeviceToHost));
        return EIK_OK;
    })
}

int tangent_status(eik_tangent *tt, eik_stream stream)
{
    EIK_GUARD({
        if (!tt) { eik::set_error("tangent is NULL"); return EIK_ERR_INVALID; }
        Tangent *t = tt->impl;
        int e[4] = {0, 0, 0, 0};
        EIK_CHECK(cudaMemcpyAsync(e, t->err, sizeof e, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
        EIK_CHECK(cudaStreamSynchronize((cudaStream_t)stream));
        EIK_CHECK(cudaMemsetAsync(t->err, 0, sizeof e, (cudaStream_t)stream));
        EIK_CHECK(cudaStreamSynchronize((cudaStream_t)stream));
        if (e[0] == eik::DEV_TIMEOUT) {
            eik::set_error("device wait timed out (source %d, step %d, item %d)", e[1], e[2], e[3]);
            return EIK_ERR_TIMEOUT;
        }
        if (e[0] == eik::DEV_SINGULAR) { eik::set_error("singular SCC block"); return EIK_ERR_SINGULAR_BLOCK; }
        if (e[0] == eik::DEV_BAD_INDEX) {
            eik::set_error("index out of range (checked build): source %d, position %d, value %d", e[1], e[2], e[3]);
            return EIK_ERR_CUDA;
        }
        if (e[0] != 0) { eik::set_error("device fault code %d", e[0]); return EIK_ERR_CUDA; }
        return EIK_OK;
    })
}

int tangent_tune(eik_tangent *tt, const eik_opts *o)
{
    if (!tt || !o) { eik::set_error("bad tangent_tune arguments"); return EIK_ERR_INVALID; }
    if (o->schedule < EIK_SCHED_PERSISTENT || o->schedule > EIK_SCHED_SYNC) { eik::set_error("bad schedule"); return EIK_ERR_INVALID; }
    if (o->rhs_chunk < 0 || o->ctas_per_sm < 0 || !(o->wait_timeout_s > 0) || o->block_lu_min < 0 || o->item_slots < 0 ||
        o->item_slots > 4) { eik::set_error("bad tuning values"); return EIK_ERR_INVALID; }
    Tangent *t = tt->impl;
    if (o->split_dirs) {
        int rc = EIK_OK;
        EIK_GUARD({ rc = eik::enable_split(t); });
        if (rc) return rc;
    }
    t->opts.split_dirs = o->split_dirs ? 1 : 0;
    t->opts.schedule = o->schedule;
    t->opts.ctas_per_sm = o->ctas_per_sm;
    t->opts.rhs_chunk = o->rhs_chunk;
    t->opts.wait_timeout_s = o->wait_timeout_s;
    t->opts.item_deps = o->item_deps;
    t->opts.cluster_size = o->cluster_size;
    t->opts.cluster_threads = o->cluster_threads;
    t->opts.pass_units = o->pass_units;
    t->opts.block_lu_min = o->block_lu_min;
    t->opts.item_slots = o->item_slots;
    return EIK_OK;
}

int tangent_debug_poke_edge(eik_tangent *tt, int source, long long edge, int value)
{
    EIK_GUARD({
        if (!tt) { eik::set_error("tangent is NULL"); return EIK_ERR_INVALID; }
#ifndef EIK_CHECKED
        (void)source; (void)edge; (void)value;
        eik::set_error("tangent_debug_poke_edge needs the checked build");
        return EIK_ERR_INVALID;
#else
        Tangent *t = tt->impl;
        if (source < 0 || source >= t->S) { eik::set_error("bad source"); return EIK_ERR_INVALID; }
        const long long ne = t->ebase[source + 1] - t->ebase[source];
        if (edge < 0 || edge >= ne) { eik::set_error("edge %lld outside [0, %lld)", edge, ne); return EIK_ERR_INVALID; }
        EIK_CHECK(cudaDeviceSynchronize());
        EIK_CHECK(cudaMemcpy(t->up_node + t->ebase[source] + edge, &value, sizeof(int), cudaMemcpyHostToDevice));
        return EIK_OK;
#endif
    })
}

int tangent_debug_hold(eik_tangent *tt, int source, int step)
{
    EIK_GUARD({
        if (!tt) { eik::set_error("tangent is NULL"); return EIK_ERR_INVALID; }
        Tangent *t = tt->impl;
        if (source < 0) {
            for (auto &h : t->holds) {
                int v = 0;
                EIK_CHECK(cudaMemcpy(&v, t->item_cnt + h, sizeof(int), cudaMemcpyDeviceToHost));
                --v;
                EIK_CHECK(cudaMemcpy(t->item_cnt + h, &v, sizeof(int), cudaMemcpyHostToDevice));
            }
            t->holds.clear();
            return EIK_OK;
        }
        if (source >= t->S || step < 0 || step >= t->nlev[source]) { eik::set_error("bad hold position"); return EIK_ERR_INVALID; }
        long long h = (long long)source * t->maxL + step;
        int v = 0;
        EIK_CHECK(cudaDeviceSynchronize());
        EIK_CHECK(cudaMemcpy(&v, t->item_cnt + h, sizeof(int), cudaMemcpyDeviceToHost));
        ++v;
        EIK_CHECK(cudaMemcpy(t->item_cnt + h, &v, sizeof(int), cudaMemcpyHostToDevice));
        t->holds.push_back(h);
        return EIK_OK;
    })
}

void tangent_free(eik_tangent *t)
{
    if (!t) return;
    cudaDeviceSynchronize();
    eik::free_tangent(t->impl);
    delete t;
}

int sweep_apply(eik_tangent *t, int transpose, const void *b, int R, void *x, int dtype, const eik_opts *opts,
                int *cycles, eik_stream stream)
{
    EIK_GUARD({
        if (!t || !b || !x || R <= 0) { eik::set_error("bad sweep_apply arguments"); return EIK_ERR_INVALID; }
        eik_opts def;
        eik_opts_default(&def);
        return eik::sweep(t->impl, transpose != 0, b, R, x, dtype, opts ? opts : &def, cycles, (cudaStream_t)stream);
    })
}

}  // extern "C"
