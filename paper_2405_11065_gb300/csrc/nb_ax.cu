// Host glue of the operator: precision and variant dispatch.
//
// Variants of the CUDA-core operator (chosen per mesh and precision by
// nb_autotune, or by the default below):
//   0, 1: k_ax_cc with the smaller / larger number of elements per block,
//         every load issued by the computing threads;
//   2:    k_ax_tma, element data streamed by bulk copies into a two-stage
//         shared-memory ring (even n, when two stages fit in shared memory,
//         and every vector 16-byte aligned).
#include <stdint.h>

#include "nb_internal.h"

namespace nb {

nb_status upload_D_f32(int n, const double *D);
nb_status upload_D_f64(int n, const double *D);
nb_status ax_cc_f32(int n, int mchoice, bool pupd, int sm_count, long long E, const float *G,
                    const float *u, float *w, const float *r, const float *dinv, float *p,
                    CgScalars *scal, double *part, int *grid, cudaStream_t s);
nb_status ax_cc_f64(int n, int mchoice, bool pupd, int sm_count, long long E, const double *G,
                    const double *u, double *w, const double *r, const double *dinv, double *p,
                    CgScalars *scal, double *part, int *grid, cudaStream_t s);
nb_status ax_tma_f32(int n, int mode, int sm_count, long long E, const float *G, const float *u,
                     float *w, const float *r, const float *dinv, float *p, CgScalars *scal,
                     double *part, int *err, int *grid, cudaStream_t s);
nb_status ax_tma_f64(int n, int mode, int sm_count, long long E, const double *G,
                     const double *u, double *w, const double *r, const double *dinv, double *p,
                     CgScalars *scal, double *part, int *err, int *grid, cudaStream_t s);
bool ax_tma_available_f32(int n, bool pupd);
bool ax_tma_available_f64(int n, bool pupd);
nb_status ax_tc(nb_mesh *m, nb_prec prec, bool pupd, const float *u, float *w, const float *r,
                const float *dinv, float *p, CgScalars *scal, double *part, int *grid,
                cudaStream_t s);
nb_status upload_D_tc(int n, const double *D);

nb_status upload_deriv_tables(int n, const double *D64)
{
    NB_TRY(upload_D_f32(n, D64));
    NB_TRY(upload_D_f64(n, D64));
    NB_TRY(upload_D_tc(n, D64));
    return NB_OK;
}

static bool tma_ok(const nb_mesh *m, nb_prec prec)
{
    // both the plain and the fused form must fit for the variant to be offered
    if (prec == NB_FP32) return ax_tma_available_f32(m->n, true) && ax_tma_available_f32(m->n, false);
    if (prec == NB_FP64) return ax_tma_available_f64(m->n, true) && ax_tma_available_f64(m->n, false);
    return false;
}

int ax_variant_count(const nb_mesh *m, nb_prec prec)
{
    if (prec == NB_FP64 || prec == NB_FP32) return tma_ok(m, prec) ? 3 : 2;
    return 1;  // tensor-core kernel: one shape
}

// Default before any autotuning: the bulk-copy kernel where available, else
// the larger element group, except FP64 at high order where two elements per
// block spill registers.
static int default_variant(const nb_mesh *m, nb_prec prec)
{
    if (tma_ok(m, prec)) return 2;
    if (prec == NB_FP64 && m->n >= 12) return 0;
    return 1;
}

static bool aligned16(const void *p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; }

template <typename T>
static nb_status run_cc(nb_mesh *m, nb_prec prec, int v, bool pupd, const T *G, const T *u, T *w,
                        const T *r, const T *dinv, T *p, CgScalars *scal, double *part,
                        int *grid, cudaStream_t s)
{
    if (v == 2 && !(aligned16(u) && aligned16(w) && aligned16(r) && aligned16(dinv) &&
                    aligned16(p)))
        v = 1;  // the bulk copies need 16-byte aligned vectors
    if (v == 2) {
        if (prec == NB_FP64)
            return ax_tma_f64(m->n, pupd ? 1 : 0, m->ctx->sm_count, m->E, (const double *)G,
                              (const double *)u, (double *)w, (const double *)r,
                              (const double *)dinv, (double *)p, scal, part, m->kerr, grid, s);
        return ax_tma_f32(m->n, pupd ? 1 : 0, m->ctx->sm_count, m->E, (const float *)G,
                          (const float *)u,
                          (float *)w, (const float *)r, (const float *)dinv, (float *)p, scal,
                          part, m->kerr, grid, s);
    }
    if (prec == NB_FP64)
        return ax_cc_f64(m->n, v, pupd, m->ctx->sm_count, m->E, (const double *)G,
                         (const double *)u, (double *)w, (const double *)r, (const double *)dinv,
                         (double *)p, scal, part, grid, s);
    return ax_cc_f32(m->n, v, pupd, m->ctx->sm_count, m->E, (const float *)G, (const float *)u,
                     (float *)w, (const float *)r, (const float *)dinv, (float *)p, scal, part,
                     grid, s);
}

static int variant_of(const nb_mesh *m, nb_prec prec)
{
    const int v = m->ax_cfg[prec].variant;
    if (v >= 0 && v < ax_variant_count(m, prec)) return v;
    return default_variant(m, prec);
}

nb_status ax_local(nb_mesh *m, nb_prec prec, const void *u, void *w, double *pap_part,
                   int *nparts, cudaStream_t s)
{
    switch (prec) {
        case NB_FP64:
            return run_cc<double>(m, prec, variant_of(m, prec), false, m->G64, (const double *)u,
                                  (double *)w, nullptr, nullptr, nullptr, nullptr, pap_part,
                                  nparts, s);
        case NB_FP32:
            return run_cc<float>(m, prec, variant_of(m, prec), false, m->G32, (const float *)u,
                                 (float *)w, nullptr, nullptr, nullptr, nullptr, pap_part, nparts,
                                 s);
        case NB_TC_F16:
        case NB_TC_BF16:
            return ax_tc(m, prec, false, (const float *)u, (float *)w, nullptr, nullptr, nullptr,
                         nullptr, pap_part, nparts, s);
    }
    set_error("bad precision %d", (int)prec);
    return NB_ERR_ARG;
}

nb_status ax_cg_step(nb_mesh *m, nb_prec prec, const void *r, const void *dinv, void *p, void *w,
                     CgScalars *scal, double *pap_part, int *nparts, cudaStream_t s)
{
    switch (prec) {
        case NB_FP64:
            return run_cc<double>(m, prec, variant_of(m, prec), true, m->G64, nullptr,
                                  (double *)w, (const double *)r, (const double *)dinv,
                                  (double *)p, scal, pap_part, nparts, s);
        case NB_FP32:
            return run_cc<float>(m, prec, variant_of(m, prec), true, m->G32, nullptr, (float *)w,
                                 (const float *)r, (const float *)dinv, (float *)p, scal,
                                 pap_part, nparts, s);
        case NB_TC_F16:
        case NB_TC_BF16:
            return ax_tc(m, prec, true, nullptr, (float *)w, (const float *)r,
                         (const float *)dinv, (float *)p, scal, pap_part, nparts, s);
    }
    set_error("bad precision %d", (int)prec);
    return NB_ERR_ARG;
}

bool ax_dir_step_available(const nb_mesh *m) { return tma_ok(m, NB_FP32); }

// The fused step of flexible CG in FP32: p = z + beta p, w = A_L p, and the
// partials of p.w (the last block forms alpha = rtz / pap).
nb_status ax_dir_step(nb_mesh *m, const float *z, float *p, float *w, CgScalars *scal,
                      double *pap_part, int *nparts, cudaStream_t s)
{
    if (!ax_dir_step_available(m) || !(aligned16(z) && aligned16(p) && aligned16(w))) {
        set_error("flexible-CG step needs the bulk-copy operator (even n, aligned vectors)");
        return NB_ERR_ARG;
    }
    return ax_tma_f32(m->n, 2, m->ctx->sm_count, m->E, m->G32, nullptr, w, z, nullptr, p, scal,
                      pap_part, m->kerr, nparts, s);
}

}  // namespace nb
