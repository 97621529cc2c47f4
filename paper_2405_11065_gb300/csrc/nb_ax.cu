// Host glue of the operator: precision and variant dispatch.
#include "nb_internal.h"

namespace nb {

nb_status upload_D_f32(int n, const double *D);
nb_status upload_D_f64(int n, const double *D);
nb_status ax_cc_f32(int n, int mchoice, bool pupd, int sm_count, long long E, const float *G,
                    const float *u, float *w, const float *r, const float *dinv, float *p,
                    const CgScalars *scal, double *part, int *grid, cudaStream_t s);
nb_status ax_cc_f64(int n, int mchoice, bool pupd, int sm_count, long long E, const double *G,
                    const double *u, double *w, const double *r, const double *dinv, double *p,
                    const CgScalars *scal, double *part, int *grid, cudaStream_t s);
nb_status ax_tc(nb_mesh *m, nb_prec prec, bool pupd, const float *u, float *w, const float *r,
                const float *dinv, float *p, const CgScalars *scal, double *part, int *grid,
                cudaStream_t s);
nb_status upload_D_tc(int n, const double *D);

nb_status upload_deriv_tables(int n, const double *D64)
{
    NB_TRY(upload_D_f32(n, D64));
    NB_TRY(upload_D_f64(n, D64));
    NB_TRY(upload_D_tc(n, D64));
    return NB_OK;
}

int ax_variant_count(const nb_mesh *m, nb_prec prec)
{
    (void)m;
    return (prec == NB_FP64 || prec == NB_FP32) ? 2 : 1;  // tensor-core kernel: one shape
}

// Default before any autotuning: the larger element group, except FP64 at
// high order where two elements per block spill registers.
static int default_mchoice(const nb_mesh *m, nb_prec prec)
{
    if (prec == NB_FP64 && m->n >= 12) return 0;
    return 1;
}

nb_status ax_local(nb_mesh *m, nb_prec prec, const void *u, void *w, double *pap_part,
                   int *nparts, cudaStream_t s)
{
    const int choice = m->ax_cfg[prec].variant >= 0 ? m->ax_cfg[prec].variant : default_mchoice(m, prec);
    switch (prec) {
        case NB_FP64:
            return ax_cc_f64(m->n, choice, false, m->ctx->sm_count, m->E, m->G64,
                             (const double *)u, (double *)w, nullptr, nullptr, nullptr, nullptr,
                             pap_part, nparts, s);
        case NB_FP32:
            return ax_cc_f32(m->n, choice, false, m->ctx->sm_count, m->E, m->G32,
                             (const float *)u, (float *)w, nullptr, nullptr, nullptr, nullptr,
                             pap_part, nparts, s);
        case NB_TC_F16:
        case NB_TC_BF16:
            return ax_tc(m, prec, false, (const float *)u, (float *)w, nullptr, nullptr, nullptr,
                         nullptr, pap_part, nparts, s);
    }
    set_error("bad precision %d", (int)prec);
    return NB_ERR_ARG;
}

nb_status ax_cg_step(nb_mesh *m, nb_prec prec, const void *r, const void *dinv, void *p, void *w,
                     const CgScalars *scal, double *pap_part, int *nparts, cudaStream_t s)
{
    const int choice = m->ax_cfg[prec].variant >= 0 ? m->ax_cfg[prec].variant : default_mchoice(m, prec);
    switch (prec) {
        case NB_FP64:
            return ax_cc_f64(m->n, choice, true, m->ctx->sm_count, m->E, m->G64, nullptr,
                             (double *)w, (const double *)r, (const double *)dinv, (double *)p,
                             scal, pap_part, nparts, s);
        case NB_FP32:
            return ax_cc_f32(m->n, choice, true, m->ctx->sm_count, m->E, m->G32, nullptr,
                             (float *)w, (const float *)r, (const float *)dinv, (float *)p, scal,
                             pap_part, nparts, s);
        case NB_TC_F16:
        case NB_TC_BF16:
            return ax_tc(m, prec, true, nullptr, (float *)w, (const float *)r,
                         (const float *)dinv, (float *)p, scal, pap_part, nparts, s);
    }
    set_error("bad precision %d", (int)prec);
    return NB_ERR_ARG;
}

}  // namespace nb
