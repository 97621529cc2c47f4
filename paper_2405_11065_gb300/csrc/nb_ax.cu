// Host glue of the operator: precision and variant dispatch.
//
// Variants of the CUDA-core operator (chosen per mesh and precision by
// nb_autotune, nb_set_ax_variant, or by the default below), numbered in this
// order among those available for the mesh's order:
//   k_ax_cc with the smaller / larger number of elements per block, every
//         load issued by the computing threads (always available);
//   k_ax_tma, element data streamed by bulk copies into a two-stage
//         shared-memory ring, one thread per (i,j) column (even n, when two
//         stages fit in shared memory);
//   k_ax_pen with two / one stages of geometric factors, pencil passes
//         (even n, when the stages and work arrays fit).
// The bulk-copy variants need every vector 16-byte aligned; with an
// unaligned vector the call falls back to the larger k_ax_cc group.
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
nb_status ax_pen_f32(int n, int mode, int stages, int sm_count, long long E, const float *G,
                     const float *u, float *w, const float *r, const float *dinv, float *p,
                     CgScalars *scal, double *part, int *err, int *grid, cudaStream_t s);
nb_status ax_pen_f64(int n, int mode, int stages, int sm_count, long long E, const double *G,
                     const double *u, double *w, const double *r, const double *dinv, double *p,
                     CgScalars *scal, double *part, int *err, int *grid, cudaStream_t s);
bool ax_pen_available_f32(int n, int stages);
bool ax_pen_available_f64(int n, int stages);
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

static bool pen_ok(const nb_mesh *m, nb_prec prec, int stages)
{
    if (prec == NB_FP32) return ax_pen_available_f32(m->n, stages);
    if (prec == NB_FP64) return ax_pen_available_f64(m->n, stages);
    return false;
}

enum AxKind { kCcSmall, kCcLarge, kTma, kPen2, kPen1 };

// The variants available for the mesh's order and the precision, in index order.
static int ax_kinds(const nb_mesh *m, nb_prec prec, AxKind out[5])
{
    if (prec != NB_FP64 && prec != NB_FP32) return 0;
    int c = 0;
    out[c++] = kCcSmall;
    out[c++] = kCcLarge;
    if (tma_ok(m, prec)) out[c++] = kTma;
    if (pen_ok(m, prec, 2)) out[c++] = kPen2;
    if (pen_ok(m, prec, 1)) out[c++] = kPen1;
    return c;
}

int ax_variant_count(const nb_mesh *m, nb_prec prec)
{
    AxKind k[5];
    const int c = ax_kinds(m, prec, k);
    return c > 0 ? c : 1;  // tensor-core kernel: one shape
}

// Default before any autotuning or explicit choice.  FP32: the pencil kernel
// with two stages where it fits, else with one, else the bulk-copy column
// kernel, else the larger element group.  FP64 (bound by the FP64 pipe): the
// bulk-copy column kernel, else the larger group, except at high order where
// two elements per block spill registers.
static AxKind default_kind(const nb_mesh *m, nb_prec prec)
{
    if (prec == NB_FP32) {
        if (pen_ok(m, prec, 2)) return kPen2;
        if (pen_ok(m, prec, 1)) return kPen1;
    }
    if (tma_ok(m, prec)) return kTma;
    if (prec == NB_FP64 && m->n >= 12) return kCcSmall;
    return kCcLarge;
}

static bool aligned16(const void *p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; }

static AxKind kind_of(const nb_mesh *m, nb_prec prec)
{
    AxKind k[5];
    const int c = ax_kinds(m, prec, k);
    const int v = m->ax_cfg[prec].variant;
    if (v >= 0 && v < c) return k[v];
    return default_kind(m, prec);
}

// Kernel name of variant v (NULL outside the range).
const char *ax_variant_name(const nb_mesh *m, nb_prec prec, int v)
{
    AxKind k[5];
    const int c = ax_kinds(m, prec, k);
    if (c == 0) return v == 0 ? "k_ax_tc (mma.sync tensor-core contractions)" : nullptr;
    if (v < 0 || v >= c) return nullptr;
    switch (k[v]) {
        case kCcSmall: return "k_ax_cc (smaller element group)";
        case kCcLarge: return "k_ax_cc (larger element group)";
        case kTma: return "k_ax_tma (column per thread, bulk-copy ring)";
        case kPen2: return "k_ax_pen (pencil passes, two bulk-copy stages)";
        case kPen1: return "k_ax_pen (pencil passes, one bulk-copy stage)";
    }
    return nullptr;
}

// Index of the variant in use for (mesh, prec) (the default when none is set).
int ax_variant_in_use(const nb_mesh *m, nb_prec prec)
{
    AxKind k[5];
    const int c = ax_kinds(m, prec, k);
    if (c == 0) return 0;
    const AxKind cur = kind_of(m, prec);
    for (int v = 0; v < c; ++v)
        if (k[v] == cur) return v;
    return 0;
}

// mode: 0 plain operator, 1 fused Jacobi CG step, 2 fused flexible-CG step
// (FP32 bulk-copy kinds only).
template <typename T>
static nb_status run_cc(nb_mesh *m, nb_prec prec, AxKind kind, int mode, const T *G, const T *u,
                        T *w, const T *r, const T *dinv, T *p, CgScalars *scal, double *part,
                        int *grid, cudaStream_t s)
{
    const bool bulk = kind == kTma || kind == kPen2 || kind == kPen1;
    if (bulk && !(aligned16(u) && aligned16(w) && aligned16(r) && aligned16(dinv) && aligned16(p)))
        kind = kCcLarge;  // the bulk copies need 16-byte aligned vectors
    constexpr bool f64 = sizeof(T) == 8;
    if (kind == kTma) {
        if (f64)
            return ax_tma_f64(m->n, mode, m->ctx->sm_count, m->E, (const double *)G,
                              (const double *)u, (double *)w, (const double *)r,
                              (const double *)dinv, (double *)p, scal, part, m->kerr, grid, s);
        return ax_tma_f32(m->n, mode, m->ctx->sm_count, m->E, (const float *)G, (const float *)u,
                          (float *)w, (const float *)r, (const float *)dinv, (float *)p, scal,
                          part, m->kerr, grid, s);
    }
    if (kind == kPen2 || kind == kPen1) {
        const int stages = kind == kPen2 ? 2 : 1;
        if (f64)
            return ax_pen_f64(m->n, mode, stages, m->ctx->sm_count, m->E, (const double *)G,
                              (const double *)u, (double *)w, (const double *)r,
                              (const double *)dinv, (double *)p, scal, part, m->kerr, grid, s);
        return ax_pen_f32(m->n, mode, stages, m->ctx->sm_count, m->E, (const float *)G,
                          (const float *)u, (float *)w, (const float *)r, (const float *)dinv,
                          (float *)p, scal, part, m->kerr, grid, s);
    }
    if (mode == 2) {
        set_error("flexible-CG step needs a bulk-copy operator variant");
        return NB_ERR_ARG;
    }
    const int v = kind == kCcSmall ? 0 : 1;
    if (f64)
        return ax_cc_f64(m->n, v, mode != 0, m->ctx->sm_count, m->E, (const double *)G,
                         (const double *)u, (double *)w, (const double *)r, (const double *)dinv,
                         (double *)p, scal, part, grid, s);
    return ax_cc_f32(m->n, v, mode != 0, m->ctx->sm_count, m->E, (const float *)G,
                     (const float *)u, (float *)w, (const float *)r, (const float *)dinv,
                     (float *)p, scal, part, grid, s);
}

nb_status ax_local(nb_mesh *m, nb_prec prec, const void *u, void *w, double *pap_part,
                   int *nparts, cudaStream_t s)
{
    switch (prec) {
        case NB_FP64:
            return run_cc<double>(m, prec, kind_of(m, prec), 0, m->G64, (const double *)u,
                                  (double *)w, nullptr, nullptr, nullptr, nullptr, pap_part,
                                  nparts, s);
        case NB_FP32:
            return run_cc<float>(m, prec, kind_of(m, prec), 0, m->G32, (const float *)u,
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
            return run_cc<double>(m, prec, kind_of(m, prec), 1, m->G64, nullptr,
                                  (double *)w, (const double *)r, (const double *)dinv,
                                  (double *)p, scal, pap_part, nparts, s);
        case NB_FP32:
            return run_cc<float>(m, prec, kind_of(m, prec), 1, m->G32, nullptr, (float *)w,
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

// The fused FP32 Jacobi CG step with the previous direction read from p_prev
// and the new one written to p (distinct buffers; the pencil kernel only).
bool ax_cg_step_from_available(const nb_mesh *m)
{
    const AxKind k = kind_of(m, NB_FP32);
    return (k == kPen2 || k == kPen1) && pen_ok(m, NB_FP32, k == kPen2 ? 2 : 1);
}

nb_status ax_cg_step_from(nb_mesh *m, const float *r, const float *dinv, const float *p_prev,
                          float *p, float *w, CgScalars *scal, double *pap_part, int *nparts,
                          cudaStream_t s)
{
    if (!ax_cg_step_from_available(m) || p_prev == nullptr || p_prev == p ||
        !(aligned16(r) && aligned16(dinv) && aligned16(p_prev) && aligned16(p) && aligned16(w))) {
        set_error("CG step from a second direction buffer needs the pencil operator");
        return NB_ERR_ARG;
    }
    const AxKind kind = kind_of(m, NB_FP32);
    return ax_pen_f32(m->n, 1, kind == kPen2 ? 2 : 1, m->ctx->sm_count, m->E, m->G32, p_prev, w,
                      r, dinv, p, scal, pap_part, m->kerr, nparts, s);
}

bool ax_dir_step_available(const nb_mesh *m)
{
    return tma_ok(m, NB_FP32) || pen_ok(m, NB_FP32, 2) || pen_ok(m, NB_FP32, 1);
}

// The fused step of flexible CG in FP32: p = z + beta p, w = A_L p, and the
// partials of p.w (the last block forms alpha = rtz / pap).  Runs the chosen
// bulk-copy variant, or the best available one if a k_ax_cc group is chosen.
nb_status ax_dir_step(nb_mesh *m, const float *z, float *p, float *w, CgScalars *scal,
                      double *pap_part, int *nparts, cudaStream_t s)
{
    if (!ax_dir_step_available(m) || !(aligned16(z) && aligned16(p) && aligned16(w))) {
        set_error("flexible-CG step needs a bulk-copy operator (even n, aligned vectors)");
        return NB_ERR_ARG;
    }
    AxKind kind = kind_of(m, NB_FP32);
    if (kind != kTma && kind != kPen2 && kind != kPen1)
        kind = pen_ok(m, NB_FP32, 2) ? kPen2 : pen_ok(m, NB_FP32, 1) ? kPen1 : kTma;
    return run_cc<float>(m, NB_FP32, kind, 2, m->G32, nullptr, w, z, nullptr, p, scal, pap_part,
                         nparts, s);
}

}  // namespace nb
