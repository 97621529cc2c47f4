// CUDA-core operator instantiations for float (see nb_ax_impl.cuh).
#include "nb_ax_impl.cuh"
#include "nb_ax_tma.cuh"
#include "nb_batch_ax.cuh"

namespace nb {

// Derivative matrices of every order: c_D[n][i][l] = D[i][l] for n = N+1.
static __constant__ float c_D[kMaxn + 1][kMaxn][kMaxn];

template <>
__device__ __forceinline__ float dtab<float>(int n, int i, int l)
{
    return c_D[n][i][l];
}

nb_status upload_D_f32(int n, const double *D)
{
    float tab[kMaxn * kMaxn] = {};
    for (int i = 0; i < n; ++i)
        for (int l = 0; l < n; ++l) tab[i * kMaxn + l] = (float)D[i * n + l];
    NB_CUDA(cudaMemcpyToSymbol(c_D, tab, sizeof(tab), sizeof(tab) * n, cudaMemcpyHostToDevice));
    return NB_OK;
}

nb_status ax_cc_f32(int n, int mchoice, bool pupd, int sm_count, long long E, const float *G,
                      const float *u, float *w, const float *r, const float *dinv, float *p,
                      CgScalars *scal, double *part, int *grid, cudaStream_t s)
{
    return dispatch_ax_cc<float>(n, mchoice, pupd, sm_count, E, G, u, w, r, dinv, p, scal, part,
                                grid, s);
}

nb_status ax_tma_f32(int n, int mode, int sm_count, long long E, const float *G,
                      const float *u, float *w, const float *r, const float *dinv, float *p,
                      CgScalars *scal, double *part, int *err, int *grid, cudaStream_t s)
{
    return dispatch_ax_tma<float>(n, mode, sm_count, E, G, u, w, r, dinv, p, scal, part, err, grid,
                               s);
}

bool ax_tma_available_f32(int n, bool pupd) { return tma_fits<float>(n, pupd); }

nb_status bax_f32(int n, int mchoice, bool pupd, int sm_count, long long E, long long e_first,
                  const int32_t *list, const int *cnt, const float *G, const float *u, float *w,
                  const float *r, const float *dinv, float *p, const int32_t *elem_prob, const BScal *bs,
                  double *part_e, cudaStream_t s)
{
    return dispatch_bax<float>(n, mchoice, pupd, sm_count, E, e_first, list, cnt, G, u, w, r, dinv,
                             p, elem_prob, bs, part_e, s);
}

nb_status bax_tma_f32(int n, int sm_count, long long E, long long e_first, const int32_t *list,
                      const int *cnt, const float *G, float *w, const float *r, const float *dinv,
                      float *p, const int32_t *elem_prob, BScal *bs, double *part_e, int *err,
                      cudaStream_t s)
{
    return dispatch_bax_tma<float>(n, sm_count, E, e_first, list, cnt, G, w, r, dinv, p,
                                   elem_prob, bs, part_e, err, s);
}

bool bax_tma_available_f32(int n) { return bax_tma_fits<float>(n); }

}  // namespace nb
