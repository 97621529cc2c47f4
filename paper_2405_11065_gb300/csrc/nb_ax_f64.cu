// CUDA-core operator instantiations for double (see nb_ax_impl.cuh).
#include "nb_ax_impl.cuh"
#include "nb_ax_tma.cuh"
#include "nb_batch_ax.cuh"

namespace nb {

// Derivative matrices of every order: c_D[n][i][l] = D[i][l] for n = N+1.
static __constant__ double c_D[kMaxn + 1][kMaxn][kMaxn];

template <>
__device__ __forceinline__ double dtab<double>(int n, int i, int l)
{
    return c_D[n][i][l];
}

nb_status upload_D_f64(int n, const double *D)
{
    double tab[kMaxn * kMaxn] = {};
    for (int i = 0; i < n; ++i)
        for (int l = 0; l < n; ++l) tab[i * kMaxn + l] = (double)D[i * n + l];
    NB_CUDA(cudaMemcpyToSymbol(c_D, tab, sizeof(tab), sizeof(tab) * n, cudaMemcpyHostToDevice));
    return NB_OK;
}

nb_status ax_cc_f64(int n, int mchoice, bool pupd, int sm_count, long long E, const double *G,
                      const double *u, double *w, const double *r, const double *dinv, double *p,
                      CgScalars *scal, double *part, int *grid, cudaStream_t s)
{
    return dispatch_ax_cc<double>(n, mchoice, pupd, sm_count, E, G, u, w, r, dinv, p, scal, part,
                                grid, s);
}

nb_status ax_tma_f64(int n, int mode, int sm_count, long long E, const double *G,
                      const double *u, double *w, const double *r, const double *dinv, double *p,
                      CgScalars *scal, double *part, int *err, int *grid, cudaStream_t s)
{
    return dispatch_ax_tma<double>(n, mode, sm_count, E, G, u, w, r, dinv, p, scal, part, err, grid,
                               s);
}

bool ax_tma_available_f64(int n, bool pupd) { return tma_fits<double>(n, pupd); }

nb_status bax_f64(int n, int mchoice, bool pupd, int sm_count, long long E, long long e_first,
                  const int32_t *list, const int *cnt, const double *G, const double *u, double *w,
                  const double *r, const double *dinv, double *p, const int32_t *elem_prob, const BScal *bs,
                  double *part_e, cudaStream_t s)
{
    return dispatch_bax<double>(n, mchoice, pupd, sm_count, E, e_first, list, cnt, G, u, w, r, dinv,
                             p, elem_prob, bs, part_e, s);
}

}  // namespace nb
