// CUDA-core operator instantiations for double (see nb_ax_impl.cuh).
#include "nb_ax_impl.cuh"
#include "nb_ax_pen.cuh"
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

// Even-odd halves of D and D^T for even n (index n / 2), h = n / 2, N = n - 1:
// c_EO[n/2][0][i][l] = (D[i][l] + D[i][N-l]) / 2, [1] = (D[i][l] - D[i][N-l]) / 2,
// [2] and [3] the same for D^T (D^T[i][l] = D[l][i]); i, l < h.
static __constant__ double c_EO[kMaxn / 2 + 1][4][kMaxn / 2][kMaxn / 2];

template <>
__device__ __forceinline__ double eotab<double>(int n, int which, int i, int l)
{
    return c_EO[n / 2][which][i][l];
}

nb_status upload_D_f64(int n, const double *D)
{
    double tab[kMaxn * kMaxn] = {};
    for (int i = 0; i < n; ++i)
        for (int l = 0; l < n; ++l) tab[i * kMaxn + l] = (double)D[i * n + l];
    NB_CUDA(cudaMemcpyToSymbol(c_D, tab, sizeof(tab), sizeof(tab) * n, cudaMemcpyHostToDevice));
    if (n % 2 == 0) {
        constexpr int H = kMaxn / 2;
        double eo[4][H][H] = {};
        const int h = n / 2, N = n - 1;
        for (int i = 0; i < h; ++i)
            for (int l = 0; l < h; ++l) {
                eo[0][i][l] = (double)(0.5 * (D[i * n + l] + D[i * n + (N - l)]));
                eo[1][i][l] = (double)(0.5 * (D[i * n + l] - D[i * n + (N - l)]));
                eo[2][i][l] = (double)(0.5 * (D[l * n + i] + D[(N - l) * n + i]));
                eo[3][i][l] = (double)(0.5 * (D[l * n + i] - D[(N - l) * n + i]));
            }
        NB_CUDA(cudaMemcpyToSymbol(c_EO, eo, sizeof(eo), sizeof(eo) * (n / 2),
                                   cudaMemcpyHostToDevice));
    }
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

nb_status ax_pen_f64(int n, int mode, int stages, int sm_count, long long E, const double *G,
                     const double *u, double *w, const double *r, const double *dinv, double *p,
                     CgScalars *scal, double *part, int *err, int *grid, cudaStream_t s)
{
    return dispatch_ax_pen<double>(n, mode, stages, sm_count, E, G, u, w, r, dinv, p, scal, part,
                                err, grid, s);
}

bool ax_pen_available_f64(int n, int stages) { return pen_fits<double>(n, stages); }

nb_status bax_f64(int n, int mchoice, bool pupd, int sm_count, long long E, long long e_first,
                  const int32_t *list, const int *cnt, const double *G, const double *u, double *w,
                  const double *r, const double *dinv, double *p, const int32_t *elem_prob, const BScal *bs,
                  double *part_e, cudaStream_t s)
{
    return dispatch_bax<double>(n, mchoice, pupd, sm_count, E, e_first, list, cnt, G, u, w, r, dinv,
                             p, elem_prob, bs, part_e, s);
}

}  // namespace nb
