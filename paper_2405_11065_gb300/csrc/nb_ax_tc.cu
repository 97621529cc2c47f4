// Tensor-core operator (filled in below by the tensor-core kernels).
#include "nb_internal.h"

namespace nb {

nb_status upload_D_tc(int n, const double *D)
{
    (void)n;
    (void)D;
    return NB_OK;
}

nb_status ax_tc(nb_mesh *m, nb_prec prec, bool pupd, const float *u, float *w, const float *r,
                const float *dinv, float *p, const CgScalars *scal, double *part, int *grid,
                cudaStream_t s)
{
    (void)m; (void)prec; (void)pupd; (void)u; (void)w; (void)r; (void)dinv; (void)p;
    (void)scal; (void)part; (void)grid; (void)s;
    set_error("tensor-core operator not available in this build");
    return NB_ERR_ARG;
}

}  // namespace nb
