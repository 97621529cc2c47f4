// Learned per-element preconditioner and flexible CG.
#include "nb_internal.h"

namespace nb {

void learned_free(nb_mesh *m) { m->learned = nullptr; }

nb_status fcg_learned(nb_mesh *m, nb_prec prec, Workspace &ws, const nb_opts *o, cudaStream_t s)
{
    (void)m; (void)prec; (void)ws; (void)o; (void)s;
    set_error("learned preconditioner not available in this build");
    return NB_ERR_STATE;
}

}  // namespace nb
