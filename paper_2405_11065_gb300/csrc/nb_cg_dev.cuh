// Device-side scalar steps of the CG iteration, run by the last block of the
// kernel that produced the partial sums ("last block done" pattern: each
// block publishes its partial, then takes a ticket; the block holding the
// final ticket sums all partials in index order, so the result does not
// depend on which block finished last).
#pragma once

#include "nb_reduce.cuh"

namespace nb {

// True in every thread of the block that arrived last; all partials written
// before the calls of the other blocks are then visible.  Resets the ticket.
__device__ __forceinline__ bool last_block(unsigned int *ticket)
{
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int t = atomicAdd(ticket, 1u);
        is_last = (t == gridDim.x - 1);
        if (is_last) *ticket = 0u;  // every block has taken its ticket
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// pap = sum of the operator's partials, alpha = rtz / pap (breakdown if
// pap <= 0 or alpha is not finite).  Called by the whole last block.
__device__ __forceinline__ void cg_finish_pap(CgScalars *sc, const double *part, int cnt,
                                              double *sred)
{
    const double pap = sum_partials(part, cnt, sred);
    if (threadIdx.x == 0) {
        sc->pap = pap;
        const double alpha = sc->rtz / pap;
        if (!(pap > 0.0) || !isfinite(alpha)) {
            sc->alpha = 0.0;
            sc->done = 1;
            sc->status = NB_BREAKDOWN;
        } else {
            sc->alpha = alpha;
        }
    }
}

// rtz and rtr of the new residual, beta, iteration count, history and the
// stopping tests (tolerance, iteration limit, non-finite values).
__device__ __forceinline__ void cg_finish_iter(CgScalars *sc, const double *part, int cnt,
                                               double *sred)
{
    const double rtz = sum_partials(part, cnt, sred);
    const double rtr = sum_partials(part + cnt, cnt, sred);
    if (threadIdx.x == 0) {
        sc->rtz_old = sc->rtz;
        sc->rtz = rtz;
        sc->rtr = rtr;
        sc->beta = rtz / sc->rtz_old;
        const int it = sc->iter + 1;
        sc->iter = it;
        const double bn = sc->bnorm2 > 0.0 ? sc->bnorm2 : 1.0;
        const double rel = sqrt(rtr / bn);
        sc->relres = rel;
        if (sc->hist && it <= sc->hist_cap) sc->hist[it - 1] = rel;
        if (!isfinite(rel) || !isfinite(sc->beta)) {
            sc->done = 1;
            sc->status = NB_BREAKDOWN;
        } else if (rel < sc->tol) {
            sc->done = 1;
        } else if (it >= sc->maxit) {
            sc->done = 1;
            sc->status = NB_NOT_CONVERGED;
        }
    }
}

}  // namespace nb
