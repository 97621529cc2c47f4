// Device-side scalar steps of the CG iteration, run by the last block of the
// kernel that produced the partial sums ("last block done" pattern: each
// block publishes its partial, then takes a ticket; the block holding the
// final ticket sums all partials in index order, so the result does not
// depend on which block finished last).
#pragma once

#include "nb_reduce.cuh"

namespace nb {

// Programmatic dependent launch (see launch_pdl): wait until the previous
// kernel of the stream has completed and its writes are visible (returns at
// once for a launch without the attribute) ...
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

// ... and let the next kernel start its prologue once every block of this
// one has called this (after its main work; without the call the next kernel
// starts as this one's blocks exit).  The loop kernels call it where the
// solve's scalars ask for it (CgScalars::pdl_early).
__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// True in every thread of the block that arrived last; the partials that
// thread 0 of each block wrote before its call are then visible to warp 0.
// Resets the ticket.  Only thread 0 fences: a fence in every thread would wait for all
// of the block's outstanding stores of the kernel's outputs, which the last
// block does not read.
__device__ __forceinline__ bool last_block(unsigned int *ticket)
{
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(ticket, 1u);
        is_last = (t == gridDim.x - 1);
        if (is_last) *ticket = 0u;  // every block has taken its ticket
    }
    __syncthreads();
    // the partials are read by warp 0 (sum_partials up to 2048 of them; it
    // fences every thread itself beyond that)
    if (is_last && threadIdx.x < 32) __threadfence();
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
    double rtz, rtr;
    sum_partials2(part, part + cnt, cnt, sred, rtz, rtr);
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

template <typename T>
struct Pair2;
template <>
struct Pair2<float> {
    using type = float2;
};
template <>
struct Pair2<double> {
    using type = double2;
};

// Direct-stiffness sum of w at two nodes (i0, j, k), (i0 + 1, j, k) of element
// (ex, ey, ez) of the box mesh, n even (N odd), l the first node's local
// index.  The copies of a node are its mirror nodes in the neighbouring
// elements: i = 0 of element ex is i = N of ex - 1 (local offset -sx,
// sx = n^3 - N), i = N is i = 0 of ex + 1, and likewise along y (sy =
// nx n^3 - N n) and z (sz = nx ny n^3 - N n^2).  A node has 1, 2, 4 or 8
// copies; they are summed in ascending local index (slot order (tz, ty, tx)
// with tx = 0 the lower x element), the order of the row-wise summation
// kernel, so the sums are bit-identical to it.  Only the first node of a pair
// can be on a lower x face and only the second on an upper one; the y / z
// copies of both nodes are one vector load each.  No mask applied.
// The sum of gs_sum_pair with its copy flags given: lxa / hxb the first
// node on a lower x face / the second on an upper one (with a neighbour
// there), ly, hy, lz, hz the pair on a lower / upper y or z face.
template <typename T, typename I>
__device__ __forceinline__ void gs_sum_pair_flags(const T *__restrict__ w, I l, bool lxa, bool hxb,
                                                  int ly, int hy, int lz, int hz, I sx, I sy, I sz,
                                                  T &wa, T &wb)
{
    using V = typename Pair2<T>::type;
    const I l0 = l - ly * sy - lz * sz;
    T va[2][2][2], vb[2][2][2];
#pragma unroll
    for (int tz = 0; tz < 2; ++tz)
#pragma unroll
        for (int ty = 0; ty < 2; ++ty) {
            const bool ok = tz <= lz + hz && ty <= ly + hy;
            const I o = l0 + ty * sy + tz * sz;
            const V own = ok ? *reinterpret_cast<const V *>(w + o) : V{T(0), T(0)};
            const T pa = ok && lxa ? w[o - sx] : T(0);
            const T pb = ok && hxb ? w[o + 1 + sx] : T(0);
            va[tz][ty][0] = lxa ? pa : own.x;
            va[tz][ty][1] = lxa ? own.x : T(0);
            vb[tz][ty][0] = own.y;
            vb[tz][ty][1] = pb;
        }
    wa = T(0);
    wb = T(0);
#pragma unroll
    for (int tz = 0; tz < 2; ++tz)
#pragma unroll
        for (int ty = 0; ty < 2; ++ty)
#pragma unroll
            for (int tx = 0; tx < 2; ++tx) {
                wa += va[tz][ty][tx];
                wb += vb[tz][ty][tx];
            }
}

template <typename T, int n, typename I>
__device__ __forceinline__ void gs_sum_pair(const T *__restrict__ w, I l, int i0, int j,
                                            int k, int ex, int ey, int ez, int nx, int ny, int nz,
                                            I sx, I sy, I sz, T &wa, T &wb)
{
    constexpr int N = n - 1;
    const bool lxa = i0 == 0 && ex > 0, hxb = i0 + 1 == N && ex < nx - 1;
    const int ly = j == 0 && ey > 0, hy = j == N && ey < ny - 1;
    const int lz = k == 0 && ez > 0, hz = k == N && ez < nz - 1;
    gs_sum_pair_flags<T, I>(w, l, lxa, hxb, ly, hy, lz, hz, sx, sy, sz, wa, wb);
}

}  // namespace nb
