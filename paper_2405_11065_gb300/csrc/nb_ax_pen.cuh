// The operator as pencil passes over each element, geometric factors streamed
// by the bulk-copy engine (cp.async.bulk, TMA) into a shared-memory ring.
//
// Every contraction of ax is a 1D product along one direction of the
// element: ur = D u along i, us along j, ut along k, and their transposes.
// Here a thread owns, in turn, one line ("pencil") of the element along each
// direction and does that direction's products in registers, with the
// derivative matrix D as compile-time constant-bank operands:
//   1. k-pencil (thread <-> (i, j)): form u (the fused CG step's p) for its
//      column from r, dinv and p loaded during passes 3-5 of the previous
//      element, keep it in registers and store it in shared memory;
//   2. i-pencil (thread <-> (j, k)): read the row of u, ur = D u along i,
//      store the row of ur; j-pencil (thread <-> (i, k)): read the column,
//      us = D u along j, store it;
//   3. k-pencil: ut = D u along k from the thread's own column, then wr, ws,
//      wt = G (ur, us, ut) per node (G from the ring), wr and ws stored in
//      place of ur and us, the transpose along k of wt accumulated in
//      registers;
//   4. i-pencil: the transpose along i of the row of wr, in place;
//      j-pencil: the transpose along j of the column of ws, in place;
//   5. k-pencil: w = (k part) + (i part) + (j part), written to HBM, and the
//      partial of p.w.
// Every 1D product uses the even-odd decomposition of D (deriv_eo): half the
// multiply-adds of the plain n x n product.
// That is four block barriers and about 19 shared-memory accesses per node
// (of which the 6 geometric factors), against one barrier per layer and
// about 33 accesses per node when one thread owns a column and reads the other
// two directions from shared memory at every layer (k_ax_tma).
//
// Work arrays are [k][j][i] with a layer stride KS >= n^2 congruent to n
// modulo 32: the k-pencil accesses of a warp (consecutive (i, j)) and the
// j-pencil accesses (consecutive (i, k)) then hit 32 distinct banks.  Rows
// (i-pencils) are read and written as 8-byte vectors.
//
// The ring holds S elements' geometric factors (S = 2: the copy of element
// t + 2 is issued as soon as element t's factors are consumed, after pass
// 3; S = 1 for the orders where two stages do not leave room for enough
// blocks).  The copies carry an L2 evict-first policy: the factors are read
// once per operator application, while the solver's vectors are re-read every
// iteration and stay in L2 instead.
//
// Forms (MODE) as k_ax_tma: 0 the plain operator w = A_L u; 1 the fused
// Jacobi CG step p = |dinv| r + beta p, w = A_L p, partials of p.w and
// alpha in the last block; 2 the fused flexible-CG step p = z + beta p.  In
// forms 1 and 2 the previous direction is read from u where u is given (the
// solver then alternates two direction buffers) and from p itself otherwise.
// Every wait on an mbarrier is bounded (one second); a block that times out
// sets *err, drains its own copies and exits.
#pragma once

#include "nb_ax_tma.cuh"

namespace nb {

// Layer stride of the work arrays for n points per direction.
constexpr int pen_ks(int n)
{
    int ks = n * n;
    while ((ks - n) % 32 != 0 || ks % 2 != 0) ++ks;
    return ks;
}

constexpr size_t pen_smem_bytes(size_t elt, int n, int S)
{
    return elt * ((size_t)S * 6 * n * n * n + 3 * (size_t)n * pen_ks(n));
}

template <typename T, int n, int S>
constexpr size_t ax_pen_smem()
{
    return pen_smem_bytes(sizeof(T), n, S);
}

// Resident blocks per SM the launch bound reserves registers for: what
// shared memory and the thread count admit, but never below 96 registers a
// thread (128 for FP64) so the pencils stay in registers.
template <typename T, int n, int S>
constexpr int pen_min_blocks()
{
    const int threads = tma_threads<n>();
    const int by_smem = (int)((228 * 1024) / (ax_pen_smem<T, n, S>() + 1024));
    const int by_threads = 2048 / threads;
    const int by_regs = 65536 / (threads * (sizeof(T) == 4 ? 96 : 128));
    int b = by_smem < by_threads ? by_smem : by_threads;
    b = b < by_regs ? b : by_regs;
    return b < 1 ? 1 : b;
}

template <typename T, int n, int MODE, int S>
__global__ void __launch_bounds__(tma_threads<n>(), (pen_min_blocks<T, n, S>()))
k_ax_pen(long long E, const T *__restrict__ G, const T *__restrict__ uin, T *__restrict__ w,
         const T *__restrict__ r, const T *__restrict__ dinv, T *__restrict__ p,
         CgScalars *__restrict__ scal, double *__restrict__ part, int *__restrict__ err)
{
    constexpr bool PUPD = MODE != 0;
    constexpr int n2 = n * n, n3 = n2 * n, KS = pen_ks(n), GST = 6 * n3;
    using V2 = typename Vec2<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *stage = reinterpret_cast<T *>(smem_raw);  // [S][6][n3] geometric factors
    T *sP = stage + S * GST;                      // [n][KS] the element's u (p)
    T *sA = sP + n * KS;                          // ur -> wr -> i-direction part of w
    T *sB = sA + n * KS;                          // us -> ws -> j-direction part of w
    __shared__ __align__(8) uint64_t bar[S];
    __shared__ double sred[32];

    const int tid = threadIdx.x;
    const bool act = tid < n2;
    // the same split serves the three pencil roles: k-pencil (i, j) =
    // (q, rr), j-pencil (i, k) = (q, rr), i-pencil (j, k) = (q, rr)
    const int q = act ? tid % n : 0, rr = act ? tid / n : 0;
    const int kcol = rr * n + q;       // k-pencil: node (q, rr, k) at k * KS + kcol
    const int jcol = rr * KS + q;      // j-pencil: node (q, j, rr) at jcol + j * n
    const int irow = rr * KS + q * n;  // i-pencil: node (i, q, rr) at irow + i
    const long long mine = E > blockIdx.x ? (E - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        mbar_init_fence();
    }
    __syncthreads();

    auto issue = [&](long long t) {  // element number t of this block into stage t % S
        const long long e = blockIdx.x + t * gridDim.x;
        const int s = (int)(t % S);
        const uint32_t bytes = (uint32_t)(GST * sizeof(T));
        mbar_expect_tx(&bar[s], bytes);
        bulk_g2s_hint(stage + s * GST, G + (size_t)e * GST, bytes, &bar[s],
                      l2_evict_first_policy());
    };
    if (tid == 0)
        for (long long t = 0; t < S && t < mine; ++t) issue(t);
    // the geometric factors are constant: their first copies go out before
    // the wait for the previous kernel (programmatic dependent launch)
    pdl_wait();
    __shared__ int sdone;
    if (tid == 0) sdone = PUPD ? scal->done : 0;  // one reading for the whole block
    __syncthreads();
    if (sdone) {  // the solve has stopped: leave p and w untouched
        if (tid == 0)
            for (long long t = 0; t < S && t < mine; ++t) mbar_wait_bounded(&bar[t], 0);
        return;
    }
    const T beta = PUPD ? (T)scal->beta : T(0);

    // the thread's k-pencil of the element's inputs, one element ahead
    const T *pin = PUPD && uin != nullptr ? uin : p;  // the previous direction
    T nr[n], nd[n], np[n];
    auto fetch = [&](long long t) {
        const size_t b = (size_t)(blockIdx.x + t * gridDim.x) * n3 + tid;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            if (PUPD) {
                nr[k] = r[b + k * n2];
                nd[k] = MODE == 1 ? dinv[b + k * n2] : T(1);
                np[k] = pin[b + k * n2];
            } else {
                nr[k] = uin[b + k * n2];
            }
        }
    };
    if (act && mine > 0) fetch(0);

    double acc = 0.0;
    long long t = 0;
    for (; t < mine; ++t) {
        const long long e = blockIdx.x + t * gridDim.x;
        const size_t gb = (size_t)e * n3 + tid;
        T u[n], row[n], o[n], wk[n];
        // pass 1: k-pencil
        if (act) {
#pragma unroll
            for (int k = 0; k < n; ++k) {
                if (MODE == 1) u[k] = fabs(nd[k]) * nr[k] + beta * np[k];
                else if (MODE == 2) u[k] = nr[k] + beta * np[k];
                else u[k] = nr[k];
            }
#pragma unroll
            for (int k = 0; k < n; ++k) {
                sP[k * KS + kcol] = u[k];
                if (PUPD) p[gb + k * n2] = u[k];
            }
        }
        __syncthreads();
        if (act) {
            // pass 2, i-pencil: ur(i) = sum_l D[i][l] u(l)
            const V2 *src = reinterpret_cast<const V2 *>(sP + irow);
#pragma unroll
            for (int l = 0; l < n; l += 2) {
                const V2 v = src[l / 2];
                row[l] = v.x;
                row[l + 1] = v.y;
            }
            deriv_eo<T, n, false>(row, o);
            V2 *dst = reinterpret_cast<V2 *>(sA + irow);
#pragma unroll
            for (int m = 0; m < n; m += 2) dst[m / 2] = V2{o[m], o[m + 1]};
            // j-pencil: us(j) = sum_l D[j][l] u(l)
#pragma unroll
            for (int l = 0; l < n; ++l) row[l] = sP[jcol + l * n];
            deriv_eo<T, n, false>(row, o);
#pragma unroll
            for (int m = 0; m < n; ++m) sB[jcol + m * n] = o[m];
        }
        const bool ok = mbar_wait_bounded(&bar[t % S], (uint32_t)((t / S) & 1));
        if (__syncthreads_or(!ok)) break;
        if (act) {
            // the next element's inputs, loading through passes 3-5
            if (t + 1 < mine) fetch(t + 1);
            // pass 3, k-pencil: the geometric factors, the transpose along k
            const T *Gs = stage + (t % S) * GST + tid;
            deriv_eo<T, n, false>(u, row);  // ut = D u along k, from the own column
#pragma unroll
            for (int k = 0; k < n; ++k) {
                const int o3 = k * KS + kcol;
                const T a = sA[o3], b = sB[o3], c = row[k];
                const T g0 = Gs[0 * n3 + k * n2], g1 = Gs[1 * n3 + k * n2];
                const T g2 = Gs[2 * n3 + k * n2], g3 = Gs[3 * n3 + k * n2];
                const T g4 = Gs[4 * n3 + k * n2], g5 = Gs[5 * n3 + k * n2];
                sA[o3] = g0 * a + g1 * b + g2 * c;
                sB[o3] = g1 * a + g3 * b + g4 * c;
                o[k] = g2 * a + g4 * b + g5 * c;  // wt
            }
            deriv_eo<T, n, true>(o, wk);  // the k part of w: D^T wt along k
        }
        __syncthreads();  // stage t % S consumed: refill it
        if (tid == 0 && t + S < mine) issue(t + S);
        if (act) {
            // pass 4, i-pencil: sum_l D[l][i] wr(l)
            const V2 *src = reinterpret_cast<const V2 *>(sA + irow);
#pragma unroll
            for (int l = 0; l < n; l += 2) {
                const V2 v = src[l / 2];
                row[l] = v.x;
                row[l + 1] = v.y;
            }
            deriv_eo<T, n, true>(row, o);
            V2 *dst = reinterpret_cast<V2 *>(sA + irow);
#pragma unroll
            for (int m = 0; m < n; m += 2) dst[m / 2] = V2{o[m], o[m + 1]};
            // j-pencil: sum_l D[l][j] ws(l)
#pragma unroll
            for (int l = 0; l < n; ++l) row[l] = sB[jcol + l * n];
            deriv_eo<T, n, true>(row, o);
#pragma unroll
            for (int m = 0; m < n; ++m) sB[jcol + m * n] = o[m];
        }
        __syncthreads();
        if (act) {
            // pass 5, k-pencil: w and the partial of p.w
            T sdot = T(0);
#pragma unroll
            for (int k = 0; k < n; ++k) {
                const int o3 = k * KS + kcol;
                const T wv = wk[k] + sA[o3] + sB[o3];
                w[gb + k * n2] = wv;
                sdot += u[k] * wv;
            }
            acc += (double)sdot;
        }
    }
    if (PUPD && scal->pdl_early) pdl_trigger();
    if (t < mine) {
        // a wait timed out: record it, let this block's copies land, stop
        if (tid == 0) {
            atomicExch(err, 1);
            if (PUPD) {  // stop the solver's loop: this iteration cannot complete
                scal->status = NB_BREAKDOWN;
                scal->done = 1;
            }
            for (long long tt = t; tt < t + S && tt < mine; ++tt)
                mbar_wait_bounded(&bar[tt % S], (uint32_t)((tt / S) & 1));
        }
        __syncthreads();
        return;
    }
    if (part) {
        const double v = block_sum(acc, sred);
        if (tid == 0) part[blockIdx.x] = v;
        if (PUPD && last_block(&scal->tick_ax)) cg_finish_pap(scal, part, gridDim.x, sred);
    }
}

template <typename T, int n, int MODE, int S>
nb_status launch_ax_pen(int sm_count, long long E, const T *G, const T *u, T *w, const T *r,
                        const T *dinv, T *p, CgScalars *scal, double *part, int *err,
                        int *grid_io, cudaStream_t s)
{
    auto kern = k_ax_pen<T, n, MODE, S>;
    constexpr size_t smem = ax_pen_smem<T, n, S>();
    constexpr int threads = tma_threads<n>();
    static int grid_cache_dev[kMaxDevices] = {};  // per device, as the smem attribute
    int &grid_cache = device_slot(grid_cache_dev);
    if (grid_cache == 0) {
        NB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
        grid_cache = (per_sm < 1 ? 1 : per_sm) * sm_count;
    }
    int grid = (int)(E < grid_cache ? E : grid_cache);
    if (grid < 1) grid = 1;
    if (grid > kMaxPartials) grid = kMaxPartials;
    NB_CUDA(launch_pdl(kern, grid, threads, smem, s, E, G, u, w, r, dinv, p, scal, part, err));
    if (grid_io) *grid_io = grid;
    return NB_OK;
}

// The pencil variant with S stages exists for even n (16-byte bulk copies,
// 8-byte rows) whose stages and work arrays fit a block's shared memory.
template <typename T>
constexpr bool pen_fits(int n, int S)
{
    return n % 2 == 0 && n >= 2 && n <= kMaxn && pen_smem_bytes(sizeof(T), n, S) <= 227 * 1024;
}

template <typename T>
nb_status dispatch_ax_pen(int n, int mode, int S, int sm_count, long long E, const T *G,
                          const T *u, T *w, const T *r, const T *dinv, T *p, CgScalars *scal,
                          double *part, int *err, int *grid, cudaStream_t s)
{
    if (!pen_fits<T>(n, S) || (S != 1 && S != 2) || (mode == 2 && sizeof(T) != 4)) {
        set_error("pencil operator variant unavailable for n=%d, %d stages", n, S);
        return NB_ERR_ARG;
    }
#define NB_PEN_ARGS sm_count, E, G, u, w, r, dinv, p, scal, part, err, grid, s
#define NB_PEN_S(NN, SS)                                                              \
    if constexpr (pen_fits<T>(NN, SS)) {                                              \
        if (S == SS) {                                                                \
            if (mode == 0) return launch_ax_pen<T, NN, 0, SS>(NB_PEN_ARGS);           \
            if (mode == 1) return launch_ax_pen<T, NN, 1, SS>(NB_PEN_ARGS);           \
            if constexpr (sizeof(T) == 4) return launch_ax_pen<T, NN, 2, SS>(NB_PEN_ARGS); \
        }                                                                             \
    }
#define NB_PEN_CASE(NN) \
    case NN:            \
        NB_PEN_S(NN, 1) \
        NB_PEN_S(NN, 2) \
        break;
    switch (n) {
        NB_PEN_CASE(2)
        NB_PEN_CASE(4)
        NB_PEN_CASE(6)
        NB_PEN_CASE(8)
        NB_PEN_CASE(10)
        NB_PEN_CASE(12)
        NB_PEN_CASE(14)
        NB_PEN_CASE(16)
        default:
            break;
    }
#undef NB_PEN_CASE
#undef NB_PEN_S
#undef NB_PEN_ARGS
    set_error("pencil operator variant unavailable for n=%d", n);
    return NB_ERR_ARG;
}

}  // namespace nb
