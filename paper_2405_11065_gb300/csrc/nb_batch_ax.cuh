// Operator for a batch of independent problems: one launch per polynomial
// order present in the batch, over the listed elements of that order (the
// elements of the problems still running; all of the order's elements when
// no list is given).  Same arithmetic and thread mapping as k_ax_cc; in
// addition each element looks up its problem, takes that problem's beta,
// skips problems that have converged (no loads, no stores), and writes its
// own partial sum p.(A_L p) so that the per-problem dot products can be
// formed in a fixed order.  Included by the FP32 and FP64 operator units,
// whose constant derivative tables it reads.
#pragma once

#include "nb_ax_impl.cuh"
#include "nb_ax_tma.cuh"
#include "nb_reduce.cuh"

namespace nb {

// The fused CG step of the batch (p = |dinv| r + beta_q p, w = A_L p, and
// each element's partial of p.w) with the element's geometric factors
// streamed by bulk copy into a two-stage ring, as k_ax_tma: blocks walk the
// order's element list; an element of a problem that has stopped gets no
// copy (its stage's barrier is completed by a plain arrival) and no work.
// Each element's partial is a block sum in a fixed order.  Waits are bounded
// by one second; on a timeout the block sets *err, stops the element's
// problem (NB_BREAKDOWN), waits (bounded) for its own copies and exits.
template <typename T, int n>
__global__ void __launch_bounds__(tma_threads<n>(), (tma_min_blocks<T, n, true>()))
k_bax_tma(long long e_first, const int32_t *__restrict__ list, const int *__restrict__ cnt,
          const T *__restrict__ G, T *__restrict__ w, const T *__restrict__ r,
          const T *__restrict__ dinv, T *__restrict__ p, const int32_t *__restrict__ elem_prob,
          BScal *__restrict__ bs, double *__restrict__ part_e, int *__restrict__ err)
{
    constexpr int n2 = n * n, n3 = n2 * n;
    constexpr int STAGE = 6 * n3;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *stage = reinterpret_cast<T *>(smem_raw);  // [2][6 n3]
    T *pbuf = stage + 2 * STAGE;                 // [n3]
    T *swr = pbuf + n3;                          // [2][n2]
    T *sws = swr + 2 * n2;                       // [2][n2]
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ double sred[32];

    const int tid = threadIdx.x;
    const bool act = tid < n2;
    const int ij = act ? tid : 0;
    const int i = ij % n, j = ij / n;
    T Di[n], Dj[n], DTi[n], DTj[n];
#pragma unroll
    for (int l = 0; l < n; ++l) {
        Di[l] = dtab<T>(n, i, l);
        Dj[l] = dtab<T>(n, j, l);
        DTi[l] = dtab<T>(n, l, i);
        DTj[l] = dtab<T>(n, l, j);
    }
    const long long ne = *cnt;
    const long long mine = ne > blockIdx.x ? (ne - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    // the problem's flags do not change while this kernel runs, so the issuer
    // and the block agree on which elements are live
    auto issue = [&](long long t) {
        const long long eb = list[blockIdx.x + t * gridDim.x];
        uint64_t *b = &bar[t & 1];
        if (bs[elem_prob[eb]].done) {
            mbar_arrive(b);
            return;
        }
        const uint32_t gbytes = (uint32_t)(6 * n3 * sizeof(T));
        mbar_expect_tx(b, gbytes);
        bulk_g2s(stage + (t & 1) * STAGE, G + (size_t)(eb - e_first) * 6 * n3, gbytes, b);
    };
    if (tid == 0 && mine > 0) issue(0);
    // the next live element's column of r, dinv and p, loaded one element
    // ahead (elements own disjoint nodes)
    T nr[n], nd[n], np[n];
    auto fetch = [&](long long tt) {
        const long long eb = list[blockIdx.x + tt * gridDim.x];
        if (bs[elem_prob[eb]].done) return;
        const size_t b2 = (size_t)(eb - e_first) * n3 + ij;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            nr[k] = r[b2 + k * n2];
            nd[k] = dinv[b2 + k * n2];
            np[k] = p[b2 + k * n2];
        }
    };
    if (mine > 0) fetch(0);
    long long t = 0;
    for (; t < mine; ++t) {
        if (tid == 0 && t + 1 < mine) issue(t + 1);  // its stage was released at the end of t-1
        const long long eb = list[blockIdx.x + t * gridDim.x];
        const int prob = elem_prob[eb];
        const bool live = !bs[prob].done;  // uniform over the block
        const size_t base = (size_t)(eb - e_first) * n3 + ij;
        T ru[n], rw[n];
        if (live) {
            const T beta = (T)bs[prob].beta;
#pragma unroll
            for (int k = 0; k < n; ++k) ru[k] = fabs(nd[k]) * nr[k] + beta * np[k];
        }
        if (t + 1 < mine) fetch(t + 1);
        const bool ok = mbar_wait_bounded(&bar[t & 1], (uint32_t)((t >> 1) & 1));
        if (__syncthreads_or(!ok)) break;
        if (!live) continue;  // nothing of this element was read or written
        const T *Gs = stage + (t & 1) * STAGE;
#pragma unroll
        for (int k = 0; k < n; ++k)
            if (act) {
                pbuf[k * n2 + ij] = ru[k];
                p[base + k * n2] = ru[k];
            }
        __syncthreads();
        tma_element<T, n>(Gs, pbuf, ru, rw, swr, sws, Di, Dj, DTi, DTj, i, j, ij, act);
        T sdot = T(0);
        if (act) {
#pragma unroll
            for (int k = 0; k < n; ++k) {
                w[base + k * n2] = rw[k];
                sdot += ru[k] * rw[k];
            }
        }
        const double v = block_sum((double)sdot, sred);  // ends with the block in step
        if (tid == 0) part_e[eb] = v;
        __syncthreads();  // every thread is done with stage t&1 and pbuf
    }
    if (t < mine) {
        if (tid == 0) {
            atomicExch(err, 1);
            const long long eb = list[blockIdx.x + t * gridDim.x];
            bs[elem_prob[eb]].status = NB_BREAKDOWN;
            bs[elem_prob[eb]].done = 1;
            mbar_wait_bounded(&bar[t & 1], (uint32_t)((t >> 1) & 1));
            if (t + 1 < mine) mbar_wait_bounded(&bar[(t + 1) & 1], (uint32_t)(((t + 1) >> 1) & 1));
        }
        __syncthreads();
    }
}

template <typename T, int n>
nb_status launch_bax_tma(int sm_count, long long E, long long e_first, const int32_t *list,
                         const int *cnt, const T *G, T *w, const T *r, const T *dinv, T *p,
                         const int32_t *elem_prob, BScal *bs, double *part_e, int *err,
                         cudaStream_t s)
{
    auto kern = k_bax_tma<T, n>;
    constexpr size_t smem = sizeof(T) * ((size_t)13 * n * n * n + 4 * n * n);
    constexpr int threads = tma_threads<n>();
    static int grid_cache_dev[kMaxDevices] = {};  // per device, as the smem attribute
    int &grid_cache = device_slot(grid_cache_dev);
    if (grid_cache == 0) {
        NB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
        grid_cache = (per_sm < 1 ? 1 : per_sm) * sm_count;
    }
    if (E <= 0) return NB_OK;
    const int grid = (int)(E < grid_cache ? E : grid_cache);
    kern<<<grid, threads, smem, s>>>(e_first, list, cnt, G, w, r, dinv, p, elem_prob, bs, part_e,
                                     err);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// The batch's bulk-copy step exists for even n whose two stages of G, p and
// the layer buffers fit in a block's shared memory.
template <typename T>
constexpr bool bax_tma_fits(int n)
{
    return (n % 2 == 0) && sizeof(T) * ((size_t)13 * n * n * n + 4 * n * n) <= 227 * 1024;
}

template <typename T>
nb_status dispatch_bax_tma(int n, int sm_count, long long E, long long e_first,
                           const int32_t *list, const int *cnt, const T *G, T *w, const T *r,
                           const T *dinv, T *p, const int32_t *elem_prob, BScal *bs,
                           double *part_e, int *err, cudaStream_t s)
{
#define NB_BTMA_CASE(NN)                                                                        \
    case NN:                                                                                    \
        if constexpr (bax_tma_fits<T>(NN))                                                      \
            return launch_bax_tma<T, NN>(sm_count, E, e_first, list, cnt, G, w, r, dinv, p,     \
                                         elem_prob, bs, part_e, err, s);                        \
        break;
    switch (n) {
        NB_BTMA_CASE(2)
        NB_BTMA_CASE(4)
        NB_BTMA_CASE(6)
        NB_BTMA_CASE(8)
        NB_BTMA_CASE(10)
        NB_BTMA_CASE(12)
        NB_BTMA_CASE(14)
        NB_BTMA_CASE(16)
        default:
            break;
    }
#undef NB_BTMA_CASE
    set_error("bulk-copy batch operator unavailable for n=%d", n);
    return NB_ERR_ARG;
}

template <typename T, int n, int M, bool PUPD>
__global__ void __launch_bounds__(M * n * n)
k_bax(long long E, long long e_first, const int32_t *__restrict__ list, const int *__restrict__ cnt,
      const T *__restrict__ G, const T *__restrict__ uin,
      T *__restrict__ w, const T *__restrict__ r, const T *__restrict__ dinv, T *__restrict__ p,
      const int32_t *__restrict__ elem_prob, const BScal *__restrict__ bs,
      double *__restrict__ part_e)
{
    constexpr int n2 = n * n, n3 = n2 * n;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *su = reinterpret_cast<T *>(smem_raw);  // [M][n3]
    T *swr = su + M * n3;                      // [M][n2]
    T *sws = swr + M * n2;                     // [M][n2]
    T *sdot = sws + M * n2;                    // [M][n2]

    const int tid = threadIdx.x;
    const int el = tid / n2, ij = tid - el * n2;
    const int i = ij % n, j = ij / n;
    T Di[n], Dj[n], DTi[n], DTj[n];
#pragma unroll
    for (int l = 0; l < n; ++l) {
        Di[l] = dtab<T>(n, i, l);
        Dj[l] = dtab<T>(n, j, l);
        DTi[l] = dtab<T>(n, l, i);
        DTj[l] = dtab<T>(n, l, j);
    }
    T *sue = su + el * n3;
    T *swre = swr + el * n2;
    T *swse = sws + el * n2;

    // list entries are batch element indices; e is the index within the order
    const long long ne = list ? (long long)*cnt : E;
    for (long long i0 = (long long)blockIdx.x * M; i0 < ne; i0 += (long long)gridDim.x * M) {
        const long long idx = i0 + el;
        const bool valid = idx < ne && el < M;
        const long long e = valid ? (list ? (long long)list[idx] - e_first : idx) : 0;
        const int prob = valid ? elem_prob[e_first + e] : 0;
        const bool live = valid && !(PUPD && bs[prob].done);
        if (!__syncthreads_or(live)) continue;  // block-uniform
        const T beta = (PUPD && live) ? (T)bs[prob].beta : T(0);
        const size_t base = (size_t)e * n3 + ij;
        T ru[n], rw[n];
#pragma unroll
        for (int k = 0; k < n; ++k) {
            T v = T(0);
            if (live) {
                if (PUPD) {
                    v = fabs(dinv[base + k * n2]) * r[base + k * n2] + beta * p[base + k * n2];
                    p[base + k * n2] = v;
                } else {
                    v = uin[base + k * n2];
                }
            }
            ru[k] = v;
            rw[k] = T(0);
            sue[k * n2 + ij] = v;
        }
        __syncthreads();
        const T *Ge = G + (size_t)e * 6 * n3 + ij;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            T g0 = T(0), g1 = T(0), g2 = T(0), g3 = T(0), g4 = T(0), g5 = T(0);
            if (live) {
                g0 = Ge[0 * n3 + k * n2];
                g1 = Ge[1 * n3 + k * n2];
                g2 = Ge[2 * n3 + k * n2];
                g3 = Ge[3 * n3 + k * n2];
                g4 = Ge[4 * n3 + k * n2];
                g5 = Ge[5 * n3 + k * n2];
            }
            T ur = T(0), us = T(0), ut = T(0);
#pragma unroll
            for (int l = 0; l < n; ++l) {
                ur += Di[l] * sue[k * n2 + j * n + l];
                us += Dj[l] * sue[k * n2 + l * n + i];
                ut += dtab<T>(n, k, l) * ru[l];
            }
            const T wr = g0 * ur + g1 * us + g2 * ut;
            const T ws = g1 * ur + g3 * us + g4 * ut;
            const T wt = g2 * ur + g4 * us + g5 * ut;
            swre[ij] = wr;
            swse[ij] = ws;
            __syncthreads();
            T a = T(0);
#pragma unroll
            for (int l = 0; l < n; ++l) {
                a += DTi[l] * swre[j * n + l];
                a += DTj[l] * swse[l * n + i];
            }
            rw[k] += a;
#pragma unroll
            for (int m = 0; m < n; ++m) rw[m] += dtab<T>(n, k, m) * wt;
            __syncthreads();
        }
        T s = T(0);
        if (live) {
#pragma unroll
            for (int k = 0; k < n; ++k) {
                w[base + k * n2] = rw[k];
                s += ru[k] * rw[k];
            }
        }
        if (part_e) {
            sdot[el * n2 + ij] = s;
            __syncthreads();
            if (ij == 0 && live) {  // the element's partial, summed in a fixed order
                double t = 0.0;
                for (int q = 0; q < n2; ++q) t += (double)sdot[el * n2 + q];
                part_e[e_first + e] = t;
            }
        }
    }
}

template <typename T, int n, int M, bool PUPD>
nb_status launch_bax(int sm_count, long long E, long long e_first, const int32_t *list,
                     const int *cnt, const T *G, const T *u, T *w, const T *r, const T *dinv, T *p,
                     const int32_t *elem_prob, const BScal *bs, double *part_e, cudaStream_t s)
{
    auto kern = k_bax<T, n, M, PUPD>;
    constexpr size_t smem = sizeof(T) * (size_t)M * (n * n * n + 3 * n * n);
    constexpr int threads = M * n * n;
    static int grid_cache_dev[kMaxDevices] = {};  // per device, as the smem attribute
    int &grid_cache = device_slot(grid_cache_dev);
    if (grid_cache == 0) {
        if (smem > 48 * 1024)
            NB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        int per_sm = 0;
        NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
        grid_cache = (per_sm < 1 ? 1 : per_sm) * sm_count;
    }
    if (E <= 0) return NB_OK;
    const long long need = (E + M - 1) / M;
    const int grid = (int)(need < grid_cache ? need : grid_cache);
    kern<<<grid, threads, smem, s>>>(E, e_first, list, cnt, G, u, w, r, dinv, p, elem_prob, bs,
                                     part_e);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

template <typename T>
nb_status dispatch_bax(int n, int mchoice, bool pupd, int sm_count, long long E, long long e_first,
                       const int32_t *list, const int *cnt, const T *G, const T *u, T *w,
                       const T *r, const T *dinv, T *p, const int32_t *elem_prob, const BScal *bs,
                       double *part_e, cudaStream_t s)
{
#define NB_BAX_ARGS sm_count, E, e_first, list, cnt, G, u, w, r, dinv, p, elem_prob, bs, part_e, s
#define NB_BAX_CASE(NN, M0, M1)                                                     \
    case NN:                                                                        \
        if (pupd)                                                                   \
            return mchoice ? launch_bax<T, NN, M1, true>(NB_BAX_ARGS)               \
                           : launch_bax<T, NN, M0, true>(NB_BAX_ARGS);              \
        return mchoice ? launch_bax<T, NN, M1, false>(NB_BAX_ARGS)                  \
                       : launch_bax<T, NN, M0, false>(NB_BAX_ARGS);
    switch (n) {
        NB_BAX_CASE(2, 16, 32)
        NB_BAX_CASE(3, 8, 16)
        NB_BAX_CASE(4, 4, 8)
        NB_BAX_CASE(5, 2, 4)
        NB_BAX_CASE(6, 2, 4)
        NB_BAX_CASE(7, 1, 2)
        NB_BAX_CASE(8, 1, 2)
        NB_BAX_CASE(9, 1, 2)
        NB_BAX_CASE(10, 1, 2)
        NB_BAX_CASE(11, 1, 2)
        NB_BAX_CASE(12, 1, 2)
        NB_BAX_CASE(13, 1, 1)
        NB_BAX_CASE(14, 1, 1)
        NB_BAX_CASE(15, 1, 1)
        NB_BAX_CASE(16, 1, 1)
        default:
            set_error("unsupported order n=%d", n);
            return NB_ERR_ARG;
    }
#undef NB_BAX_CASE
#undef NB_BAX_ARGS
}

}  // namespace nb
