// The operator with its element data streamed by the Blackwell bulk-copy
// engine (TMA, cp.async.bulk) into a two-stage shared-memory ring.
//
// Same arithmetic and thread mapping as k_ax_cc (nb_ax_impl.cuh): one thread
// per (i,j) column, k layers fully unrolled, the thread's u and w columns in
// registers, wr/ws of one layer exchanged through shared memory.  What
// changes is how the 6 geometric factors and the input vectors reach the
// SM: one elected thread issues bulk copies of the whole element (G: 6 n^3
// values, and u for the plain operator) into the stage that the
// block will use for its next element, completing on an mbarrier, while the
// block computes the current element from the other stage.  The loads are
// no longer tied to registers or warps in flight, so the kernel keeps about
// one element per resident block in flight from HBM.
//
// Forms (MODE): 0 the plain operator w = A_L u; 1 the fused CG step
// p = |dinv| r + beta p, w = A_L p (Jacobi direction); 2 the fused step of
// flexible CG, p = z + beta p with the preconditioned residual z given in
// place of r.  Forms 1 and 2 read r (or z), dinv and p directly from HBM,
// add each block's partial of p.w and let the last block form alpha.
//
// Every wait on an mbarrier is bounded by one second of %globaltimer; a block
// that times out sets *err, waits (bounded) for its own copies and exits.
#pragma once

#include "nb_ax_impl.cuh"
#include "nb_bulk.cuh"
#include "nb_reduce.cuh"

namespace nb {

template <int n>
constexpr int tma_threads()
{
    return ((n * n + 31) / 32) * 32;
}

template <typename T, int n, bool PUPD>
constexpr size_t ax_tma_stage_elems()
{
    // G[6][n3] per stage, plus the element's u for the plain operator (the
    // fused CG step forms p itself into one buffer shared by both stages)
    return (size_t)(PUPD ? 6 : 7) * n * n * n;
}

template <typename T, int n, bool PUPD>
constexpr size_t ax_tma_smem()
{
    return sizeof(T) * (2 * ax_tma_stage_elems<T, n, PUPD>() + (PUPD ? n * n * n : 0) + 4 * n * n);
}

// Blocks per SM that the launch bound asks the compiler to keep room for
// (registers): as many as shared memory admits, for FP32 at n >= 8.
template <typename T, int n, bool PUPD>
constexpr int tma_min_blocks()
{
    if (sizeof(T) != 4 || n < 8) return 1;
    const int by_smem = (int)((228 * 1024) / (ax_tma_smem<T, n, PUPD>() + 1024));
    const int by_threads = 2048 / tma_threads<n>();
    const int b = by_smem < by_threads ? by_smem : by_threads;
    return b < 1 ? 1 : b;
}

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

// One element's operator from shared memory: Gs = G[6][n3] and su = u (n3)
// of the element; ru holds the thread's (i,j) column of u, rw receives that
// column of A_e u.  wr/ws of layer k go through buffer k&1 of swr/sws (ws
// stored transposed, so that both are read as 8-byte rows), with one
// barrier per layer: layer k+1 writes the other buffer, and layer k+2 (this
// buffer again) follows layer k+1's barrier.
template <typename T, int n>
__device__ __forceinline__ void tma_element(const T *Gs, const T *su, const T (&ru)[n], T (&rw)[n],
                                            T *swr, T *sws, const T (&Di)[n], const T (&Dj)[n],
                                            const T (&DTi)[n], const T (&DTj)[n], int i, int j,
                                            int ij, bool act)
{
    constexpr int n2 = n * n, n3 = n2 * n;
    using V2 = typename Vec2<T>::type;
#pragma unroll
    for (int k = 0; k < n; ++k) rw[k] = T(0);
#pragma unroll
    for (int k = 0; k < n; ++k) {
        T *wrb = swr + (k & 1) * n2;
        T *wsb = sws + (k & 1) * n2;
        const T g0 = Gs[0 * n3 + k * n2 + ij], g1 = Gs[1 * n3 + k * n2 + ij];
        const T g2 = Gs[2 * n3 + k * n2 + ij], g3 = Gs[3 * n3 + k * n2 + ij];
        const T g4 = Gs[4 * n3 + k * n2 + ij], g5 = Gs[5 * n3 + k * n2 + ij];
        // even / odd partial sums: six independent chains for latency
        T ur = T(0), us = T(0), ut = T(0), ur1 = T(0), us1 = T(0), ut1 = T(0);
        const V2 *urow = reinterpret_cast<const V2 *>(su + k * n2 + j * n);
#pragma unroll
        for (int l = 0; l < n; l += 2) {
            const V2 v = urow[l / 2];
            ur += Di[l] * v.x;
            ur1 += Di[l + 1] * v.y;
        }
#pragma unroll
        for (int l = 0; l < n; l += 2) {
            us += Dj[l] * su[k * n2 + l * n + i];
            us1 += Dj[l + 1] * su[k * n2 + (l + 1) * n + i];
            ut += dtab<T>(n, k, l) * ru[l];
            ut1 += dtab<T>(n, k, l + 1) * ru[l + 1];
        }
        ur += ur1;
        us += us1;
        ut += ut1;
        const T wr = g0 * ur + g1 * us + g2 * ut;
        const T ws = g1 * ur + g3 * us + g4 * ut;
        const T wt = g2 * ur + g4 * us + g5 * ut;
        if (act) {
            wrb[ij] = wr;
            wsb[i * n + j] = ws;  // transposed: the reads below are rows
        }
        __syncthreads();
        // two independent chains (the wr and ws terms) for latency
        T a = T(0), b = T(0);
        const V2 *wrow = reinterpret_cast<const V2 *>(wrb + j * n);
#pragma unroll
        for (int l = 0; l < n; l += 2) {
            const V2 v = wrow[l / 2];
            a += DTi[l] * v.x;
            a += DTi[l + 1] * v.y;
        }
        const V2 *wsrow = reinterpret_cast<const V2 *>(wsb + i * n);
#pragma unroll
        for (int l = 0; l < n; l += 2) {
            const V2 v = wsrow[l / 2];
            b += DTj[l] * v.x;
            b += DTj[l + 1] * v.y;
        }
        rw[k] += a + b;
#pragma unroll
        for (int m = 0; m < n; ++m) rw[m] += dtab<T>(n, k, m) * wt;
    }
}

template <typename T, int n, int MODE>
__global__ void __launch_bounds__(tma_threads<n>(), (tma_min_blocks<T, n, MODE != 0>()))
k_ax_tma(long long E, const T *__restrict__ G, const T *__restrict__ uin, T *__restrict__ w,
         const T *__restrict__ r, const T *__restrict__ dinv, T *__restrict__ p,
         CgScalars *__restrict__ scal, double *__restrict__ part, int *__restrict__ err)
{
    constexpr bool PUPD = MODE != 0;
    constexpr int n2 = n * n, n3 = n2 * n;
    constexpr int STAGE = (int)ax_tma_stage_elems<T, n, PUPD>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *stage = reinterpret_cast<T *>(smem_raw);  // [2][STAGE]: G[6][n3], then u
    T *pbuf = stage + 2 * STAGE;                 // [n3] the fused step's p (PUPD only)
    T *swr = pbuf + (PUPD ? n3 : 0);             // [2][n2] (double-buffered by layer)
    T *sws = swr + 2 * n2;                       // [2][n2]
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ double sred[32];

    if (PUPD && scal->done) return;
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
    const T beta = PUPD ? (T)scal->beta : T(0);
    const long long mine = E > blockIdx.x ? (E - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();

    // the elected thread streams element number t of this block into stage
    // t&1: its geometric factors, and for the plain operator its u
    auto issue = [&](long long t) {
        const long long e = blockIdx.x + t * gridDim.x;
        T *dst = stage + (t & 1) * STAGE;
        uint64_t *b = &bar[t & 1];
        const uint32_t gbytes = (uint32_t)(6 * n3 * sizeof(T));
        const uint32_t ubytes = PUPD ? 0u : (uint32_t)(n3 * sizeof(T));
        mbar_expect_tx(b, gbytes + ubytes);
        bulk_g2s(dst, G + (size_t)e * 6 * n3, gbytes, b);
        if (!PUPD) bulk_g2s(dst + 6 * n3, uin + (size_t)e * n3, ubytes, b);
    };
    if (tid == 0 && mine > 0) issue(0);

    // the fused forms read their column of r (or z), dinv and p straight from
    // HBM, one element ahead: the loads for element t+1 are in flight while
    // element t is computed (elements own disjoint nodes, so p of t+1 is not
    // written by t)
    T nr[n], nd[n], np[n];
    auto fetch = [&](long long tt) {
        const size_t b2 = (size_t)(blockIdx.x + tt * gridDim.x) * n3 + ij;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            nr[k] = r[b2 + k * n2];
            nd[k] = MODE == 1 ? dinv[b2 + k * n2] : T(1);
            np[k] = p[b2 + k * n2];
        }
    };
    if (PUPD && mine > 0) fetch(0);

    double acc = 0.0;
    long long t = 0;
    for (; t < mine; ++t) {
        if (tid == 0 && t + 1 < mine) issue(t + 1);  // its stage was released at the end of t-1
        const long long e = blockIdx.x + t * gridDim.x;
        const size_t base = (size_t)e * n3 + ij;
        T ru[n], rw[n];
        if (PUPD) {
#pragma unroll
            for (int k = 0; k < n; ++k) ru[k] = fabs(nd[k]) * nr[k] + beta * np[k];
            if (t + 1 < mine) fetch(t + 1);
        }
        const bool ok = mbar_wait_bounded(&bar[t & 1], (uint32_t)((t >> 1) & 1));
        if (__syncthreads_or(!ok)) break;
        T *s = stage + (t & 1) * STAGE;
        const T *Gs = s;
        T *su = PUPD ? pbuf : s + 6 * n3;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            if (PUPD) {
                if (act) {
                    su[k * n2 + ij] = ru[k];
                    p[base + k * n2] = ru[k];
                }
            } else {
                ru[k] = su[k * n2 + ij];
            }
        }
        if (PUPD) __syncthreads();
        tma_element<T, n>(Gs, su, ru, rw, swr, sws, Di, Dj, DTi, DTj, i, j, ij, act);
        if (act) {
            T sdot = T(0);
#pragma unroll
            for (int k = 0; k < n; ++k) {
                w[base + k * n2] = rw[k];
                sdot += ru[k] * rw[k];
            }
            acc += (double)sdot;
        }
        __syncthreads();  // every thread is done with stage t&1: it may be refilled
    }
    if (t < mine) {
        // a wait timed out: record it, let this block's copies land, stop
        if (tid == 0) {
            atomicExch(err, 1);
            if (PUPD) {  // stop the solver's loop: this iteration cannot complete
                scal->status = NB_BREAKDOWN;
                scal->done = 1;
            }
            mbar_wait_bounded(&bar[t & 1], (uint32_t)((t >> 1) & 1));
            if (t + 1 < mine) mbar_wait_bounded(&bar[(t + 1) & 1], (uint32_t)(((t + 1) >> 1) & 1));
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

template <typename T, int n, int MODE>
nb_status launch_ax_tma(int sm_count, long long E, const T *G, const T *u, T *w, const T *r,
                        const T *dinv, T *p, CgScalars *scal, double *part, int *err,
                        int *grid_io, cudaStream_t s)
{
    auto kern = k_ax_tma<T, n, MODE>;
    constexpr size_t smem = ax_tma_smem<T, n, MODE != 0>();
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
    kern<<<grid, threads, smem, s>>>(E, G, u, w, r, dinv, p, scal, part, err);
    NB_CUDA(cudaGetLastError());
    if (grid_io) *grid_io = grid;
    return NB_OK;
}

// The bulk-copy variant needs 16-byte multiples (n even) and two stages in
// the 227 KB of shared memory a block may use.
template <typename T>
constexpr bool tma_fits(int n, bool pupd)
{
    (void)pupd;  // both forms stage G and u
    // the plain form's stages (2 x 7 n^3) are the larger of the two
    return (n % 2 == 0) && sizeof(T) * (2 * (size_t)7 * n * n * n + 4 * n * n) <= 227 * 1024;
}

template <typename T>
nb_status dispatch_ax_tma(int n, int mode, int sm_count, long long E, const T *G, const T *u,
                          T *w, const T *r, const T *dinv, T *p, CgScalars *scal,
                          double *part, int *err, int *grid, cudaStream_t s)
{
    if (!tma_fits<T>(n, mode != 0) || (mode == 2 && sizeof(T) != 4)) {
        set_error("bulk-copy operator variant unavailable for n=%d", n);
        return NB_ERR_ARG;
    }
#define NB_TMA_ARGS sm_count, E, G, u, w, r, dinv, p, scal, part, err, grid, s
#define NB_TMA_CASE(NN)                                                            \
    case NN:                                                                       \
        if constexpr (tma_fits<T>(NN, true)) {                                     \
            if (mode == 0) return launch_ax_tma<T, NN, 0>(NB_TMA_ARGS);            \
            if (mode == 1) return launch_ax_tma<T, NN, 1>(NB_TMA_ARGS);            \
            if constexpr (sizeof(T) == 4) return launch_ax_tma<T, NN, 2>(NB_TMA_ARGS); \
        }                                                                          \
        break;
    switch (n) {
        NB_TMA_CASE(2)
        NB_TMA_CASE(4)
        NB_TMA_CASE(6)
        NB_TMA_CASE(8)
        NB_TMA_CASE(10)
        NB_TMA_CASE(12)
        NB_TMA_CASE(14)
        NB_TMA_CASE(16)
        default:
            break;
    }
#undef NB_TMA_CASE
#undef NB_TMA_ARGS
    set_error("bulk-copy operator variant unavailable for n=%d", n);
    return NB_ERR_ARG;
}

}  // namespace nb
