// The matrix-free spectral-element operator on CUDA cores (FP64 or FP32).
//
// ax (Table 1 line 5) applies, element by element, the three reference
// derivatives (local_grad3), the symmetric 3x3 geometric tensor per node, and
// the three transposed derivatives summed (local_grad3_t + add2):
//   ur = sum_l D[i][l] u(l,j,k), us = sum_l D[j][l] u(i,l,k), ut = sum_l D[k][l] u(i,j,l)
//   (wr, ws, wt) = G (ur, us, ut)
//   w(i,j,k) = sum_l D[l][i] wr(l,j,k) + D[l][j] ws(i,l,k) + D[l][k] wt(i,j,l)
//
// GPU mapping.  A thread owns one (i,j) column of an element and walks the k
// layers; M elements share a block.  The element's u is staged in shared
// memory; the thread keeps its own column u(i,j,:) and its output column
// w(i,j,:) in registers, so the t-direction contraction and its transpose
// never touch shared memory.  Per layer only wr and ws go through shared
// memory.  The rows D[i][:], D[j][:] and columns D[:][i], D[:][j] that a thread
// needs live in registers; the layer-indexed entries D[k][:] are compile-time
// constant-bank operands (the k loop is fully unrolled).  Geometric factors
// stream from HBM once, coalesced along (i,j).
//
// CG fusion: with PUPD the kernel first forms the search direction
// p = dinv*r + beta*p (add2s1 with the Jacobi solveM folded in) for its
// nodes, writes p, and applies the operator to it.  With a partial-sum buffer
// it also returns per-block FP64 partials of sum_l p_l (A_L p)_l, which equals
// glsc3(w, c, p) of the assembled w for a continuous masked p.
#pragma once

#include "nb_cg_dev.cuh"

namespace nb {

template <typename T>
__device__ __forceinline__ T dtab(int n, int i, int l);  // defined per translation unit

// Even-odd halves of the derivative matrix (even n), defined per translation
// unit: which = 0, 1 the even / odd half of D, 2, 3 those of D^T.
template <typename T>
__device__ __forceinline__ T eotab(int n, int which, int i, int l);

// out = D in (TRANS false) or D^T in (TRANS true) along one line of n points,
// n even, by the even-odd decomposition (Solomonoff 1992): D is
// centro-antisymmetric, D[N-i][N-l] = -D[i][l], and so is D^T; with
// e_l = in[l] + in[N-l], o_l = in[l] - in[N-l] (l < n/2), P = A e and Q = B o
// for the n/2 x n/2 halves A = (D[i][l] + D[i][N-l]) / 2 and
// B = (D[i][l] - D[i][N-l]) / 2, out[i] = Q + P and out[N-i] = Q - P.
// n^2 / 2 multiply-adds and 2n additions instead of n^2 multiply-adds.
template <typename T, int n, bool TRANS>
__device__ __forceinline__ void deriv_eo(const T (&in)[n], T (&out)[n])
{
    static_assert(n % 2 == 0, "even-odd decomposition needs an even n");
    constexpr int h = n / 2, N = n - 1, wa = TRANS ? 2 : 0;
    T e[h], o[h];
#pragma unroll
    for (int l = 0; l < h; ++l) {
        e[l] = in[l] + in[N - l];
        o[l] = in[l] - in[N - l];
    }
#pragma unroll
    for (int i = 0; i < h; ++i) {
        T P = T(0), Q = T(0);
#pragma unroll
        for (int l = 0; l < h; ++l) {
            P += eotab<T>(n, wa, i, l) * e[l];
            Q += eotab<T>(n, wa + 1, i, l) * o[l];
        }
        out[i] = Q + P;
        out[N - i] = Q - P;
    }
}

template <typename T, int n, int M, bool PUPD>
__global__ void __launch_bounds__(M * n * n)
k_ax_cc(long long E, const T *__restrict__ G, const T *__restrict__ uin, T *__restrict__ w,
        const T *__restrict__ r, const T *__restrict__ dinv, T *__restrict__ p,
        CgScalars *__restrict__ scal, double *__restrict__ part)
{
    constexpr int n2 = n * n, n3 = n2 * n;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *su = reinterpret_cast<T *>(smem_raw);        // [M][n3]
    T *swr = su + M * n3;                            // [M][n2]
    T *sws = swr + M * n2;                           // [M][n2]
    __shared__ double sred[32];

    if (PUPD && scal->done) return;  // the solve has stopped: leave p and w untouched
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
    T beta = T(0);
    if (PUPD) beta = (T)scal->beta;
    double acc = 0.0;
    T *sue = su + el * n3;
    T *swre = swr + el * n2;
    T *swse = sws + el * n2;

    for (long long e0 = (long long)blockIdx.x * M; e0 < E; e0 += (long long)gridDim.x * M) {
        const long long e = e0 + el;
        const bool valid = e < E;
        const size_t base = (size_t)e * n3 + ij;
        T ru[n], rw[n];
#pragma unroll
        for (int k = 0; k < n; ++k) {
            T v = T(0);
            if (valid) {
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
        const T *Ge = G + (size_t)(valid ? e : 0) * 6 * n3 + ij;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            T g0 = Ge[0 * n3 + k * n2], g1 = Ge[1 * n3 + k * n2], g2 = Ge[2 * n3 + k * n2];
            T g3 = Ge[3 * n3 + k * n2], g4 = Ge[4 * n3 + k * n2], g5 = Ge[5 * n3 + k * n2];
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
        if (valid) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < n; ++k) {
                w[base + k * n2] = rw[k];
                s += ru[k] * rw[k];
            }
            acc += (double)s;
        }
    }
    if (part) {
        const double v = block_sum(acc, sred);
        if (tid == 0) part[blockIdx.x] = v;
        // in the solver, the last block to finish turns the partials into alpha
        if (PUPD && last_block(&scal->tick_ax)) cg_finish_pap(scal, part, gridDim.x, sred);
    }
}

template <typename T, int n, int M>
constexpr size_t ax_cc_smem()
{
    return sizeof(T) * (size_t)M * (n * n * n + 2 * n * n);
}

// Launch helper: computes a persistent grid once from the occupancy.
template <typename T, int n, int M, bool PUPD>
nb_status launch_ax_cc(int sm_count, long long E, const T *G, const T *u, T *w, const T *r,
                       const T *dinv, T *p, CgScalars *scal, double *part, int *grid_io,
                       cudaStream_t s)
{
    auto kern = k_ax_cc<T, n, M, PUPD>;
    constexpr size_t smem = ax_cc_smem<T, n, M>();
    constexpr int threads = M * n * n;
    static int grid_cache_dev[kMaxDevices] = {};  // per device, as the smem attribute
    int &grid_cache = device_slot(grid_cache_dev);
    if (grid_cache == 0) {
        if (smem > 48 * 1024)
            NB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        int per_sm = 0;
        NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
        if (per_sm < 1) per_sm = 1;
        grid_cache = per_sm * sm_count;
    }
    long long need = (E + M - 1) / M;
    int grid = (int)(need < grid_cache ? need : grid_cache);
    if (grid < 1) grid = 1;
    if (grid > kMaxPartials) grid = kMaxPartials;
    kern<<<grid, threads, smem, s>>>(E, G, u, w, r, dinv, p, scal, part);
    NB_CUDA(cudaGetLastError());
    if (grid_io) *grid_io = grid;
    return NB_OK;
}

// Dispatch over the order for one value type: choice = elements per block
// index (0: small M, 1: large M).
template <typename T>
nb_status dispatch_ax_cc(int n, int mchoice, bool pupd, int sm_count, long long E, const T *G,
                         const T *u, T *w, const T *r, const T *dinv, T *p,
                         CgScalars *scal, double *part, int *grid, cudaStream_t s)
{
#define NB_AX_CASE(NN, M0, M1)                                                                 \
    case NN:                                                                                   \
        if (pupd)                                                                              \
            return mchoice ? launch_ax_cc<T, NN, M1, true>(sm_count, E, G, u, w, r, dinv, p,   \
                                                           scal, part, grid, s)                \
                           : launch_ax_cc<T, NN, M0, true>(sm_count, E, G, u, w, r, dinv, p,   \
                                                           scal, part, grid, s);               \
        return mchoice ? launch_ax_cc<T, NN, M1, false>(sm_count, E, G, u, w, r, dinv, p,      \
                                                        scal, part, grid, s)                   \
                       : launch_ax_cc<T, NN, M0, false>(sm_count, E, G, u, w, r, dinv, p,      \
                                                        scal, part, grid, s);
    switch (n) {
        NB_AX_CASE(2, 16, 32)
        NB_AX_CASE(3, 8, 16)
        NB_AX_CASE(4, 4, 8)
        NB_AX_CASE(5, 2, 4)
        NB_AX_CASE(6, 2, 4)
        NB_AX_CASE(7, 1, 2)
        NB_AX_CASE(8, 1, 2)
        NB_AX_CASE(9, 1, 2)
        NB_AX_CASE(10, 1, 2)
        NB_AX_CASE(11, 1, 2)
        NB_AX_CASE(12, 1, 2)
        NB_AX_CASE(13, 1, 2)
        NB_AX_CASE(14, 1, 2)
        NB_AX_CASE(15, 1, 2)
        NB_AX_CASE(16, 1, 2)
        default:
            set_error("unsupported order n=%d", n);
            return NB_ERR_ARG;
    }
#undef NB_AX_CASE
}

}  // namespace nb
