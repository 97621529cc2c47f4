// Learned per-element preconditioner and flexible CG.
//
// The network maps an element's residual, divided by its norm, to a
// correction of the same length d = (N+1)^3: one hidden layer of width h with
// GELU whose output layer reuses the input weights (tied), with per-unit
// gains a:  y(x) = W (a * gelu(W^T x)).  Its Jacobian
// W diag(a gelu'(W^T x)) W^T is symmetric at every input, which the
// short-recurrence flexible CG needs.  The preconditioner is Jacobi plus the
// scaled network output on the element's interior nodes:
//     z = Dinv r + M_int ( |r_e| y(r_e / |r_e|) )
// Interior nodes belong to one element only, so z is continuous without a
// summation.  The network is trained to supply what Jacobi misses inside an
// element: its targets are (A_ii^-1 r_i - Dinv r_i) / |r_e|, the
// element-interior solve minus the Jacobi step, for residuals that the
// solver itself produces (Jacobi-PCG iterates first, then flexible-CG
// iterates with the network being trained).  Being nonlinear, it is used
// inside flexible CG (Notay 2000, one-vector truncation), with Jacobi-PCG as
// the fallback when the flexible iteration fails and the FP64 residual of the
// refinement deciding convergence.
//
// Matrix products: BF16 operands on the fifth-generation tensor cores
// (tcgen05.mma, FP32 accumulators in tensor memory); master weights and Adam
// moments in FP32.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "nb_bulk.cuh"
#include "nb_cg_dev.cuh"
#include "nb_tc.cuh"

struct nb_model {
    nb_ctx *ctx = nullptr;
    int N = 0, d = 0, h = 0;
    float *W = nullptr, *a = nullptr;  // FP32 master: W (d x h, row-major), gains a (h)
    float *m = nullptr, *v = nullptr;  // Adam moments over all parameters (contiguous)
    float *grad = nullptr;             // gradients, same layout
    int64_t nparam = 0;
    int64_t step = 0;
    // scratch for a batch (grown on demand)
    int cap = 0;
    float *Z = nullptr, *H = nullptr, *Y = nullptr, *dY = nullptr, *dH = nullptr, *nrm = nullptr;
    float *gpart = nullptr;  // per-block partials of the gain gradient
    // BF16 shared-memory image of W for the fused preconditioner (core
    // matrices, k_w_image); refreshed when the weights changed (step)
    __nv_bfloat16 *Wimg = nullptr;
    int64_t wimg_step = -1;
    float *X = nullptr;
    double *lpart = nullptr;
};

namespace nb {

// ---------------------------------------------------------------------------
// BF16 tensor-core matrix product: C = op(A) op(B) (+ epilogue)
//   A: M x K (TA: stored K x M), B: K x N (TB: stored N x K), FP32 in memory,
//   rounded to BF16 when staged in shared memory; FP32 accumulation in
//   tensor memory (tcgen05.mma, issued by one thread, completion on an
//   mbarrier).
// ---------------------------------------------------------------------------

constexpr int GBM = 128, GBN = 64, GBK = 32;  // tile: the MMA's M and N, K per stage

enum GemmEpi { EPI_STORE = 0, EPI_GELU_GAIN = 1, EPI_ADD = 2, EPI_PRECOND = 3 };

struct GemmArgs {
    int M, N, K;
    const float *A;
    int lda;
    const float *B;
    int ldb;
    float *C;
    int ldc;
    const float *gain;     // [N] (EPI_GELU_GAIN)
    float *C2;             // EPI_GELU_GAIN: gain * gelu(C) written here (ldc)
    const float *rowscale; // EPI_PRECOND: per-row factor |r_e|
    const float *rvec;     // EPI_PRECOND: the residual (M x N, ldc)
    const float *dinv;     // EPI_PRECOND: signed Jacobi inverse diagonal (M x N, ldc)
    int n;                 // EPI_PRECOND: points per direction (N = n^3 columns)
};

__device__ __forceinline__ float gelu_f(float z)
{
    const float c = 0.7978845608028654f;  // sqrt(2/pi)
    return 0.5f * z * (1.0f + tanhf(c * (z + 0.044715f * z * z * z)));
}

__device__ __forceinline__ float gelu_grad_f(float z)
{
    const float c = 0.7978845608028654f;
    const float u = c * (z + 0.044715f * z * z * z);
    const float t = tanhf(u);
    const float du = c * (1.0f + 3.0f * 0.044715f * z * z);
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * du;
}

// One 128 x 64 tile of C per CTA (4 warps).  Per K stage of 32 the threads
// stage op(A) (128 x 32) and op(B)^T (64 x 32) as BF16 in the K-major
// core-matrix layout (two buffers; a buffer is rewritten once the MMAs that
// read it have signalled their mbarrier), thread 0 issues two MMAs of K = 16.
// Warp w then reads the accumulator rows 32 w .. 32 w + 31 (its tensor-memory
// lanes) and applies the epilogue.  Every wait is bounded (one second); on a
// timeout the kernel sets *err, skips the epilogue and frees its tensor
// memory.
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128) k_gemm_tc(GemmArgs g, int *err)
{
    __shared__ __align__(1024) __nv_bfloat16 As[2][GBM * GBK];
    __shared__ __align__(1024) __nv_bfloat16 Bs[2][GBN * GBK];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&tslot, 64);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    constexpr uint32_t idesc = tc::idesc_bf16(GBM, GBN, false, false);
    const int nk = (g.K + GBK - 1) / GBK;
    bool ok = true;
    for (int kc = 0; kc < nk; ++kc) {
        const int buf = kc & 1, k0 = kc * GBK;
        // the MMAs of stage kc - 2 read this buffer
        if (kc >= 2 && __syncthreads_or(tid == 0 && !mbar_wait_bounded(&bar[buf], ((kc - 2) >> 1) & 1))) {
            ok = false;
            break;
        }
        // op(A)[m][k]: consecutive threads along the stored row
        for (int q = tid; q < GBM * GBK; q += 128) {
            int mm, kk;
            if (TA) { mm = q % GBM; kk = q / GBM; } else { kk = q % GBK; mm = q / GBK; }
            const int gm = m0 + mm, gk = k0 + kk;
            float v = 0.f;
            if (gm < g.M && gk < g.K) v = TA ? g.A[(size_t)gk * g.lda + gm] : g.A[(size_t)gm * g.lda + gk];
            As[buf][tc::kmajor_off(mm, kk, GBK / 8)] = __float2bfloat16_rn(v);
        }
        // op(B)^T[n][k] = op(B)[k][n]
        for (int q = tid; q < GBN * GBK; q += 128) {
            int nn, kk;
            if (TB) { kk = q % GBK; nn = q / GBK; } else { nn = q % GBN; kk = q / GBN; }
            const int gn = n0 + nn, gk = k0 + kk;
            float v = 0.f;
            if (gn < g.N && gk < g.K) v = TB ? g.B[(size_t)gn * g.ldb + gk] : g.B[(size_t)gk * g.ldb + gn];
            Bs[buf][tc::kmajor_off(nn, kk, GBK / 8)] = __float2bfloat16_rn(v);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            const uint32_t a0 = smem_u32(As[buf]), b0 = smem_u32(Bs[buf]);
#pragma unroll
            for (int ks = 0; ks < GBK / 16; ++ks)
                tc::mma_bf16(tmem, tc::sdesc(a0 + 256u * ks, 128u, 16u * GBK),
                             tc::sdesc(b0 + 256u * ks, 128u, 16u * GBK), idesc, kc > 0 || ks > 0);
            tc::commit(&bar[buf]);
        }
    }
    // the last stage's commit covers every MMA issued before it
    if (ok && nk > 0 &&
        __syncthreads_or(tid == 0 && !mbar_wait_bounded(&bar[(nk - 1) & 1], ((nk - 1) >> 1) & 1)))
        ok = false;
    if (!ok) {
        if (tid == 0) {
            atomicExch(err, 1);
            for (int b = 0; b < 2; ++b) mbar_wait_bounded(&bar[b], 0);  // let the MMAs land
        }
    } else {
        tc::fence_after_sync();
        const int row = m0 + 32 * warp + lane;
#pragma unroll
        for (int c0 = 0; c0 < GBN; c0 += 16) {
            float acc[16];
            if (nk > 0) {
                tc::ld_x16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, acc);
                tc::wait_ld();
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[j] = 0.f;
            }
            if (row >= g.M) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int col = n0 + c0 + j;
                if (col >= g.N) continue;
                const float v = acc[j];
                const size_t o = (size_t)row * g.ldc + col;
                if (EPI == EPI_GELU_GAIN) {
                    if (g.C) g.C[o] = v;
                    g.C2[o] = g.gain[col] * gelu_f(v);
                } else if (EPI == EPI_ADD) {
                    g.C[o] += v;
                } else if (EPI == EPI_PRECOND) {
                    // Jacobi everywhere, plus the learned correction on the
                    // element's interior nodes (which have a single copy)
                    const int ci = col % g.n, cj = (col / g.n) % g.n, ck = col / (g.n * g.n);
                    const bool inner = ci > 0 && ci < g.n - 1 && cj > 0 && cj < g.n - 1 &&
                                       ck > 0 && ck < g.n - 1;
                    float z = fabsf(g.dinv[o]) * g.rvec[o];
                    if (inner) z += v * g.rowscale[row];
                    g.C[o] = z;
                } else {
                    g.C[o] = v;
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// Error flag of the product kernel (device memory, zero while no wait timed out).
static int *gemm_err()
{
    static int *flag_dev[kMaxDevices] = {};
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return nullptr;
    if (!flag_dev[d]) {
        if (cudaMalloc(&flag_dev[d], sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(flag_dev[d], 0, sizeof(int)) != cudaSuccess) return nullptr;
    }
    return flag_dev[d];
}

// After a synchronisation: NB_ERR_CUDA (and the flag cleared) if a product's
// wait timed out since the last check.
static nb_status gemm_check()
{
    int *err = gemm_err();
    if (!err) return NB_OK;
    int v = 0;
    NB_CUDA(cudaMemcpy(&v, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (v) {
        cudaMemset(err, 0, sizeof(int));
        set_error("matrix product: a wait inside the kernel timed out");
        return NB_ERR_CUDA;
    }
    return NB_OK;
}

template <bool TA, bool TB, int EPI>
static nb_status gemm(const GemmArgs &a, cudaStream_t s)
{
    int *err = gemm_err();
    if (!err) {
        set_error("matrix product: no device error flag");
        return NB_ERR_CUDA;
    }
    dim3 grid((a.N + GBN - 1) / GBN, (a.M + GBM - 1) / GBM);
    k_gemm_tc<TA, TB, EPI><<<grid, 128, 0, s>>>(a, err);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// ---------------------------------------------------------------------------
// element-wise kernels
// ---------------------------------------------------------------------------

// Row norms of an L-vector viewed as rows of d values and the rows divided
// by them (zero rows stay zero).  One block per row.
template <typename T>
__global__ void k_rownorm(int rows, int d, const T *__restrict__ r, float *__restrict__ X,
                          float *__restrict__ nrm)
{
    __shared__ double sred[32];
    for (int e = blockIdx.x; e < rows; e += gridDim.x) {
        double acc = 0.0;
        for (int q = threadIdx.x; q < d; q += blockDim.x) {
            const double v = (double)r[(size_t)e * d + q];
            acc += v * v;
        }
        __shared__ float snrm;
        const double t = block_sum(acc, sred);
        if (threadIdx.x == 0) snrm = (float)sqrt(t);
        __syncthreads();
        const float nv = snrm;
        const float inv = nv > 0.f ? 1.0f / nv : 0.f;
        for (int q = threadIdx.x; q < d; q += blockDim.x)
            X[(size_t)e * d + q] = (float)r[(size_t)e * d + q] * inv;
        if (threadIdx.x == 0) nrm[e] = nv;
        __syncthreads();
    }
}

// Training pairs for the element-interior correction.  For each listed
// element: X = r_e / |r_e|, and T = (A_ii^-1 r_i - Dinv r_i) / |r_e| on the
// element's interior nodes (0 on its boundary nodes), where A_ii is the block
// of the operator on the element's interior nodes (they belong to this
// element only) and Dinv the Jacobi inverse diagonal.  A_ii^-1 r_i is computed
// by conjugate gradients on the element, one block per element, with the
// element operator applied node by node in FP64 (training data, not the hot
// path).  Shared memory: p, w, wr, ws, wt, x, res (7 n^3 doubles) and D.
__device__ __forceinline__ bool interior_node(int q, int n)
{
    const int i = q % n, j = (q / n) % n, k = q / (n * n);
    return i > 0 && i < n - 1 && j > 0 && j < n - 1 && k > 0 && k < n - 1;
}

// Block-wide sum returned to every thread (block_sum gives it to thread 0).
__device__ __forceinline__ double block_sum_all(double v, double *sred, double *slot)
{
    const double t = block_sum(v, sred);
    if (threadIdx.x == 0) *slot = t;
    __syncthreads();
    const double r = *slot;
    __syncthreads();
    return r;
}

__global__ void k_interior_pairs(int count, int n, const int32_t *__restrict__ elems,
                                 const double *__restrict__ r, const double *__restrict__ G,
                                 const double *__restrict__ Dg, const double *__restrict__ dinv,
                                 double tol, int maxit, float *__restrict__ X,
                                 float *__restrict__ T)
{
    extern __shared__ double shd[];
    const int n3 = n * n * n;
    double *sp = shd, *sw = sp + n3, *swr = sw + n3, *sws = swr + n3, *swt = sws + n3;
    double *sx = swt + n3, *sres = sx + n3, *sD = sres + n3;  // sD: n*n
    __shared__ double sred[32];
    __shared__ double slot;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) sD[t] = Dg[t];
    __syncthreads();
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        const int64_t e = elems[q];
        const double *re = r + e * n3;
        const double *Ge = G + e * 6 * n3;
        double acc = 0.0;
        for (int t = threadIdx.x; t < n3; t += blockDim.x) acc += re[t] * re[t];
        const double rn = sqrt(block_sum_all(acc, sred, &slot));
        const double inv = rn > 0.0 ? 1.0 / rn : 0.0;
        acc = 0.0;
        for (int t = threadIdx.x; t < n3; t += blockDim.x) {
            X[(size_t)q * n3 + t] = (float)(re[t] * inv);
            const double bi = interior_node(t, n) ? re[t] * inv : 0.0;  // the scaled system
            sx[t] = 0.0;
            sres[t] = bi;
            sp[t] = bi;
            acc += bi * bi;
        }
        // every thread holds the same rr, so the loop below is uniform
        double rr = block_sum_all(acc, sred, &slot);
        const double rr0 = rr;
        for (int it = 0; it < maxit && rr > tol * tol * rr0; ++it) {
            // w = M_int A_e M_int p (p is zero off the interior)
            for (int t = threadIdx.x; t < n3; t += blockDim.x) {
                const int i = t % n, j = (t / n) % n, k = t / (n * n);
                double ur = 0.0, us = 0.0, ut = 0.0;
                for (int l = 0; l < n; ++l) {
                    ur += sD[i * n + l] * sp[(k * n + j) * n + l];
                    us += sD[j * n + l] * sp[(k * n + l) * n + i];
                    ut += sD[k * n + l] * sp[(l * n + j) * n + i];
                }
                const double g0 = Ge[t], g1 = Ge[n3 + t], g2 = Ge[2 * n3 + t];
                const double g3 = Ge[3 * n3 + t], g4 = Ge[4 * n3 + t], g5 = Ge[5 * n3 + t];
                swr[t] = g0 * ur + g1 * us + g2 * ut;
                sws[t] = g1 * ur + g3 * us + g4 * ut;
                swt[t] = g2 * ur + g4 * us + g5 * ut;
            }
            __syncthreads();
            acc = 0.0;
            for (int t = threadIdx.x; t < n3; t += blockDim.x) {
                const int i = t % n, j = (t / n) % n, k = t / (n * n);
                double s = 0.0;
                if (interior_node(t, n)) {
                    for (int l = 0; l < n; ++l) s += sD[l * n + i] * swr[(k * n + j) * n + l];
                    for (int l = 0; l < n; ++l) s += sD[l * n + j] * sws[(k * n + l) * n + i];
                    for (int l = 0; l < n; ++l) s += sD[l * n + k] * swt[(l * n + j) * n + i];
                }
                sw[t] = s;
                acc += s * sp[t];
            }
            const double pap = block_sum_all(acc, sred, &slot);
            if (!(pap > 0.0)) break;  // uniform
            const double alpha = rr / pap;
            acc = 0.0;
            for (int t = threadIdx.x; t < n3; t += blockDim.x) {
                sx[t] += alpha * sp[t];
                sres[t] -= alpha * sw[t];
                acc += sres[t] * sres[t];
            }
            const double rr1 = block_sum_all(acc, sred, &slot);
            const double beta = rr1 / rr;
            for (int t = threadIdx.x; t < n3; t += blockDim.x) sp[t] = sres[t] + beta * sp[t];
            __syncthreads();
            rr = rr1;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < n3; t += blockDim.x) {
            const double v =
                interior_node(t, n) ? sx[t] - fabs(dinv[e * n3 + t]) * re[t] * inv : 0.0;
            T[(size_t)q * n3 + t] = (float)v;
        }
        __syncthreads();
    }
}

// dY = 2 (Y - T) / (B d) and per-block partials of sum (Y - T)^2.
__global__ void k_mse(int64_t n, const float *__restrict__ Y, const float *__restrict__ T,
                      float scale, float *__restrict__ dY, double *__restrict__ part)
{
    __shared__ double sred[32];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float e = Y[i] - T[i];
        dY[i] = 2.0f * e * scale;
        acc += (double)e * (double)e;
    }
    const double t = block_sum(acc, sred);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Backward through the hidden layer of the tied network.  G = dY W holds the
// gradient with respect to the scaled activations a * gelu(Z); in place it
// becomes dZ = G * a * gelu'(Z), and each block leaves its partial of the
// gain gradient sum_b G * gelu(Z) per unit in gpart[block][h] (rows in a
// fixed order: block-strided, then summed by k_colsum in block order).
__global__ void k_tied_back(int rows, int h, const float *__restrict__ Z,
                            const float *__restrict__ gain, float *__restrict__ G,
                            float *__restrict__ gpart)
{
    for (int c = threadIdx.x; c < h; c += blockDim.x) {
        const float ac = gain[c];
        float s = 0.f;
        for (int r = blockIdx.x; r < rows; r += gridDim.x) {
            const size_t o = (size_t)r * h + c;
            const float z = Z[o], gv = G[o];
            s += gv * gelu_f(z);
            G[o] = gv * ac * gelu_grad_f(z);
        }
        gpart[(size_t)blockIdx.x * h + c] = s;
    }
}

// Column sums of a rows x cols matrix, each column summed in row order by
// one thread.
__global__ void k_colsum(int rows, int cols, const float *__restrict__ A, float *__restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += A[(size_t)r * cols + c];
    out[c] = s;
}

__global__ void k_adam(int64_t n, float *__restrict__ p, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, float lr, float b1, float b2,
                       float c1, float c2, float eps)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// z += |dinv| * r (optional Jacobi term of the learned preconditioner)
// ---------------------------------------------------------------------------
// model helpers
// ---------------------------------------------------------------------------

constexpr int kBackBlocks = 64;  // blocks of k_tied_back (partials of the gain gradient)

static nb_status model_scratch(nb_model *md, int rows)
{
    if (!gemm_err()) {  // allocated here, before any graph capture
        set_error("matrix product: no device error flag");
        return NB_ERR_OOM;
    }
    if (rows <= md->cap) return NB_OK;
    float *bufs[] = {md->Z, md->H, md->Y, md->dY, md->dH, md->nrm, md->X, md->gpart};
    for (float *b : bufs) cudaFree(b);
    cudaFree(md->lpart);
    const size_t R = (size_t)rows;
    NB_CUDA(cudaMalloc(&md->Z, sizeof(float) * R * md->h));
    NB_CUDA(cudaMalloc(&md->H, sizeof(float) * R * md->h));
    NB_CUDA(cudaMalloc(&md->dH, sizeof(float) * R * md->h));
    NB_CUDA(cudaMalloc(&md->Y, sizeof(float) * R * md->d));
    NB_CUDA(cudaMalloc(&md->dY, sizeof(float) * R * md->d));
    NB_CUDA(cudaMalloc(&md->X, sizeof(float) * R * md->d));
    NB_CUDA(cudaMalloc(&md->nrm, sizeof(float) * R));
    NB_CUDA(cudaMalloc(&md->lpart, sizeof(double) * 4096));
    NB_CUDA(cudaMalloc(&md->gpart, sizeof(float) * kBackBlocks * md->h));
    md->cap = rows;
    return NB_OK;
}

// Forward pass of B rows of X: Z = X W, H = a * gelu(Z), Y = H W^T.
static nb_status model_forward(nb_model *md, const float *X, int B, cudaStream_t s)
{
    GemmArgs a = {};
    a.M = B; a.N = md->h; a.K = md->d;
    a.A = X; a.lda = md->d; a.B = md->W; a.ldb = md->h;
    a.C = md->Z; a.ldc = md->h; a.gain = md->a; a.C2 = md->H;
    NB_TRY((gemm<false, false, EPI_GELU_GAIN>(a, s)));
    GemmArgs b = {};  // op(B) = W^T: B stored d x h
    b.M = B; b.N = md->d; b.K = md->h;
    b.A = md->H; b.lda = md->h; b.B = md->W; b.ldb = md->h;
    b.C = md->Y; b.ldc = md->d;
    return gemm<false, true, EPI_STORE>(b, s);
}

// Loss and gradients (into md->grad) for B pairs; *loss_dev = sum (Y-T)^2.
static nb_status model_backward(nb_model *md, const float *X, const float *T, int B,
                                double *loss_dev, cudaStream_t s)
{
    NB_TRY(model_forward(md, X, B, s));
    const int64_t ny = (int64_t)B * md->d;
    const int g = 256;
    k_mse<<<g, 256, 0, s>>>(ny, md->Y, T, 1.0f / (float)ny, md->dY, md->lpart);
    NB_CUDA(cudaGetLastError());
    if (loss_dev) NB_TRY(sum_partials_dev(md->lpart, g, loss_dev, s));
    float *gW = md->grad, *ga = gW + (size_t)md->d * md->h;
    GemmArgs a = {};  // G = dY W   (B x h)
    a.M = B; a.N = md->h; a.K = md->d;
    a.A = md->dY; a.lda = md->d; a.B = md->W; a.ldb = md->h; a.C = md->dH; a.ldc = md->h;
    NB_TRY((gemm<false, false, EPI_STORE>(a, s)));
    const int nb_ = std::min(kBackBlocks, B);
    k_tied_back<<<nb_, 128, 0, s>>>(B, md->h, md->Z, md->a, md->dH, md->gpart);
    k_colsum<<<(md->h + 127) / 128, 128, 0, s>>>(nb_, md->h, md->gpart, ga);
    NB_CUDA(cudaGetLastError());
    GemmArgs c = {};  // gW = X^T dZ   (d x h): the input use of W
    c.M = md->d; c.N = md->h; c.K = B;
    c.A = X; c.lda = md->d; c.B = md->dH; c.ldb = md->h; c.C = gW; c.ldc = md->h;
    NB_TRY((gemm<true, false, EPI_STORE>(c, s)));
    GemmArgs e = {};  // gW += dY^T H  (d x h): the output use of W
    e.M = md->d; e.N = md->h; e.K = B;
    e.A = md->dY; e.lda = md->d; e.B = md->H; e.ldb = md->h; e.C = gW; e.ldc = md->h;
    return gemm<true, false, EPI_ADD>(e, s);
}

// z = |dinv| r + M_int(|r_e| y(r_e/|r_e|)): the preconditioner.
static nb_status model_apply(nb_mesh *m, nb_model *md, const float *r, float *z, cudaStream_t s)
{
    const int E = (int)m->E;
    NB_TRY(model_scratch(md, E));
    k_rownorm<float><<<std::min(E, m->ctx->sm_count * 8), 256, 0, s>>>(E, md->d, r, md->X, md->nrm);
    NB_CUDA(cudaGetLastError());
    GemmArgs a = {};
    a.M = E; a.N = md->h; a.K = md->d;
    a.A = md->X; a.lda = md->d; a.B = md->W; a.ldb = md->h;
    a.C = nullptr; a.ldc = md->h; a.gain = md->a; a.C2 = md->H;
    NB_TRY((gemm<false, false, EPI_GELU_GAIN>(a, s)));
    GemmArgs b = {};
    b.M = E; b.N = md->d; b.K = md->h;
    b.A = md->H; b.lda = md->h; b.B = md->W; b.ldb = md->h;
    b.C = z; b.ldc = md->d; b.rowscale = md->nrm;
    b.rvec = r; b.dinv = m->dinv32; b.n = m->n;
    // interior nodes have one copy and Jacobi is continuous: no summation needed
    return gemm<false, true, EPI_PRECOND>(b, s);
}

// ---------------------------------------------------------------------------
// fused preconditioner for the flexible CG: z, (z, w_prev), (r, z) in one pass
// ---------------------------------------------------------------------------
//
// Both products of the network run on the fifth-generation tensor cores
// (tcgen05.mma, BF16 operands in shared memory, FP32 accumulators in tensor
// memory), transposed so that the weights are the M side and a tile of up to
// 32 elements the N side:
//     H^T (h x NT)  = W^T (h x d) X^T (d x NT)      A = W^T: MN-major view of W
//     C^T (d x NT)  = W   (d x h) Hs^T (h x NT)     A = W chunks of 128 rows, K-major
// with X = r_e / |r_e| in BF16 and Hs = a * gelu(H) in BF16.  One resident
// copy of W serves both products: its image in shared memory is the core
// matrices of W (8 nodes x 8 hidden units each, units contiguous), stored
// unit-group-major, so that for the first product LBO (along K = nodes) is
// 128 bytes and SBO (along M = units) is 16 dp bytes, and for the second LBO
// (along K = units) is 16 dp bytes and SBO (along M = nodes) 128 bytes.
// The first product reads 128 rows of W^T; rows beyond h fall on the
// buffers after the image (their outputs are never read).
//
// One persistent CTA per SM (16 warps) takes a balanced contiguous range of
// elements in tiles of up to 32.  All of a tile's HBM reads are requested at
// its start: its residual rows by bulk copies into shared memory (rows padded
// by 16 bytes, so that the column reads below spread over the banks), its
// dinv and w_prev rows by bulk prefetches into L2.  Then:
//   1. row norms from shared memory (a warp per element), and X = r / |r| in
//      BF16 written in the order of the core-matrix image (each thread 4
//      nodes of one element; a warp's stores are contiguous);
//   2. one thread issues the first product, the tensor core signals an
//      mbarrier; warps read H^T out of tensor memory (thread = hidden unit),
//      apply the gain and GELU, and write Hs;
//   3. one thread issues the second product; each warp then reads 32 nodes x
//      all tile elements of C^T (thread = node), and for each element forms
//      z = |dinv| r + |r_e| C on interior nodes (Jacobi elsewhere), stores z
//      (32 consecutive nodes per warp: coalesced) and accumulates (z, w_prev)
//      over every copy and (r, z) over owner copies.
// The last block forms the flexible-CG beta = -(z, w_prev) / pap_prev (0 on
// the first step) and rtz = (r, z); since r_k is orthogonal to p_(k-1),
// (r, p) = (r, z) and the operator's last block forms alpha = rtz / pap.
// Every wait is bounded (one second): on a timeout the kernel records an
// error, stops the solve, waits (bounded) for its own copies and products,
// frees its tensor memory and returns.

constexpr int kLpcThreads = 512;
constexpr int kLpcTile = 32;       // elements per tile: the N of both products
constexpr int kLpcTmemCols = 256;  // H^T: 32 columns; C^T: 32 per 128-node chunk

__host__ __device__ constexpr int lpc_dk(int d) { return (d + 15) / 16 * 16; }     // K of product 1
__host__ __device__ constexpr int lpc_dp(int d) { return (d + 127) / 128 * 128; }  // M of product 2
__host__ __device__ constexpr int lpc_hp(int h) { return (h + 15) / 16 * 16; }
__host__ __device__ constexpr int lpc_rs(int d) { return 4 * d + 16; }  // bytes per staged row

// Dynamic shared memory: the W image, the X tile, the Hs tile, the staged
// residual rows, at least the 128 rows of W^T that the first product reads,
// plus alignment slack.
static size_t lpc_smem(int d, int h)
{
    const size_t img = 2 * (size_t)lpc_hp(h) * lpc_dp(d);
    const size_t used = img + 2 * (size_t)kLpcTile * lpc_dk(d) +
                        2 * (size_t)kLpcTile * lpc_hp(h) + (size_t)kLpcTile * lpc_rs(d);
    const size_t wt_span = 2 * (size_t)128 * lpc_dp(d);
    return std::max(used, wt_span) + 1024;
}

static bool lpc_fits(int d, int h)
{
    return d % 4 == 0 && d <= 512 && h >= 1 && h <= 128 && lpc_smem(d, h) <= 227 * 1024;
}

// The shared-memory image of W (d x h, FP32, row-major) in BF16: core matrix
// (node group g, unit group c) at element offset (c dp/8 + g) 64, rows of 8
// units; zero beyond d and h.
__global__ void k_w_image(int d, int h, const float *__restrict__ W,
                          __nv_bfloat16 *__restrict__ img)
{
    const int dp = lpc_dp(d), hp = lpc_hp(h);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < dp * hp;
         i += gridDim.x * blockDim.x) {
        const int q = i / hp, u = i - q * hp;  // node, unit
        const float v = q < d && u < h ? W[(size_t)q * h + u] : 0.f;
        img[((u >> 3) * (dp >> 3) + (q >> 3)) * 64 + (q & 7) * 8 + (u & 7)] =
            __float2bfloat16_rn(v);
    }
}

template <int n>
__global__ void __launch_bounds__(kLpcThreads, 1)
k_lpc_tc(int E, int h, const float *__restrict__ r, const float *__restrict__ dinv,
         const float *__restrict__ wold, float *__restrict__ z,
         const __nv_bfloat16 *__restrict__ Wimg, const float *__restrict__ gain, CgScalars *sc,
         double *__restrict__ part, int *err)
{
    constexpr int d = n * n * n, dk = lpc_dk(d), dp = lpc_dp(d), NT = kLpcTile, NQ = dp / 128;
    constexpr int RS = lpc_rs(d) / 4;  // staged row stride in floats
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int hp = lpc_hp(h);
    __nv_bfloat16 *Ws = reinterpret_cast<__nv_bfloat16 *>(sm);  // W image (hp x dp)
    __nv_bfloat16 *Xs = Ws + (size_t)hp * dp;                    // [NT][dk] K-major
    __nv_bfloat16 *Hs = Xs + (size_t)NT * dk;                    // [NT][hp] K-major
    float *Rs = reinterpret_cast<float *>(Hs + (size_t)NT * hp); // [NT][RS] residual rows
    __shared__ __align__(8) uint64_t bar[4];  // W image, product 1, product 2, residual rows
    __shared__ uint32_t tslot;
    __shared__ float snrm[NT], sinv[NT];
    __shared__ double sred[32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int e_beg = (int)((int64_t)E * blockIdx.x / gridDim.x);
    const int e_end = (int)((int64_t)E * (blockIdx.x + 1) / gridDim.x);
    const uint32_t img_bytes = 2u * (uint32_t)hp * dp;
    // a tile's residual rows into Rs (bar[3]): warp 0, one row per lane after
    // lane 0 has announced the bytes
    auto request = [&](int t0, int cnt) {
        if (lane == 0) mbar_expect_tx(&bar[3], (uint32_t)(4 * d * cnt));
        __syncwarp();
        for (int e = lane; e < cnt; e += 32)
            bulk_g2s(Rs + (size_t)e * RS, r + (size_t)(t0 + e) * d, 4u * d, &bar[3]);
    };
    // prologue (weights, barriers, tensor memory: nothing the previous kernel
    // writes), then the wait for it (programmatic dependent launch)
    if (warp == 0) {
        if (lane == 0) {
            for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1);
            mbar_init_fence();
        }
        __syncwarp();
        if (lane == 0) mbar_expect_tx(&bar[0], img_bytes);
        __syncwarp();
        for (uint32_t o = 16384u * lane; o < img_bytes; o += 16384u * 32)
            bulk_g2s(reinterpret_cast<unsigned char *>(Ws) + o,
                     reinterpret_cast<const unsigned char *>(Wimg) + o,
                     img_bytes - o < 16384u ? img_bytes - o : 16384u, &bar[0]);
    }
    if (warp == 1) tc::tmem_alloc(&tslot, kLpcTmemCols);
    // thread roles in tensor memory: lanes 32 (warp % 4) + lane
    const int sp = warp & 3, grp = warp >> 2;
    const uint32_t lane_base = (uint32_t)(32 * sp) << 16;
    const int unit = 32 * sp + lane;  // hidden unit of the GELU pass
    const float gu = unit < h ? gain[unit] : 0.f;
    // epilogue node of this thread (chunk grp of 128 nodes)
    const int q = 128 * grp + 32 * sp + lane;
    const bool q_in = grp < NQ && q < d;
    bool inside = false;
    if (q_in) {
        const int i = q % n, j = (q / n) % n, k = q / (n * n);
        inside = i > 0 && i < n - 1 && j > 0 && j < n - 1 && k > 0 && k < n - 1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    pdl_wait();
    __shared__ int sdone;
    if (tid == 0) sdone = sc->done;  // one reading for the whole block
    __syncthreads();
    if (sdone) {  // the solve has stopped: let the weight copy land, free, leave
        if (tid == 0) mbar_wait_bounded(&bar[0], 0);
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 1) tc::tmem_dealloc(tmem, kLpcTmemCols);
        return;
    }
    if (warp == 0 && e_beg < e_end) request(e_beg, min(NT, e_end - e_beg));
    const uint32_t ws_a = smem_u32(Ws), xs_a = smem_u32(Xs), hs_a = smem_u32(Hs);
    constexpr uint32_t id1 = tc::idesc_bf16(128, NT, true, false);
    constexpr uint32_t id2 = tc::idesc_bf16(128, NT, false, false);
    DotAcc<float> zw, rz;
    bool bad = false;
    int it = 0;
    for (int t0 = e_beg; t0 < e_end; t0 += NT, ++it) {
        const int cnt = min(NT, e_end - t0);
        const uint32_t ph = (uint32_t)(it & 1);
        if (__syncthreads_or(warp == 0 && !mbar_wait_bounded(&bar[3], ph))) {
            bad = true;
            break;
        }
        // 1. row norms (warp per element; zero beyond the tile's elements)
        {
            constexpr int NW = kLpcThreads / 32, R4 = (d / 4 + 31) / 32;
            float ss[NT / NW];
#pragma unroll
            for (int m = 0; m < NT / NW; ++m) {
                const int e = warp + m * NW;
                ss[m] = 0.f;
#pragma unroll
                for (int u = 0; u < R4; ++u) {
                    const int c = lane + 32 * u;
                    if (e < cnt && c < d / 4) {
                        const float4 v =
                            *reinterpret_cast<const float4 *>(Rs + (size_t)e * RS + 4 * c);
                        ss[m] += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < NT / NW; ++m) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) ss[m] += __shfl_xor_sync(0xffffffffu, ss[m], o);
                if (lane == 0) {
                    const int e = warp + m * NW;
                    const float nv = sqrtf(ss[m]);
                    snrm[e] = nv;
                    sinv[e] = nv > 0.f ? 1.0f / nv : 0.f;
                }
            }
        }
        __syncthreads();
        //    X in BF16: chunk i = 4 nodes of one element, at element offset 4 i
        //    of the image (core c = i / 16: element group c / (dk/8), node
        //    group c % (dk/8); row (i % 16) / 2, half i % 2)
#pragma unroll
        for (int i = tid; i < NT * dk / 4; i += kLpcThreads) {
            const int c = i >> 4, rr = (i & 15) >> 1;
            const int e = (c / (dk / 8)) * 8 + rr;
            const int k = (c % (dk / 8)) * 8 + (i & 1) * 4;
            uint2 pk = make_uint2(0u, 0u);
            if (e < cnt && k < d) {
                const float4 v = *reinterpret_cast<const float4 *>(Rs + (size_t)e * RS + k);
                const float inv = sinv[e];
                __nv_bfloat162 lo = __floats2bfloat162_rn(v.x * inv, v.y * inv);
                __nv_bfloat162 hi = __floats2bfloat162_rn(v.z * inv, v.w * inv);
                pk.x = *reinterpret_cast<uint32_t *>(&lo);
                pk.y = *reinterpret_cast<uint32_t *>(&hi);
            }
            *reinterpret_cast<uint2 *>(Xs + 4 * (size_t)i) = pk;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        // 2. H^T = W^T X^T (tensor memory columns [0, NT))
        if (tid == 0) {
            bool ok = true;
            if (it == 0) ok = mbar_wait_bounded(&bar[0], 0);
            if (ok) {
                tc::fence_after_sync();
#pragma unroll 1
                for (int ks = 0; ks < dk / 16; ++ks)
                    tc::mma_bf16(tmem, tc::sdesc(ws_a + 256u * ks, 128u, 16u * dp),
                                 tc::sdesc(xs_a + 256u * ks, 128u, 16u * dk), id1, ks > 0);
                tc::commit(&bar[1]);
            } else {
                atomicExch(err, 1);
            }
        }
        if (__syncthreads_or(warp == 0 && !mbar_wait_bounded(&bar[1], ph))) {
            bad = true;
            break;
        }
        tc::fence_after_sync();
        // Hs = a * gelu(H): thread = hidden unit, elements 8 grp .. 8 grp + 7
        {
            float hv[8];
            tc::ld_x8(tmem + lane_base + 8u * grp, hv);
            tc::wait_ld();
            if (unit < hp) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int e = 8 * grp + j;
                    const float val = unit < h ? gu * gelu_f(hv[j]) : 0.f;
                    Hs[tc::kmajor_off(e, unit, hp / 8)] = __float2bfloat16_rn(val);
                }
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        // 3. C^T = W Hs^T, chunk mq of 128 nodes into columns NT (1 + mq)
        if (tid == 0) {
#pragma unroll 1
            for (int mq = 0; mq < NQ; ++mq)
#pragma unroll 1
                for (int ks = 0; ks < hp / 16; ++ks)
                    tc::mma_bf16(tmem + (uint32_t)(NT * (1 + mq)),
                                 tc::sdesc(ws_a + 2u * ks * 16u * dp + 2048u * mq, 16u * dp, 128u),
                                 tc::sdesc(hs_a + 256u * ks, 128u, 16u * hp), id2, ks > 0);
            tc::commit(&bar[2]);
        }
        // the epilogue's dinv and w_prev of this thread's node for the whole
        // tile, in flight while the product runs
        float dv[NT], wv[NT];
        if (q_in) {
#pragma unroll
            for (int j = 0; j < NT; ++j)
                if (j < cnt) {
                    const size_t o = (size_t)(t0 + j) * d + q;
                    dv[j] = dinv[o];
                    wv[j] = wold[o];
                }
        }
        if (__syncthreads_or(warp == 0 && !mbar_wait_bounded(&bar[2], ph))) {
            bad = true;
            break;
        }
        tc::fence_after_sync();
        if (grp < NQ) {  // warp-uniform: the loads below are warp-collective
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float c[NT / 2];
                tc::ld_x16(tmem + lane_base + (uint32_t)(NT * (1 + grp) + half * (NT / 2)), c);
                tc::wait_ld();
                if (q_in) {
                    // two elements per compensated addition: their products
                    // summed in FP32 first
#pragma unroll
                    for (int j = 0; j < NT / 2; j += 2) {
                        float tzw = 0.f, trz = 0.f;
#pragma unroll
                        for (int jj = 0; jj < 2; ++jj) {
                            const int e = half * (NT / 2) + j + jj;
                            if (e < cnt) {
                                const float rv = Rs[(size_t)e * RS + q];
                                float zv = fabsf(dv[e]) * rv;
                                if (inside) zv += c[j + jj] * snrm[e];
                                z[(size_t)(t0 + e) * d + q] = zv;
                                tzw = fmaf(zv, wv[e], tzw);
                                if (!signbit(dv[e])) trz = fmaf(rv, zv, trz);
                            }
                        }
                        zw.add(tzw);
                        rz.add(trz);
                    }
                }
            }
        }
        // the tile's buffers and tensor memory are free again; the next
        // tile's residual rows may land in Rs
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (warp == 0 && t0 + NT < e_end) request(t0 + NT, min(NT, e_end - t0 - NT));
    }
    if (sc->pdl_early) pdl_trigger();
    if (bad) {
        // a copy or a product never completed: record it, stop the solve, let
        // what is in flight land, free the tensor memory
        if (tid == 0) {
            atomicExch(err, 1);
            sc->status = NB_BREAKDOWN;
            sc->done = 1;
            mbar_wait_bounded(&bar[0], 0);
            mbar_wait_bounded(&bar[1], (uint32_t)(it & 1));
            mbar_wait_bounded(&bar[2], (uint32_t)(it & 1));
            mbar_wait_bounded(&bar[3], (uint32_t)(it & 1));
        }
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 1) tc::tmem_dealloc(tmem, kLpcTmemCols);
        return;
    }
    if (e_beg >= e_end && tid == 0) mbar_wait_bounded(&bar[0], 0);  // no tile: the copy lands
    const double tzw = block_sum_acc(zw, sred);
    const double trz = block_sum_acc(rz, sred);
    if (tid == 0) {
        part[blockIdx.x] = tzw;
        part[gridDim.x + blockIdx.x] = trz;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, kLpcTmemCols);
    if (last_block(&sc->tick_upd)) {
        double szw, srz;
        sum_partials2(part, part + gridDim.x, gridDim.x, sred, szw, srz);
        if (tid == 0) {
            sc->beta = sc->pap_prev > 0.0 ? -szw / sc->pap_prev : 0.0;  // 0: first step
            sc->fcg_zw = szw;
            sc->rtz = srz;
            sc->rp = srz;
            if (!isfinite(sc->beta) || !isfinite(srz)) {
                sc->done = 1;
                sc->status = NB_BREAKDOWN;
            }
        }
    }
}

// The block's partial of (r, c, r); the last block: pap_prev, rtr, the
// iteration count, the relative residual (history) and the stopping tests.
__device__ __forceinline__ void fcg_step_finish(CgScalars *sc, const DotAcc<float> &mine,
                                                double *part, double *sred)
{
    const double t = block_sum_acc(mine, sred);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    if (!last_block(&sc->tick_upd)) return;
    const double rtr = sum_partials(part, gridDim.x, sred);
    if (threadIdx.x == 0) {
        sc->pap_prev = sc->pap;
        sc->rtr = rtr;
        const int it = sc->iter + 1;
        sc->iter = it;
        const double bn = sc->bnorm2 > 0.0 ? sc->bnorm2 : 1.0;
        const double rel = sqrt(rtr / bn);
        sc->relres = rel;
        if (sc->hist && it <= sc->hist_cap) sc->hist[it - 1] = rel;
        if (!isfinite(rel)) {
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

// The flexible-CG update with the direct-stiffness summation of w folded in
// (FP32, even n, two nodes of a row per thread, gs_sum_pair): w_asm = mask *
// sum of w over the node's copies, x += alpha p, r -= alpha w_asm, the
// partial of (r, c, r), and with SCATTER the owner values of the new r into
// rg (the Schwarz preconditioner's global vector).  w stays unassembled, so
// the preconditioner kernels form (z, w_prev) over every copy (z continuous).
template <int n, bool SCATTER>
__global__ void __launch_bounds__(256)
k_fcg_update_gs2(int64_t E, int nx, int ny, int nz, CgScalars *sc, float *__restrict__ x,
                 float *__restrict__ r, const float *__restrict__ p, const float *__restrict__ w,
                 const float *__restrict__ sgn, double *__restrict__ part,
                 float *__restrict__ rg, const int32_t *__restrict__ gid)
{
    static_assert(n % 2 == 0, "pairs of nodes need an even n");
    constexpr int N = n - 1, n2 = n * n, n3 = n2 * n, h = n / 2, P = n3 / 2;
    __shared__ double sred[32];
    pdl_wait();  // the previous kernel's alpha, w and p (programmatic dependent launch)
    if (sc->done) return;
    const float alpha = (float)sc->alpha;
    const int64_t sx = n3 - N, sy = (int64_t)nx * n3 - N * n, sz = (int64_t)nx * ny * n3 - N * n2;
    DotAcc<float> acc;
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
        for (int t = threadIdx.x; t < P; t += blockDim.x) {
            const int i0 = 2 * (t % h), j = (t / h) % n, k = t / (h * n);
            const int64_t l = e * n3 + (int64_t)k * n2 + j * n + i0;
            float wa, wb;
            gs_sum_pair<float, n>(w, l, i0, j, k, ex, ey, ez, nx, ny, nz, sx, sy, sz, wa, wb);
            float2 xv = *reinterpret_cast<float2 *>(x + l), rv = *reinterpret_cast<float2 *>(r + l);
            const float2 pv = *reinterpret_cast<const float2 *>(p + l);
            const float2 dv = *reinterpret_cast<const float2 *>(sgn + l);
            if (dv.x == 0.f) wa = 0.f;  // Dirichlet node
            if (dv.y == 0.f) wb = 0.f;
            xv.x += alpha * pv.x;
            xv.y += alpha * pv.y;
            rv.x -= alpha * wa;
            rv.y -= alpha * wb;
            if (!signbit(dv.x)) {
                acc.add(rv.x * rv.x);
                if (SCATTER) rg[gid[l]] = rv.x;
            }
            if (!signbit(dv.y)) {
                acc.add(rv.y * rv.y);
                if (SCATTER) rg[gid[l + 1]] = rv.y;
            }
            *reinterpret_cast<float2 *>(x + l) = xv;
            *reinterpret_cast<float2 *>(r + l) = rv;
        }
    }
    if (sc->pdl_early) pdl_trigger();
    fcg_step_finish(sc, acc, part, sred);
}

// k_fcg_update_gs2 for the mesh's order (even n <= 16; the flexible-CG paths
// that use it need an even n).
bool launch_fcg_update_el(nb_mesh *m, Workspace &ws, float *x, float *r, const float *p,
                          const float *w, double *part, float *rg, cudaStream_t s);

static nb_status fcg_update_folded(nb_mesh *m, Workspace &ws, float *x, float *r, const float *p,
                                   const float *w, double *part, float *rg, cudaStream_t s)
{
    // element ranges where built (even n <= 10), else one block per element
    if (launch_fcg_update_el(m, ws, x, r, p, w, part, rg, s)) {
        NB_CUDA(cudaGetLastError());
        return NB_OK;
    }
    const int grid = (int)std::min<int64_t>(m->E, (int64_t)m->ctx->sm_count * 8);
    const float *sgn = m->dinv32;
#define NB_FU(NN)                                                                                 \
    case NN:                                                                                      \
        if (rg)                                                                                   \
            k_fcg_update_gs2<NN, true><<<grid, 256, 0, s>>>(m->E, m->nx, m->ny, m->nz, ws.scal,   \
                                                            x, r, p, w, sgn, part, rg, m->gid);   \
        else                                                                                      \
            NB_CUDA(launch_pdl(k_fcg_update_gs2<NN, false>, grid, 256, 0, s, m->E, m->nx, m->ny,  \
                               m->nz, ws.scal, x, r, p, w, sgn, part, (float *)nullptr,           \
                               (const int32_t *)nullptr));                                        \
        break;
    switch (m->n) {
        NB_FU(2) NB_FU(4) NB_FU(6) NB_FU(8) NB_FU(10) NB_FU(12) NB_FU(14) NB_FU(16)
        default:
            set_error("flexible-CG update: n=%d not built (even n <= 16)", m->n);
            return NB_ERR_ARG;
    }
#undef NB_FU
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// k_lpc_tc for the orders it is built for (d = n^3 <= 512, n even).
static bool lpc_order(int n) { return n == 2 || n == 4 || n == 6 || n == 8; }

static nb_status lpc_attr(int n, size_t smem)
{
    switch (n) {
        case 2: NB_CUDA(cudaFuncSetAttribute(k_lpc_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); break;
        case 4: NB_CUDA(cudaFuncSetAttribute(k_lpc_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); break;
        case 6: NB_CUDA(cudaFuncSetAttribute(k_lpc_tc<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); break;
        case 8: NB_CUDA(cudaFuncSetAttribute(k_lpc_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); break;
        default: set_error("fused preconditioner unavailable for n=%d", n); return NB_ERR_ARG;
    }
    return NB_OK;
}

static nb_status launch_lpc(int n, int grid, size_t smem, cudaStream_t s, int E, int h,
                            const float *r, const float *dinv, const float *wold, float *z,
                            const __nv_bfloat16 *Wimg, const float *gain, CgScalars *sc,
                            double *part, int *err)
{
#define NB_LPC(NN)                                                                           \
    NB_CUDA(launch_pdl(k_lpc_tc<NN>, grid, kLpcThreads, smem, s, E, h, r, dinv, wold, z, Wimg, \
                       gain, sc, part, err))
    switch (n) {
        case 2: NB_LPC(2); break;
        case 4: NB_LPC(4); break;
        case 6: NB_LPC(6); break;
        case 8: NB_LPC(8); break;
        default: set_error("fused preconditioner unavailable for n=%d", n); return NB_ERR_ARG;
    }
#undef NB_LPC
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// The BF16 shared-memory image of W for k_lpc_tc, rebuilt when the weights
// changed (training step).
static nb_status ensure_wimg(nb_model *md, cudaStream_t s)
{
    const size_t bytes = sizeof(__nv_bfloat16) * (size_t)lpc_hp(md->h) * lpc_dp(md->d);
    if (!md->Wimg) NB_CUDA(cudaMalloc(&md->Wimg, bytes));
    if (md->wimg_step != md->step || md->wimg_step < 0) {
        k_w_image<<<64, 256, 0, s>>>(md->d, md->h, md->W, md->Wimg);
        NB_CUDA(cudaGetLastError());
        md->wimg_step = md->step;
    }
    return NB_OK;
}

// ---------------------------------------------------------------------------
// flexible CG (inner solve of the refinement) with the learned preconditioner
// ---------------------------------------------------------------------------

// Owner-copy dot product partials of (a, b) (continuous vectors).
__global__ void k_fdot(int64_t n, const float *__restrict__ a, const float *__restrict__ b,
                       const float *__restrict__ sgn, double *__restrict__ part)
{
    __shared__ double sred[32];
    DotAcc<float> acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!signbit(sgn[i])) acc.add(a[i] * b[i]);
    const double t = block_sum_acc(acc, sred);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// p = z + beta p with beta = -(z, w_prev) / pap_prev (0 on the first step),
// then partials of (r, p).  beta is formed by the first block from the
// partials of (z, w_prev) in part_zw (read-only here).
__global__ void k_fcg_p(int64_t n, CgScalars *sc, const double *__restrict__ part_zw, int cnt,
                        const float *__restrict__ z, const float *__restrict__ r,
                        float *__restrict__ p, const float *__restrict__ sgn,
                        double *__restrict__ part)
{
    __shared__ double sred[32];
    __shared__ float sbeta;
    if (sc->done) return;
    const double zw = sum_partials(part_zw, cnt, sred);
    if (threadIdx.x == 0) sbeta = sc->pap_prev > 0.0 ? (float)(-zw / sc->pap_prev) : 0.f;
    __syncthreads();
    const float beta = sbeta;
    DotAcc<float> acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float pv = z[i] + beta * p[i];
        p[i] = pv;
        if (!signbit(sgn[i])) acc.add(r[i] * pv);
    }
    const double t = block_sum_acc(acc, sred);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// alpha = (r, p) / (p, A p); x += alpha p; r -= alpha w; partials of (r, r).
__global__ void k_fcg_update(int64_t n, CgScalars *sc, const double *__restrict__ part_rp,
                             const double *__restrict__ part_pap, int cnt_rp, int cnt_pap,
                             float *__restrict__ x, float *__restrict__ r,
                             const float *__restrict__ p, const float *__restrict__ w,
                             const float *__restrict__ sgn, double *__restrict__ part)
{
    __shared__ double sred[32];
    __shared__ float salpha;
    __shared__ int sbad;
    if (sc->done) return;
    const double rp = sum_partials(part_rp, cnt_rp, sred);
    const double pap = sum_partials(part_pap, cnt_pap, sred);
    if (threadIdx.x == 0) {
        const double a = rp / pap;
        sbad = !(pap > 0.0) || !isfinite(a);
        salpha = sbad ? 0.f : (float)a;
        if (blockIdx.x == 0) {
            sc->pap = pap;
            sc->alpha = a;
            sc->rp = rp;
        }
    }
    __syncthreads();
    if (sbad) return;  // uniform; the finish kernel records the breakdown
    const float alpha = salpha;
    DotAcc<float> acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        const float rv = r[i] - alpha * w[i];
        r[i] = rv;
        if (!signbit(sgn[i])) acc.add(rv * rv);
    }
    const double t = block_sum_acc(acc, sred);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_fcg_finish(CgScalars *sc, const double *__restrict__ part, int cnt)
{
    __shared__ double sred[32];
    if (sc->done) return;
    const double rtr = sum_partials(part, cnt, sred);
    if (threadIdx.x == 0) {
        if (!(sc->pap > 0.0) || !isfinite(sc->alpha)) {
            sc->done = 1;
            sc->status = NB_BREAKDOWN;
            return;
        }
        sc->pap_prev = sc->pap;
        sc->rtr = rtr;
        const int it = sc->iter + 1;
        sc->iter = it;
        const double bn = sc->bnorm2 > 0.0 ? sc->bnorm2 : 1.0;
        const double rel = sqrt(rtr / bn);
        sc->relres = rel;
        if (sc->hist && it <= sc->hist_cap) sc->hist[it - 1] = rel;
        if (!isfinite(rel)) {
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

// While-node condition of the captured flexible CG (two steps per body): stop
// when the scalars say so, and in any case after maxit / 2 + 1 bodies.
__global__ void k_fcg_cond(CgScalars *sc, cudaGraphConditionalHandle h)
{
    const int loops = sc->loops + 1;
    sc->loops = loops;
    const bool stop = sc->done != 0 || 2 * loops > sc->maxit + 2;
    cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// keep: the iteration resumes after a residual replacement with its previous
// direction (pap_prev, p and w_prev kept; the flexible-CG beta
// -(z, A p_prev) / (p_prev, A p_prev) does not depend on the scale of p_prev,
// so nothing is rescaled); otherwise pap_prev = 0 makes the first beta 0.
__global__ void k_fcg_init(CgScalars *sc, const double *__restrict__ part, int cnt, int keep)
{
    __shared__ double sred[32];
    const double rtr = sum_partials(part, cnt, sred);
    if (threadIdx.x == 0) {
        sc->rtr = rtr;
        sc->bnorm2 = rtr;
        sc->relres = rtr > 0.0 ? 1.0 : 0.0;
        if (!keep) sc->pap_prev = 0.0;
        if (!isfinite(rtr)) {
            sc->done = 1;
            sc->status = NB_BREAKDOWN;
        } else if (rtr == 0.0 || sc->maxit <= 0) {
            sc->done = 1;
            if (rtr != 0.0) sc->status = NB_NOT_CONVERGED;
        }
    }
}

bool ax_dir_step_available(const nb_mesh *m);
nb_status ax_dir_step(nb_mesh *m, const float *z, float *p, float *w, CgScalars *scal,
                      double *pap_part, int *nparts, cudaStream_t s);

// Direction state at the start of an inner flexible-CG solve.  Fresh: p = 0,
// w_prev = 0.  Kept (reliable update): p and the last A p stay; a step writes
// A p into ws.w on odd and ws.aux on even step numbers and reads w_prev from
// the other buffer, and every solve starts with an odd step, so after an odd
// number of steps the last A p is copied from ws.w into ws.aux.
static nb_status fcg_prepare(nb_mesh *m, Workspace &ws, bool keep, bool odd, cudaStream_t s)
{
    const size_t bytes = sizeof(float) * m->nL;
    if (!keep) {
        NB_CUDA(cudaMemsetAsync(ws.p, 0, bytes, s));
        NB_CUDA(cudaMemsetAsync(ws.aux, 0, bytes, s));
    } else if (odd) {
        NB_CUDA(cudaMemcpyAsync(ws.aux, ws.w, bytes, cudaMemcpyDeviceToDevice, s));
    }
    return NB_OK;
}

// The inner solve of a refinement step: ws.r holds the scaled residual, ws.x
// starts at zero.  One flexible-CG step is three kernels when the fused forms
// apply (k_lpc_tc; the operator's direction form with alpha; k_fcg_update_gs2
// with the summation folded in), otherwise the general path below.  Captured in a graph
// with a while node (two steps per body), or host-launched with the stopping
// state checked every few steps (all kernels skip their work once it is set).
nb_status fcg_learned(nb_mesh *m, nb_prec prec, Workspace &ws, const nb_opts *o, bool keep,
                      bool odd, cudaStream_t s)
{
    (void)o;
    nb_model *md = (nb_model *)m->learned;
    if (!md) {
        set_error("no learned preconditioner attached");
        return NB_ERR_STATE;
    }
    const int g = vec_grid(m->ctx, m->nL);
    const float *sgn = m->dinv32;
    float *x = (float *)ws.x, *r = (float *)ws.r, *p = (float *)ws.p, *w = (float *)ws.w;
    float *z = (float *)ws.z, *wprev = (float *)ws.aux;
    double *P0 = ws.part, *P1 = ws.part + kMaxPartials, *P2 = ws.part + 2 * kMaxPartials;
    NB_TRY(model_scratch(md, (int)m->E));  // before any capture: it may allocate
    const bool fast = prec == NB_FP32 && ax_dir_step_available(m) && lpc_order(m->n) &&
                      lpc_fits(md->d, md->h);
    const size_t lsm = lpc_smem(md->d, md->h);
    const int lgrid = std::max(1, (int)std::min<int64_t>(m->E, m->ctx->sm_count));
    if (fast) {
        NB_TRY(ensure_wimg(md, s));  // outside any capture: refreshed in place when W changed
        NB_TRY(lpc_attr(m->n, lsm));
    }
    keep = keep && fast;
    NB_TRY(fcg_prepare(m, ws, keep, odd, s));
    k_fdot<<<g, kVecThreads, 0, s>>>(m->nL, r, r, sgn, P2);
    k_fcg_init<<<1, kFinalizeThreads, 0, s>>>(ws.scal, P2, g, keep ? 1 : 0);
    NB_CUDA(cudaGetLastError());
    m->launches += 2;
    // one flexible-CG step; w receives A p, wprev holds the previous A p
    auto step = [&](float *wcur, float *wold) -> nb_status {
        if (fast) {
            PdlScope pdl(true);  // the three kernels wait for their predecessor themselves
            NB_TRY(launch_lpc(m->n, lgrid, lsm, s, (int)m->E, md->h, r, sgn, wold, z, md->Wimg,
                              md->a, ws.scal, P0, m->kerr));
            int nparts = 0;
            NB_TRY(ax_dir_step(m, z, p, wcur, ws.scal, P1, &nparts, s));
            // w stays unassembled: the update folds the summation in, and
            // k_lpc_tc forms (z, w_prev) over every copy
            return fcg_update_folded(m, ws, x, r, p, wcur, P2, nullptr, s);
        }
        NB_TRY(model_apply(m, md, r, z, s));
        k_fdot<<<g, kVecThreads, 0, s>>>(m->nL, z, wold, sgn, P0);
        k_fcg_p<<<g, kVecThreads, 0, s>>>(m->nL, ws.scal, P0, g, z, r, p, sgn, P1);
        NB_CUDA(cudaGetLastError());
        int nparts = 0;
        NB_TRY(ax_local(m, prec, p, wcur, P0, &nparts, s));
        NB_TRY(dssum(m, prec, wcur, 1, s));
        k_fcg_update<<<g, kVecThreads, 0, s>>>(m->nL, ws.scal, P1, P0, g, nparts, x, r, p, wcur,
                                               sgn, P2);
        k_fcg_finish<<<1, kFinalizeThreads, 0, s>>>(ws.scal, P2, g);
        NB_CUDA(cudaGetLastError());
        return NB_OK;
    };
    if (o->use_graph) {
        // the loop body is two steps (the roles of w and wprev swap between
        // them), repeated by a while node until the scalars say stop
        const intptr_t key = (intptr_t)md;
        if (!ws.exec2 || ws.graph2_key != key || ws.graph2_epoch != m->ax_epoch) {
            if (ws.exec2) NB_CUDA(cudaGraphExecDestroy(ws.exec2));
            if (ws.graph2) NB_CUDA(cudaGraphDestroy(ws.graph2));
            ws.exec2 = nullptr;
            ws.graph2 = nullptr;
            cudaGraph_t gr;
            NB_CUDA(cudaGraphCreate(&gr, 0));
            cudaGraphConditionalHandle h;
            NB_CUDA(cudaGraphConditionalHandleCreate(&h, gr, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t node;
            NB_CUDA(cudaGraphAddNode(&node, gr, nullptr, nullptr, 0, &cp));
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            NB_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed));
            nb_status st = step(w, wprev);
            if (st == NB_OK) st = step(wprev, w);
            if (st == NB_OK) {
                k_fcg_cond<<<1, 1, 0, s>>>(ws.scal, h);
                if (cudaGetLastError() != cudaSuccess) st = NB_ERR_CUDA;
            }
            cudaGraph_t captured = nullptr;
            cudaError_t ce = cudaStreamEndCapture(s, &captured);
            if (st != NB_OK || ce != cudaSuccess) {
                cudaGraphDestroy(gr);
                if (st != NB_OK) return st;
                set_error("flexible-CG graph capture failed: %s", cudaGetErrorString(ce));
                return NB_ERR_CUDA;
            }
            NB_CUDA(cudaGraphInstantiate(&ws.exec2, gr, 0));
            ws.graph2 = gr;
            ws.graph2_key = key;
            ws.graph2_epoch = m->ax_epoch;
        }
        NB_CUDA(cudaGraphLaunch(ws.exec2, s));
        NB_CUDA(cudaMemcpyAsync(ws.scal_host, ws.scal, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
        NB_CUDA(cudaStreamSynchronize(s));
        m->launches += (fast ? 7 : 19) * (int64_t)((std::max(ws.scal_host->iter, 1) + 1) / 2);
        return NB_OK;
    }
    for (int it = 0;; ++it) {
        NB_TRY(step(w, wprev));
        std::swap(w, wprev);  // w of this step is w_prev of the next
        // fused: preconditioner, operator, update (summation folded in);
        // general: row norms, 2 products, 2 dots, operator, summation,
        // update, finish
        m->launches += fast ? 3 : 9;
        if ((it & 7) == 7) {
            NB_CUDA(cudaMemcpyAsync(ws.scal_host, ws.scal, sizeof(CgScalars),
                                    cudaMemcpyDeviceToHost, s));
            NB_CUDA(cudaStreamSynchronize(s));
            if (ws.scal_host->done) break;
            if (it > ws.scal_host->maxit + 8) break;  // bounded even if the state is stuck
        }
    }
    // keep ws.w / ws.aux as allocated (the swap only exchanged roles)
    return NB_OK;
}

nb_status schwarz_setup(nb_mesh *m);
nb_status schwarz_gather(nb_mesh *m, const float *r, cudaStream_t s);
nb_status schwarz_solve_sum(nb_mesh *m, const float *r, float *z, const float *wold,
                            CgScalars *sc, double *part, cudaStream_t s, bool coarse);
nb_status schwarz_coarse_setup(nb_mesh *m);
float *schwarz_rg(nb_mesh *m);

// The inner solve of a refinement step with the Schwarz preconditioner (FP32,
// even n): flexible CG -- for this linear, symmetric preconditioner it is
// preconditioned CG up to rounding -- one step being the local solves, their
// sum with the flexible-CG dots (z, w_prev), (r, z) and beta, the operator's
// direction form with alpha, the summation, and the update, which also
// scatters the new residual's owner values for the next local solves.
// Graph-captured like fcg_learned.
nb_status fcg_schwarz(nb_mesh *m, nb_prec prec, Workspace &ws, const nb_opts *o, bool keep,
                      bool odd, cudaStream_t s)
{
    if (prec != NB_FP32 || !ax_dir_step_available(m)) {
        set_error("the Schwarz preconditioner runs in FP32 refinement steps with even n");
        return NB_ERR_ARG;
    }
    const bool two = o->pc == NB_PC_SCHWARZ2;  // with the coarse-grid level
    NB_TRY(schwarz_setup(m));  // before any capture: it allocates once
    if (two) NB_TRY(schwarz_coarse_setup(m));
    const int g = vec_grid(m->ctx, m->nL);
    const float *sgn = m->dinv32;
    float *x = (float *)ws.x, *r = (float *)ws.r, *p = (float *)ws.p, *w = (float *)ws.w;
    float *z = (float *)ws.z, *wprev = (float *)ws.aux;
    double *P0 = ws.part, *P1 = ws.part + kMaxPartials, *P2 = ws.part + 2 * kMaxPartials;
    NB_TRY(fcg_prepare(m, ws, keep, odd, s));
    float *rg = schwarz_rg(m);
    k_fdot<<<g, kVecThreads, 0, s>>>(m->nL, r, r, sgn, P2);
    k_fcg_init<<<1, kFinalizeThreads, 0, s>>>(ws.scal, P2, g, keep ? 1 : 0);
    NB_CUDA(cudaGetLastError());
    NB_TRY(schwarz_gather(m, r, s));
    m->launches += 3;
    auto step = [&](float *wcur, float *wold) -> nb_status {
        NB_TRY(schwarz_solve_sum(m, r, z, wold, ws.scal, P0, s, two));
        int nparts = 0;
        NB_TRY(ax_dir_step(m, z, p, wcur, ws.scal, P1, &nparts, s));
        // w stays unassembled (the update folds the summation in; the sum
        // kernel forms (z, w_prev) over every copy)
        return fcg_update_folded(m, ws, x, r, p, wcur, P2, rg, s);
    };
    // local solves, (coarse restrictions and solve,) their sum, operator, update
    const int kPerStep = two ? 7 : 4;
    if (o->use_graph) {
        const intptr_t key = (intptr_t)m->schwarz + (two ? 1 : 0);
        if (!ws.exec2 || ws.graph2_key != key || ws.graph2_epoch != m->ax_epoch) {
            if (ws.exec2) NB_CUDA(cudaGraphExecDestroy(ws.exec2));
            if (ws.graph2) NB_CUDA(cudaGraphDestroy(ws.graph2));
            ws.exec2 = nullptr;
            ws.graph2 = nullptr;
            cudaGraph_t gr;
            NB_CUDA(cudaGraphCreate(&gr, 0));
            cudaGraphConditionalHandle h;
            NB_CUDA(cudaGraphConditionalHandleCreate(&h, gr, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t node;
            NB_CUDA(cudaGraphAddNode(&node, gr, nullptr, nullptr, 0, &cp));
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            NB_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed));
            nb_status st = step(w, wprev);
            if (st == NB_OK) st = step(wprev, w);
            if (st == NB_OK) {
                k_fcg_cond<<<1, 1, 0, s>>>(ws.scal, h);
                if (cudaGetLastError() != cudaSuccess) st = NB_ERR_CUDA;
            }
            cudaGraph_t captured = nullptr;
            cudaError_t ce = cudaStreamEndCapture(s, &captured);
            if (st != NB_OK || ce != cudaSuccess) {
                cudaGraphDestroy(gr);
                if (st != NB_OK) return st;
                set_error("Schwarz flexible-CG graph capture failed: %s", cudaGetErrorString(ce));
                return NB_ERR_CUDA;
            }
            NB_CUDA(cudaGraphInstantiate(&ws.exec2, gr, 0));
            ws.graph2 = gr;
            ws.graph2_key = key;
            ws.graph2_epoch = m->ax_epoch;
        }
        NB_CUDA(cudaGraphLaunch(ws.exec2, s));
        NB_CUDA(cudaMemcpyAsync(ws.scal_host, ws.scal, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
        NB_CUDA(cudaStreamSynchronize(s));
        m->launches += (2 * kPerStep + 1) * (int64_t)((std::max(ws.scal_host->iter, 1) + 1) / 2);
        return NB_OK;
    }
    for (int it = 0;; ++it) {
        NB_TRY(step(w, wprev));
        std::swap(w, wprev);
        m->launches += kPerStep;
        if ((it & 7) == 7) {
            NB_CUDA(cudaMemcpyAsync(ws.scal_host, ws.scal, sizeof(CgScalars),
                                    cudaMemcpyDeviceToHost, s));
            NB_CUDA(cudaStreamSynchronize(s));
            if (ws.scal_host->done) break;
            if (it > ws.scal_host->maxit + 8) break;  // bounded even if the state is stuck
        }
    }
    return NB_OK;
}

void learned_free(nb_mesh *m) { m->learned = nullptr; }

}  // namespace nb

using namespace nb;

extern "C" nb_status nb_model_create(nb_ctx *ctx, int N, int hidden, uint64_t seed,
                                     nb_model **out)
{
    if (!ctx || !out || N < 1 || N > kMaxN || hidden < 1 || hidden > 4096) {
        set_error("invalid argument: model shape");
        return NB_ERR_ARG;
    }
    *out = nullptr;
    NB_DEVICE_SCOPE(ctx->device);
    nb_model *md = new nb_model();
    md->ctx = ctx;
    ctx_retain(ctx);
    md->N = N;
    md->d = (N + 1) * (N + 1) * (N + 1);
    md->h = hidden;
    const size_t d = md->d, h = md->h;
    md->nparam = (int64_t)(d * h + h);
    // deterministic initialisation: W uniform(-1,1)/sqrt(d) from SplitMix64, a = 1
    std::vector<float> host(md->nparam, 1.f);
    uint64_t st = seed * 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    };
    for (size_t i = 0; i < d * h; ++i) host[i] = (float)(next() / sqrt((double)d));
    cudaError_t e = cudaMalloc(&md->W, sizeof(float) * md->nparam);
    if (e == cudaSuccess) e = cudaMalloc(&md->grad, sizeof(float) * md->nparam);
    if (e == cudaSuccess) e = cudaMalloc(&md->m, sizeof(float) * md->nparam);
    if (e == cudaSuccess) e = cudaMalloc(&md->v, sizeof(float) * md->nparam);
    if (e == cudaSuccess)
        e = cudaMemcpy(md->W, host.data(), sizeof(float) * md->nparam, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(md->m, 0, sizeof(float) * md->nparam);
    if (e == cudaSuccess) e = cudaMemset(md->v, 0, sizeof(float) * md->nparam);
    if (e != cudaSuccess) {
        set_error("model allocation: %s", cudaGetErrorString(e));
        cudaFree(md->W); cudaFree(md->grad); cudaFree(md->m); cudaFree(md->v);
        delete md;
        return NB_ERR_OOM;
    }
    md->a = md->W + d * h;
    *out = md;
    return NB_OK;
}

extern "C" nb_status nb_model_destroy(nb_model *md)
{
    if (!md) return NB_OK;
    ::nb::DeviceGuard nb_device_guard_(md->ctx->device);
    float *bufs[] = {md->W, md->grad, md->m, md->v, md->Z, md->H, md->Y, md->dY, md->dH,
                     md->nrm, md->X, md->gpart};
    for (float *b : bufs) cudaFree(b);
    cudaFree(md->lpart);
    cudaFree(md->Wimg);
    nb_ctx *ctx = md->ctx;
    delete md;
    ctx_release(ctx);
    return NB_OK;
}

extern "C" nb_status nb_model_params(nb_model *md, float *get_host, const float *set_host,
                                     int64_t *nparam)
{
    if (!md) {
        set_error("invalid argument: model is NULL");
        return NB_ERR_ARG;
    }
    NB_DEVICE_SCOPE(md->ctx->device);
    if (nparam) *nparam = md->nparam;
    if (set_host) {
        NB_CUDA(cudaMemcpy(md->W, set_host, sizeof(float) * md->nparam, cudaMemcpyHostToDevice));
        md->wimg_step = -1;  // the BF16 image of the fused preconditioner is stale
    }
    if (get_host)
        NB_CUDA(cudaMemcpy(get_host, md->W, sizeof(float) * md->nparam, cudaMemcpyDeviceToHost));
    return NB_OK;
}

extern "C" nb_status nb_model_grad(nb_model *md, const float *X, const float *T, int B,
                                   double *loss_host, float *grad_host)
{
    if (!md || !X || !T || B < 1) {
        set_error("invalid argument: model, batch or size");
        return NB_ERR_ARG;
    }
    NB_DEVICE_SCOPE(md->ctx->device);
    cudaStream_t s = md->ctx->stream;
    NB_TRY(model_scratch(md, B));
    double *dl = md->lpart + 4000;
    NB_TRY(model_backward(md, X, T, B, dl, s));
    double l = 0.0;
    NB_CUDA(cudaMemcpyAsync(&l, dl, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (grad_host)
        NB_CUDA(cudaMemcpyAsync(grad_host, md->grad, sizeof(float) * md->nparam,
                                cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    NB_TRY(gemm_check());
    if (loss_host) *loss_host = l / ((double)B * md->d);
    return NB_OK;
}

extern "C" nb_status nb_model_train(nb_model *md, const float *X, const float *T, int npairs,
                                    int epochs, int batch, float lr, double *final_loss)
{
    if (!md || !X || !T || npairs < 1 || epochs < 0 || batch < 1 || !(lr > 0.f)) {
        set_error("invalid argument: training set-up");
        return NB_ERR_ARG;
    }
    NB_DEVICE_SCOPE(md->ctx->device);
    cudaStream_t s = md->ctx->stream;
    batch = std::min(batch, npairs);
    NB_TRY(model_scratch(md, batch));
    const float b1 = 0.9f, b2 = 0.999f;
    double *dl = md->lpart + 4000;
    double lsum = 0.0;
    int lcnt = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        lsum = 0.0;
        lcnt = 0;
        for (int off = 0; off + batch <= npairs; off += batch) {
            NB_TRY(model_backward(md, X + (size_t)off * md->d, T + (size_t)off * md->d, batch,
                                  ep == epochs - 1 ? dl : nullptr, s));
            md->step += 1;
            const float c1 = 1.f - powf(b1, (float)md->step), c2 = 1.f - powf(b2, (float)md->step);
            k_adam<<<256, 256, 0, s>>>(md->nparam, md->W, md->grad, md->m, md->v, lr, b1, b2, c1,
                                       c2, 1e-8f);
            NB_CUDA(cudaGetLastError());
            if (ep == epochs - 1) {
                double l = 0.0;
                NB_CUDA(cudaMemcpyAsync(&l, dl, sizeof(double), cudaMemcpyDeviceToHost, s));
                NB_CUDA(cudaStreamSynchronize(s));
                lsum += l / ((double)batch * md->d);
                ++lcnt;
            }
        }
    }
    NB_CUDA(cudaStreamSynchronize(s));
    NB_TRY(gemm_check());
    if (final_loss) *final_loss = lcnt ? lsum / lcnt : 0.0;
    return NB_OK;
}

__global__ void k_sub64(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                        double *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

extern "C" nb_status nb_learned_collect(nb_mesh *m, const double *b, int nsnap,
                                        const int *snap_iters, int per_snap, uint64_t seed,
                                        int use_learned, float *X, float *T, int *count)
{
    if (!m || !b || nsnap < 1 || !snap_iters || per_snap < 1 || !X || !T || !count) {
        set_error("invalid argument: pair collection");
        return NB_ERR_ARG;
    }
    if (!m->gs_ready) {
        set_error("call nb_setup_gs first");
        return NB_ERR_STATE;
    }
    if (m->n > 12) {
        set_error("the learned preconditioner supports orders N <= 11");
        return NB_ERR_ARG;
    }
    if (use_learned && !m->learned) {
        set_error("use_learned needs an attached model");
        return NB_ERR_STATE;
    }
    NB_DEVICE_SCOPE(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    const size_t bytes = sizeof(double) * m->nL;
    const size_t smem = sizeof(double) * (7 * (size_t)m->n3 + (size_t)m->n * m->n);
    NB_CUDA(cudaFuncSetAttribute(k_interior_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    double *xk = nullptr, *rk = nullptr;
    int32_t *el = nullptr;
    std::vector<int32_t> pick(per_snap);
    nb_status st = NB_OK;
    cudaError_t ce = cudaMalloc(&xk, bytes);
    if (ce == cudaSuccess) ce = cudaMalloc(&rk, bytes);
    if (ce == cudaSuccess) ce = cudaMalloc(&el, sizeof(int32_t) * per_snap);
    if (ce != cudaSuccess) {
        set_error("pair collection buffers: %s", cudaGetErrorString(ce));
        st = NB_ERR_OOM;
    }
    uint64_t state = seed * 0x9E3779B97F4A7C15ull + 12345u;
    int total = 0;
    for (int q = 0; q < nsnap && st == NB_OK; ++q) {
        // the solver's iterate after snap_iters[q] steps from zero: Jacobi-PCG
        // in FP64, or the refinement's flexible CG with the attached network
        nb_opts o;
        nb_default_opts(&o);
        if (use_learned) {
            o.prec = NB_FP32;
            o.pc = NB_PC_LEARNED;
            o.max_outer = 1;
            o.inner_rtol = 1e-12;
        } else {
            o.prec = NB_FP64;
        }
        o.rtol = 1e-14;
        o.maxiter = snap_iters[q];
        if (solve(m, &o, b, xk, nullptr) < 0) { st = NB_ERR_CUDA; break; }
        // its residual r_k = b - A x_k
        if ((st = ax_local(m, NB_FP64, xk, rk, nullptr, nullptr, s)) != NB_OK) break;
        if ((st = dssum(m, NB_FP64, rk, 1, s)) != NB_OK) break;
        k_sub64<<<m->ctx->sm_count * 4, 256, 0, s>>>(m->nL, b, rk, rk);
        for (int i = 0; i < per_snap; ++i) {  // elements drawn with SplitMix64
            uint64_t z = (state += 0x9E3779B97F4A7C15ull);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            pick[i] = (int32_t)(z % (uint64_t)m->E);
        }
        if (cudaMemcpyAsync(el, pick.data(), sizeof(int32_t) * per_snap, cudaMemcpyHostToDevice,
                            s) != cudaSuccess) { st = NB_ERR_CUDA; break; }
        k_interior_pairs<<<std::min(per_snap, m->ctx->sm_count * 8), 256, smem, s>>>(
            per_snap, m->n, el, rk, m->G64, m->D64, m->dinv64, 1e-9, 1000,
            X + (size_t)total * m->n3, T + (size_t)total * m->n3);
        if (cudaGetLastError() != cudaSuccess) { st = NB_ERR_CUDA; break; }
        if (cudaStreamSynchronize(s) != cudaSuccess) { st = NB_ERR_CUDA; break; }
        total += per_snap;
    }
    cudaStreamSynchronize(s);
    cudaFree(xk);
    cudaFree(rk);
    cudaFree(el);
    *count = total;
    return st;
}

extern "C" nb_status nb_learned_targets(nb_mesh *m, const double *r_dev, const int32_t *elems_dev,
                                        int count, float *X_dev, float *T_dev)
{
    if (!m || !r_dev || !elems_dev || count < 0 || !X_dev || !T_dev) {
        set_error("invalid argument: targets");
        return NB_ERR_ARG;
    }
    if (!m->gs_ready || m->n > 12) {
        set_error("needs nb_setup_gs and N <= 11");
        return NB_ERR_STATE;
    }
    if (count == 0) return NB_OK;
    NB_DEVICE_SCOPE(m->ctx->device);
    const size_t smem = sizeof(double) * (7 * (size_t)m->n3 + (size_t)m->n * m->n);
    NB_CUDA(cudaFuncSetAttribute(k_interior_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    k_interior_pairs<<<std::min(count, m->ctx->sm_count * 8), 256, smem, m->ctx->stream>>>(
        count, m->n, elems_dev, r_dev, m->G64, m->D64, m->dinv64, 1e-9, 1000, X_dev, T_dev);
    NB_CUDA(cudaGetLastError());
    NB_CUDA(cudaStreamSynchronize(m->ctx->stream));
    return NB_OK;
}

extern "C" nb_status nb_learned_attach(nb_mesh *m, nb_model *md)
{
    if (!m) {
        set_error("invalid argument: mesh is NULL");
        return NB_ERR_ARG;
    }
    if (md && md->d != m->n3) {
        set_error("model order does not match the mesh");
        return NB_ERR_ARG;
    }
    m->learned = md;
    return NB_OK;
}

extern "C" nb_status nb_learned_apply(nb_mesh *m, const float *r_dev, float *z_dev)
{
    if (!m || !r_dev || !z_dev || !m->learned || !m->gs_ready) {
        set_error("invalid argument or no model attached");
        return NB_ERR_ARG;
    }
    NB_DEVICE_SCOPE(m->ctx->device);
    NB_TRY(model_apply(m, (nb_model *)m->learned, r_dev, z_dev, m->ctx->stream));
    NB_CUDA(cudaStreamSynchronize(m->ctx->stream));
    return gemm_check();
}

extern "C" nb_status nb_learned_step(nb_mesh *m, const float *r_dev, const float *wprev_dev,
                                     float *z_dev, double *zw, double *rz)
{
    if (!m || !r_dev || !wprev_dev || !z_dev || !zw || !rz) {
        set_error("invalid argument: NULL pointer");
        return NB_ERR_ARG;
    }
    nb_model *md = (nb_model *)m->learned;
    if (!md || !m->gs_ready) {
        set_error("no model attached or no gather-scatter set up");
        return NB_ERR_STATE;
    }
    if (!lpc_order(m->n) || !lpc_fits(md->d, md->h)) {
        set_error("the fused preconditioner needs N in {1,3,5,7} and hidden width <= 128");
        return NB_ERR_ARG;
    }
    NB_DEVICE_SCOPE(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    Workspace &ws = m->ws32;
    NB_TRY(ensure_ws(m, ws, 4, 0));
    NB_TRY(ensure_wimg(md, s));
    const size_t lsm = lpc_smem(md->d, md->h);
    NB_TRY(lpc_attr(m->n, lsm));
    NB_CUDA(cudaMemsetAsync(ws.scal, 0, sizeof(CgScalars), s));
    NB_CUDA(cudaMemsetAsync(m->kerr, 0, sizeof(int), s));
    const int grid = std::max(1, (int)std::min<int64_t>(m->E, m->ctx->sm_count));
    NB_TRY(launch_lpc(m->n, grid, lsm, s, (int)m->E, md->h, r_dev, m->dinv32, wprev_dev, z_dev,
                      md->Wimg, md->a, ws.scal, ws.part, m->kerr));
    m->launches += 1;
    int kerr = 0;
    NB_CUDA(cudaMemcpyAsync(ws.scal_host, ws.scal, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaMemcpyAsync(&kerr, m->kerr, sizeof(int), cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    if (kerr || ws.scal_host->status != 0) {
        set_error("fused preconditioner: a wait inside the kernel timed out");
        return NB_ERR_CUDA;
    }
    *zw = ws.scal_host->fcg_zw;
    *rz = ws.scal_host->rtz;
    return NB_OK;
}
