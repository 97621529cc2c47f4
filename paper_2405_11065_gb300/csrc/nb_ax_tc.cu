// Operator with the derivative contractions on tensor cores (FP16 or BF16
// operands, FP32 accumulation): the "tensor-core ax" precision variant.
//
// Each of the six contractions of ax -- ur, us, ut = (D x I x I, I x D x I,
// I x I x D) u and the three transposed ones -- is a batch of small matrix
// products with K = n <= 16 (padded to 16) and N = n (two n8 tiles):
//   direction r, layer k:  C[j][i'] = sum_l U[k][j][l] D[i'][l]
//   direction s, layer k:  C[i][j'] = sum_l U[k][l][i] D[j'][l]
//   direction t, row j:    C[i][k'] = sum_l U[l][j][i] D[k'][l]
// (and the same with D^T for the transposed terms).  The element is staged
// in shared memory as a zero-padded 16x16x16 half-precision cube, so every A
// tile is one ldmatrix.x4 (direction r) or ldmatrix.x4.trans (s, t) with
// per-row addresses; the B fragments (D or D^T) stay in registers for the
// whole kernel.  The outputs go through FP32 shared memory to meet at each
// node for the geometric factors, whose products are FP32.
//
// Range: before each rounding to 16 bits the element's values are scaled by
// an exact power of two so that their maximum magnitude is at most 1; the
// scale is undone exactly on the FP32 result.  The rounding of u and of
// (wr, ws, wt) to 11 (FP16) or 8 (BF16) significant bits is the variant's
// only error source beyond FP32 arithmetic; it is measured against the FP64
// oracle by the tests.
//
// The operator is HBM-bound (about 4 flop per byte); the tensor cores remove
// the CUDA-core contraction work, not the memory traffic.  These are
// warp-level mma.sync m16n8k16 instructions.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "nb_cg_dev.cuh"

namespace nb {

static __device__ float g_dtc[(kMaxn + 1) * kMaxn * kMaxn];  // FP32 D of every order

nb_status upload_D_tc(int n, const double *D)
{
    float tab[kMaxn * kMaxn] = {};
    for (int i = 0; i < n; ++i)
        for (int l = 0; l < n; ++l) tab[i * kMaxn + l] = (float)D[i * n + l];
    NB_CUDA(cudaMemcpyToSymbol(g_dtc, tab, sizeof(tab), sizeof(tab) * n, cudaMemcpyHostToDevice));
    return NB_OK;
}

template <typename H>
__device__ __forceinline__ uint32_t pack2(float a, float b);
template <>
__device__ __forceinline__ uint32_t pack2<__half>(float a, float b)
{
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
template <>
__device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

template <typename H>
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1);
template <>
__device__ __forceinline__ void mma16816<__half>(float c[4], const uint32_t a[4], uint32_t b0,
                                                 uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
template <>
__device__ __forceinline__ void mma16816<__nv_bfloat16>(float c[4], const uint32_t a[4],
                                                        uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t a[4], const void *row_addr)
{
    uint32_t s = (uint32_t)__cvta_generic_to_shared(row_addr);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(s));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t a[4], const void *row_addr)
{
    uint32_t s = (uint32_t)__cvta_generic_to_shared(row_addr);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(s));
}

constexpr int kTcThreads = 128;  // four warps per block

// Smallest power-of-two exponent e with max |v| * 2^-e <= 1 (0 if v == 0).
__device__ __forceinline__ int pow2_exponent(float vmax)
{
    if (!(vmax > 0.f)) return 0;
    int e;
    frexpf(vmax, &e);  // vmax = f * 2^e, f in [0.5, 1)
    return e;
}

// One batch of 16x16x16 contractions for the warp's tiles.  MODE selects the
// A-tile addressing (0: rows j of layer k, K along i; 1: rows i of layer k, K
// along j; 2: rows i of row j, K along k).  The FP32 results are written
// (ACC = false) or added (ACC = true) to out[k][j][i] (compact n^3).
template <typename H, int n, int MODE, bool ACC>
__device__ __forceinline__ void tc_pass(const H *cube, const uint32_t bfrag[2][2], float *out,
                                        int warp, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    const int q = lane >> 3, r = lane & 7;
    for (int tile = warp; tile < n; tile += kTcThreads / 32) {
        uint32_t a[4];
        if (MODE == 0) {
            // A[j][l] = cube[tile=k][j][l]
            const int j = r + 8 * (q & 1), l0 = 8 * (q >> 1);
            ldsm_x4(a, cube + ((tile * 16 + j) * 16 + l0));
        } else if (MODE == 1) {
            // A[i][l] = cube[tile=k][l][i]: memory rows l, eight consecutive i
            const int l = r + 8 * (q >> 1), i0 = 8 * (q & 1);
            ldsm_x4_t(a, cube + ((tile * 16 + l) * 16 + i0));
        } else {
            // A[i][l] = cube[l][tile=j][i]
            const int l = r + 8 * (q >> 1), i0 = 8 * (q & 1);
            ldsm_x4_t(a, cube + ((l * 16 + tile) * 16 + i0));
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            mma16816<H>(c, a, bfrag[nt][0], bfrag[nt][1]);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int row = g + 8 * (h >> 1);          // A row index
                const int col = 8 * nt + 2 * t + (h & 1);  // output index
                int i, j, k;
                if (MODE == 0) { k = tile; j = row; i = col; }
                else if (MODE == 1) { k = tile; i = row; j = col; }
                else { j = tile; i = row; k = col; }
                if (i < n && j < n && k < n) {
                    float *o = out + (k * n + j) * n + i;
                    if (ACC) *o += c[h];
                    else *o = c[h];
                }
            }
        }
    }
}

template <typename H, int n, bool PUPD>
__global__ void __launch_bounds__(kTcThreads)
k_ax_tc(long long E, const float *__restrict__ G, const float *__restrict__ uin,
        float *__restrict__ w, const float *__restrict__ r, const float *__restrict__ dinv,
        float *__restrict__ p, CgScalars *__restrict__ scal, double *__restrict__ part)
{
    constexpr int n3 = n * n * n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    H *cube = reinterpret_cast<H *>(smem_raw);        // [16][16][16], zero padded
    float *f0 = reinterpret_cast<float *>(cube + 4096);  // [n3] ur -> wr -> w
    float *f1 = f0 + n3;                                 // [n3] us -> ws
    float *f2 = f1 + n3;                                 // [n3] ut -> wt
    __shared__ float sred[32];
    __shared__ double sredd[32];
    if (PUPD && scal->done) return;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    // B fragments: forward B[l][i'] = D[i'][l]; transposed B[l][i] = D[l][i]
    const float *Dn = g_dtc + n * kMaxn * kMaxn;
    uint32_t bf[2][2], bt[2][2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int col = g + 8 * nt;
        float v[4], vt[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int kk = 2 * t + (h & 1) + 8 * (h >> 1);
            v[h] = (col < n && kk < n) ? Dn[col * kMaxn + kk] : 0.f;
            vt[h] = (col < n && kk < n) ? Dn[kk * kMaxn + col] : 0.f;
        }
        bf[nt][0] = pack2<H>(v[0], v[1]);
        bf[nt][1] = pack2<H>(v[2], v[3]);
        bt[nt][0] = pack2<H>(vt[0], vt[1]);
        bt[nt][1] = pack2<H>(vt[2], vt[3]);
    }
    for (int q = tid; q < 4096; q += kTcThreads) cube[q] = H(0.f);
    const float beta = PUPD ? (float)scal->beta : 0.f;
    double acc = 0.0;
    __syncthreads();

    for (long long e = blockIdx.x; e < E; e += gridDim.x) {
        const size_t base = (size_t)e * n3;
        // 1. load (or form) u, its max magnitude
        float umax = 0.f;
        for (int q = tid; q < n3; q += kTcThreads) {
            float v;
            if (PUPD) {
                v = fabsf(dinv[base + q]) * r[base + q] + beta * p[base + q];
                p[base + q] = v;
            } else {
                v = uin[base + q];
            }
            f0[q] = v;
            umax = fmaxf(umax, fabsf(v));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
        if (lane == 0) sred[warp] = umax;
        __syncthreads();
        umax = fmaxf(fmaxf(sred[0], sred[1]), fmaxf(sred[2], sred[3]));
        const int eu = pow2_exponent(umax);
        for (int q = tid; q < n3; q += kTcThreads) {
            const int i = q % n, j = (q / n) % n, k = q / (n * n);
            cube[(k * 16 + j) * 16 + i] = H(ldexpf(f0[q], -eu));
        }
        __syncthreads();
        // 2. forward contractions into f0, f1, f2
        tc_pass<H, n, 0, false>(cube, bf, f0, warp, lane);
        tc_pass<H, n, 1, false>(cube, bf, f1, warp, lane);
        tc_pass<H, n, 2, false>(cube, bf, f2, warp, lane);
        __syncthreads();
        // 3. geometric factors (FP32), max of the results
        float wmax = 0.f;
        const float *Ge = G + (size_t)e * 6 * n3;
        for (int q = tid; q < n3; q += kTcThreads) {
            const float ur = f0[q], us = f1[q], ut = f2[q];
            const float g0 = Ge[q], g1 = Ge[n3 + q], g2 = Ge[2 * n3 + q];
            const float g3 = Ge[3 * n3 + q], g4 = Ge[4 * n3 + q], g5 = Ge[5 * n3 + q];
            const float wr = g0 * ur + g1 * us + g2 * ut;
            const float ws = g1 * ur + g3 * us + g4 * ut;
            const float wt = g2 * ur + g4 * us + g5 * ut;
            f0[q] = wr;
            f1[q] = ws;
            f2[q] = wt;
            wmax = fmaxf(wmax, fmaxf(fabsf(wr), fmaxf(fabsf(ws), fabsf(wt))));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
        __syncthreads();  // everyone has read sred (umax) and finished step 3
        if (lane == 0) sred[warp] = wmax;
        __syncthreads();
        wmax = fmaxf(fmaxf(sred[0], sred[1]), fmaxf(sred[2], sred[3]));
        const int ew = pow2_exponent(wmax);
        // 4. transposed contractions: one rounded cube per term, summed in f0
        //    (term r), then f1 (+ term s) ... accumulated into f0 at the end
        for (int q = tid; q < n3; q += kTcThreads) {
            const int i = q % n, j = (q / n) % n, k = q / (n * n);
            cube[(k * 16 + j) * 16 + i] = H(ldexpf(f0[q], -ew));
        }
        __syncthreads();
        tc_pass<H, n, 0, false>(cube, bt, f0, warp, lane);  // f0 = term r
        __syncthreads();
        for (int q = tid; q < n3; q += kTcThreads) {
            const int i = q % n, j = (q / n) % n, k = q / (n * n);
            cube[(k * 16 + j) * 16 + i] = H(ldexpf(f1[q], -ew));
        }
        __syncthreads();
        tc_pass<H, n, 1, true>(cube, bt, f0, warp, lane);   // f0 += term s
        __syncthreads();
        for (int q = tid; q < n3; q += kTcThreads) {
            const int i = q % n, j = (q / n) % n, k = q / (n * n);
            cube[(k * 16 + j) * 16 + i] = H(ldexpf(f2[q], -ew));
        }
        __syncthreads();
        tc_pass<H, n, 2, true>(cube, bt, f0, warp, lane);   // f0 += term t
        __syncthreads();
        // 5. undo the scales, write w, partial of p.w
        float s = 0.f;
        const int esum = eu + ew;
        for (int q = tid; q < n3; q += kTcThreads) {
            const float v = ldexpf(f0[q], esum);
            w[base + q] = v;
            s += (PUPD ? p[base + q] : uin[base + q]) * v;
        }
        acc += (double)s;
        __syncthreads();  // f0 and cube are reused by the next element
    }
    if (part) {
        double tsum = block_sum(acc, sredd);
        if (tid == 0) part[blockIdx.x] = tsum;
        if (PUPD && last_block(&scal->tick_ax)) cg_finish_pap(scal, part, gridDim.x, sredd);
    }
}

template <typename H, int n, bool PUPD>
static nb_status launch_tc(int sm_count, long long E, const float *G, const float *u, float *w,
                           const float *r, const float *dinv, float *p, CgScalars *scal,
                           double *part, int *grid_io, cudaStream_t s)
{
    auto kern = k_ax_tc<H, n, PUPD>;
    const size_t smem = 4096 * sizeof(H) + 3 * sizeof(float) * n * n * n;
    static int grid_cache_dev[kMaxDevices] = {};  // per device, as the smem attribute
    int &grid_cache = device_slot(grid_cache_dev);
    if (grid_cache == 0) {
        NB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTcThreads, smem));
        grid_cache = (per_sm < 1 ? 1 : per_sm) * sm_count;
    }
    int grid = (int)(E < grid_cache ? E : grid_cache);
    if (grid < 1) grid = 1;
    kern<<<grid, kTcThreads, smem, s>>>(E, G, u, w, r, dinv, p, scal, part);
    NB_CUDA(cudaGetLastError());
    if (grid_io) *grid_io = grid;
    return NB_OK;
}

template <typename H>
static nb_status dispatch_tc(int n, bool pupd, int sm_count, long long E, const float *G,
                             const float *u, float *w, const float *r, const float *dinv, float *p,
                             CgScalars *scal, double *part, int *grid, cudaStream_t s)
{
#define NB_TC_CASE(NN)                                                                        \
    case NN:                                                                                  \
        return pupd ? launch_tc<H, NN, true>(sm_count, E, G, u, w, r, dinv, p, scal, part,    \
                                             grid, s)                                         \
                    : launch_tc<H, NN, false>(sm_count, E, G, u, w, r, dinv, p, scal, part,   \
                                              grid, s);
    switch (n) {
        NB_TC_CASE(2)
        NB_TC_CASE(3)
        NB_TC_CASE(4)
        NB_TC_CASE(5)
        NB_TC_CASE(6)
        NB_TC_CASE(7)
        NB_TC_CASE(8)
        NB_TC_CASE(9)
        NB_TC_CASE(10)
        NB_TC_CASE(11)
        NB_TC_CASE(12)
        NB_TC_CASE(13)
        NB_TC_CASE(14)
        NB_TC_CASE(15)
        NB_TC_CASE(16)
        default:
            set_error("unsupported order n=%d", n);
            return NB_ERR_ARG;
    }
#undef NB_TC_CASE
}

nb_status ax_tc(nb_mesh *m, nb_prec prec, bool pupd, const float *u, float *w, const float *r,
                const float *dinv, float *p, CgScalars *scal, double *part, int *grid,
                cudaStream_t s)
{
    if (prec == NB_TC_F16)
        return dispatch_tc<__half>(m->n, pupd, m->ctx->sm_count, m->E, m->G32, u, w, r, dinv, p,
                                   scal, part, grid, s);
    return dispatch_tc<__nv_bfloat16>(m->n, pupd, m->ctx->sm_count, m->E, m->G32, u, w, r, dinv,
                                      p, scal, part, grid, s);
}

}  // namespace nb
