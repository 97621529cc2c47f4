// Gather-scatter (dssum + Dirichlet mask), global<->local maps, glsc3, and the
// Jacobi diagonal.
#include <algorithm>

#include "nb_reduce.cuh"

namespace nb {

// Direct-stiffness summation over the rows of shared or Dirichlet nodes: one
// thread per row sums the local copies in ascending local index and writes
// the (masked) sum back to every copy.  Rows are disjoint, so there are no
// races and no atomics; the order of the sum is fixed, so the result is
// bit-identical run to run.
template <typename T>
__global__ void k_gs(int64_t rows, const int32_t *__restrict__ off, const int32_t *__restrict__ loc,
                     const uint8_t *__restrict__ rmask, T *__restrict__ u, int masked)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < rows;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int o0 = off[a], o1 = off[a + 1];
        T s = T(0);
        for (int o = o0; o < o1; ++o) s += u[loc[o]];
        if (masked && rmask[a] == 0) s = T(0);
        for (int o = o0; o < o1; ++o) u[loc[o]] = s;
    }
}

nb_status gs_rows_launch(const nb_ctx *ctx, int64_t rows, const int32_t *off, const int32_t *loc,
                         const uint8_t *rmask, nb_prec prec, void *u, int masked, cudaStream_t s)
{
    if (rows == 0) return NB_OK;
    int grid = (int)std::min<int64_t>((rows + 255) / 256, (int64_t)ctx->sm_count * 8);
    if (prec == NB_FP64)
        k_gs<double><<<grid, 256, 0, s>>>(rows, off, loc, rmask, (double *)u, masked);
    else
        k_gs<float><<<grid, 256, 0, s>>>(rows, off, loc, rmask, (float *)u, masked);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// Masked summation from the rows split by kind: copies of Dirichlet nodes are
// zeroed without being read; free shared nodes with 2, 4 or 8 copies fetch
// their ascending copy list with one or two vector loads and sum in that
// order, so the result is the same as k_gs with masking.
template <typename T>
__global__ void k_gs_kinds(int64_t nz, int64_t np, int64_t nq, int64_t no,
                           const int32_t *__restrict__ zl, const int2 *__restrict__ pl,
                           const int4 *__restrict__ ql, const int4 *__restrict__ ol,
                           T *__restrict__ u)
{
    const int64_t total = nz + np + nq + no;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < total;
         a += (int64_t)gridDim.x * blockDim.x) {
        if (a < nz) {
            u[zl[a]] = T(0);
        } else if (a < nz + np) {
            const int2 c = pl[a - nz];
            const T s = u[c.x] + u[c.y];
            u[c.x] = s;
            u[c.y] = s;
        } else if (a < nz + np + nq) {
            const int4 c = ql[a - nz - np];
            const T s = ((u[c.x] + u[c.y]) + u[c.z]) + u[c.w];
            u[c.x] = s;
            u[c.y] = s;
            u[c.z] = s;
            u[c.w] = s;
        } else {
            const int64_t o = a - nz - np - nq;
            const int4 c = ol[2 * o], d = ol[2 * o + 1];
            const T s = ((((((u[c.x] + u[c.y]) + u[c.z]) + u[c.w]) + u[d.x]) + u[d.y]) + u[d.z]) +
                        u[d.w];
            u[c.x] = s;
            u[c.y] = s;
            u[c.z] = s;
            u[c.w] = s;
            u[d.x] = s;
            u[d.y] = s;
            u[d.z] = s;
            u[d.w] = s;
        }
    }
}

nb_status dssum(nb_mesh *m, nb_prec prec, void *u, int masked, cudaStream_t s)
{
    if (!masked || !m->gs_pair)
        return gs_rows_launch(m->ctx, m->gs_rows, m->gs_off, m->gs_loc, m->gs_mask, prec, u,
                              masked, s);
    const int64_t total = m->n_zero + m->n_pair + m->n_quad + m->n_oct;
    if (total == 0) return NB_OK;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)m->ctx->sm_count * 8);
    if (prec == NB_FP64)
        k_gs_kinds<double><<<grid, 256, 0, s>>>(m->n_zero, m->n_pair, m->n_quad, m->n_oct,
                                                m->gs_zero, m->gs_pair, m->gs_quad, m->gs_oct,
                                                (double *)u);
    else
        k_gs_kinds<float><<<grid, 256, 0, s>>>(m->n_zero, m->n_pair, m->n_quad, m->n_oct,
                                               m->gs_zero, m->gs_pair, m->gs_quad, m->gs_oct,
                                               (float *)u);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

template <typename T>
__global__ void k_to_local(int64_t nL, const int32_t *__restrict__ gid,
                           const uint8_t *__restrict__ mask, const T *__restrict__ ug,
                           T *__restrict__ uL, int masked)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = gid[l];
        T v = ug[g];
        if (masked && mask[g] == 0) v = T(0);
        uL[l] = v;
    }
}

template <typename T>
__global__ void k_to_global(int64_t nG, const int32_t *__restrict__ first,
                            const T *__restrict__ uL, T *__restrict__ ug)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nG;
         g += (int64_t)gridDim.x * blockDim.x)
        ug[g] = uL[first[g]];
}

nb_status to_local(nb_mesh *m, nb_prec prec, const void *ug, void *uL, int masked, cudaStream_t s)
{
    int grid = vec_grid(m->ctx, m->nL);
    if (prec == NB_FP64)
        k_to_local<double><<<grid, kVecThreads, 0, s>>>(m->nL, m->gid, m->mask_g,
                                                        (const double *)ug, (double *)uL, masked);
    else
        k_to_local<float><<<grid, kVecThreads, 0, s>>>(m->nL, m->gid, m->mask_g,
                                                       (const float *)ug, (float *)uL, masked);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status to_global(nb_mesh *m, nb_prec prec, const void *uL, void *ug, cudaStream_t s)
{
    int grid = vec_grid(m->ctx, m->nG);
    if (prec == NB_FP64)
        k_to_global<double><<<grid, kVecThreads, 0, s>>>(m->nG, m->g_first, (const double *)uL,
                                                         (double *)ug);
    else
        k_to_global<float><<<grid, kVecThreads, 0, s>>>(m->nG, m->g_first, (const float *)uL,
                                                        (float *)ug);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// glsc3: per-block partials of sum a*b*c (product in T, accumulated in FP64),
// then one block sums the partials in index order.
template <typename T>
__global__ void k_glsc3_part(int64_t n, const T *__restrict__ a, const T *__restrict__ b,
                             const float *__restrict__ c, double *__restrict__ part)
{
    __shared__ double sred[32];
    double acc = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x)
        acc += (double)(a[l] * b[l] * (T)c[l]);
    double t = block_sum(acc, sred);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_sum_partials(const double *__restrict__ part, int cnt, double *__restrict__ out)
{
    __shared__ double sred[32];
    double t = sum_partials(part, cnt, sred);
    if (threadIdx.x == 0) *out = t;
}

nb_status sum_partials_dev(const double *part, int cnt, double *out_dev, cudaStream_t s)
{
    k_sum_partials<<<1, kFinalizeThreads, 0, s>>>(part, cnt, out_dev);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status glsc3_dev(nb_mesh *m, nb_prec prec, const void *a, const void *b, double *part,
                    double *out_dev, cudaStream_t s)
{
    int grid = vec_grid(m->ctx, m->nL);
    if (prec == NB_FP64)
        k_glsc3_part<double><<<grid, kVecThreads, 0, s>>>(m->nL, (const double *)a,
                                                          (const double *)b, m->c32, part);
    else
        k_glsc3_part<float><<<grid, kVecThreads, 0, s>>>(m->nL, (const float *)a,
                                                         (const float *)b, m->c32, part);
    NB_CUDA(cudaGetLastError());
    k_sum_partials<<<1, kFinalizeThreads, 0, s>>>(part, grid, out_dev);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// Diagonal of the local operator (set-up, FP64):
//   sum_l D[l][i]^2 Grr(l,j,k) + D[l][j]^2 Gss(i,l,k) + D[l][k]^2 Gtt(i,j,l)
//   + 2 (D[i][i] D[j][j] Grs + D[i][i] D[k][k] Grt + D[j][j] D[k][k] Gst)(i,j,k)
__global__ void k_local_diag(int64_t E, int n, const double *__restrict__ D,
                             const double *__restrict__ G, double *__restrict__ d)
{
    const int n3 = n * n * n;
    const int64_t total = E * n3;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t / n3;
        const int q = (int)(t - e * n3);
        const int i = q % n, j = (q / n) % n, k = q / (n * n);
        const double *Ge = G + e * 6 * n3;
        double s = 0.0;
        for (int l = 0; l < n; ++l) {
            s += D[l * n + i] * D[l * n + i] * Ge[0 * n3 + (k * n + j) * n + l];
            s += D[l * n + j] * D[l * n + j] * Ge[3 * n3 + (k * n + l) * n + i];
            s += D[l * n + k] * D[l * n + k] * Ge[5 * n3 + (l * n + j) * n + i];
        }
        s += 2.0 * D[i * n + i] * D[j * n + j] * Ge[1 * n3 + q];
        s += 2.0 * D[i * n + i] * D[k * n + k] * Ge[2 * n3 + q];
        s += 2.0 * D[j * n + j] * D[k * n + k] * Ge[4 * n3 + q];
        d[t] = s;
    }
}

nb_status local_diag(nb_mesh *m, double *diag, cudaStream_t s)
{
    int grid = vec_grid(m->ctx, m->nL);
    k_local_diag<<<grid, kVecThreads, 0, s>>>(m->E, m->n, m->D64, m->G64, diag);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// Inverse assembled diagonal (0 on Dirichlet nodes) and the identity
// preconditioner (the mask).  The sign bit of both marks the copy that owns
// its global node (+ on the first local copy, - on the others): the solver's
// dot products sum over owner copies instead of weighting every copy by
// 1/multiplicity, and the preconditioner applies |value|.
// The first copy of a global node owns it, except on a slab's lower
// interface plane (global indices below lo_plane), which the slab below owns.
__global__ void k_finish_jacobi(int64_t nL, const double *__restrict__ diag,
                                const int32_t *__restrict__ gid,
                                const int32_t *__restrict__ first, int64_t lo_plane,
                                double *dinv64, float *dinv32, double *ones64, float *ones32)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x) {
        const double d = diag[l];
        const int32_t g = gid[l];
        const double sgn = first[g] == (int32_t)l && g >= lo_plane ? 1.0 : -1.0;
        const double v = sgn * (d != 0.0 ? 1.0 / d : 0.0);
        const double one = sgn * (d != 0.0 ? 1.0 : 0.0);
        dinv64[l] = v;
        dinv32[l] = (float)v;
        ones64[l] = one;
        ones32[l] = (float)one;
    }
}

nb_status finish_jacobi(nb_mesh *m, double *diag, cudaStream_t s)
{
    int grid = vec_grid(m->ctx, m->nL);
    const int64_t lo_plane =
        m->iface_lo ? ((int64_t)m->nx * m->N + 1) * ((int64_t)m->ny * m->N + 1) : 0;
    k_finish_jacobi<<<grid, kVecThreads, 0, s>>>(m->nL, diag, m->gid, m->g_first, lo_plane,
                                                 m->dinv64, m->dinv32, m->ones64, m->ones32);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// Evict the L2 cache between timed launches: write the caller's buffer
// (larger than L2), then read it back, so that the dirty lines the writes
// leave are written back to DRAM before the timed kernel starts and it
// begins, like a profiler's cache flush, on a clean cache holding none of its
// data.  The read's sum is stored only if it equals an impossible value.
__global__ void k_flush_read(const uint4 *__restrict__ buf, int64_t n16, unsigned int *sink)
{
    unsigned int acc = 0u;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n16;
         q += (int64_t)gridDim.x * blockDim.x) {
        const uint4 v = buf[q];
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x9e3779b9u && sink) *sink = acc;
}

nb_status l2_flush(const nb_ctx *ctx, void *buf, size_t bytes, int pattern, cudaStream_t s)
{
    if (!buf || bytes < 16) return NB_OK;
    NB_CUDA(cudaMemsetAsync(buf, pattern & 0xff, bytes, s));
    const int64_t n16 = (int64_t)(bytes / 16);
    k_flush_read<<<ctx->sm_count * 8, 256, 0, s>>>((const uint4 *)buf, n16, nullptr);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

}  // namespace nb
