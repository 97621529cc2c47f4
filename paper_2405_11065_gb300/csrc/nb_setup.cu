// Mesh set-up: GLL points, derivative matrix, device geometric factors,
// global numbering and gather-scatter lists, Jacobi diagonal.
//
// The case study keeps the initialisation in double precision and converts
// only the CG-loop variables (Section 6, steps 3-4); here the geometry is
// computed once in FP64 on the device and a rounded FP32 copy is kept for the
// reduced-precision operator.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "nb_internal.h"

namespace nb {

// Legendre P_N and P_{N-1} at x by the three-term recurrence.
static void legendre2(int N, double x, double *pn, double *pnm1)
{
    double a = 1.0, b = x;
    if (N == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
    for (int k = 2; k <= N; ++k) {
        double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
        a = b;
        b = c;
    }
    *pn = b;
    *pnm1 = a;
}

// GLL points: the endpoints and the zeros of P'_N, found by Newton's method on
// P'_N itself, with P'_N = N (x P_N - P_{N-1}) / (x^2 - 1) and P''_N from the
// Legendre equation (1-x^2) P'' = 2x P' - N(N+1) P.  Weights 2/(N(N+1)P_N^2).
nb_status gll_host(int N, double *xi, double *w)
{
    if (N < 1 || N > kMaxN) return NB_ERR_ARG;
    const double pi = 3.14159265358979323846;
    for (int j = 0; j <= N; ++j) {
        double x = -cos(pi * j / N);
        if (j > 0 && j < N) {
            for (int it = 0; it < 60; ++it) {
                double pn, pm;
                legendre2(N, x, &pn, &pm);
                double d1 = N * (x * pn - pm) / (x * x - 1.0);
                double d2 = (2.0 * x * d1 - N * (N + 1.0) * pn) / (1.0 - x * x);
                double step = d1 / d2;
                x -= step;
                if (fabs(step) <= 1e-16) break;
            }
        }
        xi[j] = x;
    }
    xi[0] = -1.0;
    xi[N] = 1.0;
    for (int j = 0; j <= N / 2; ++j) {  // enforce the symmetry of the point set
        double h = 0.5 * (xi[N - j] - xi[j]);
        xi[j] = -h;
        xi[N - j] = h;
    }
    if ((N & 1) == 0) xi[N / 2] = 0.0;
    for (int j = 0; j <= N; ++j) {
        double pn, pm;
        legendre2(N, xi[j], &pn, &pm);
        w[j] = 2.0 / (N * (N + 1.0) * pn * pn);
    }
    return NB_OK;
}

// D[i*n+j] = derivative of the j-th GLL Lagrange polynomial at xi_i.
void deriv_host(int N, const double *xi, double *D)
{
    const int n = N + 1;
    double P[kMaxn];
    for (int j = 0; j < n; ++j) {
        double pm;
        legendre2(N, xi[j], &P[j], &pm);
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v = 0.0;
            if (i != j) v = P[i] / (P[j] * (xi[i] - xi[j]));
            else if (i == 0) v = -0.25 * N * (N + 1);
            else if (i == N) v = 0.25 * N * (N + 1);
            D[i * n + j] = v;
        }
}

// One block per element (grid-stride): coordinates of the n^3 nodes into
// shared memory, then per node the Jacobian matrix by the derivative matrix,
// its determinant and inverse, and the six factors
// G_ab = w_i w_j w_k J sum_d (dr_a/dx_d)(dr_b/dx_d).
// The elements are ez = 0..nz-1 of the mesh, at position ez + zoff of a box
// of nzg elements along z (a slab of it; zoff = 0, nzg = nz for a whole box).
__global__ void k_geometry(int nx, int ny, int nz, int zoff, int nzg, int n, double amp,
                           const double *__restrict__ xi,
                           const double *__restrict__ wq, const double *__restrict__ D,
                           double *__restrict__ G64, float *__restrict__ G32, int *bad)
{
    extern __shared__ double sh[];
    const int n3 = n * n * n;
    double *X = sh, *Y = sh + n3, *Z = sh + 2 * n3;
    const double pi = 3.14159265358979323846;
    const long long E = (long long)nx * ny * nz;
    for (long long e = blockIdx.x; e < E; e += gridDim.x) {
        const long long ex = e % nx, ey = (e / nx) % ny, ez = e / ((long long)nx * ny);
        for (int q = threadIdx.x; q < n3; q += blockDim.x) {
            int i = q % n, j = (q / n) % n, k = q / (n * n);
            double x0 = (ex + 0.5 * (1.0 + xi[i])) / nx;
            double y0 = (ey + 0.5 * (1.0 + xi[j])) / ny;
            double z0 = (ez + zoff + 0.5 * (1.0 + xi[k])) / nzg;
            double d = amp * sin(pi * x0) * sin(pi * y0) * sin(pi * z0);
            X[q] = x0 + d;
            Y[q] = y0 + d;
            Z[q] = z0 + d;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < n3; q += blockDim.x) {
            int i = q % n, j = (q / n) % n, k = q / (n * n);
            double a[3][3];  // a[c][r] = d x_c / d r_r
            const double *C[3] = {X, Y, Z};
            for (int c = 0; c < 3; ++c) {
                double sr = 0, ss = 0, st = 0;
                for (int l = 0; l < n; ++l) {
                    sr += D[i * n + l] * C[c][(k * n + j) * n + l];
                    ss += D[j * n + l] * C[c][(k * n + l) * n + i];
                    st += D[k * n + l] * C[c][(l * n + j) * n + i];
                }
                a[c][0] = sr;
                a[c][1] = ss;
                a[c][2] = st;
            }
            double c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
            double c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
            double c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
            double J = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
            if (!(J > 0.0)) atomicAdd(bad, 1);
            // inverse Jacobian inv[r][c] = d r_r / d x_c = cofactor(c, r) / J
            double inv[3][3];
            inv[0][0] = c00 / J;
            inv[1][0] = c01 / J;
            inv[2][0] = c02 / J;
            inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / J;
            inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / J;
            inv[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / J;
            inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / J;
            inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / J;
            inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / J;
            const double scale = wq[i] * wq[j] * wq[k] * J;
            const int ra[6] = {0, 0, 0, 1, 1, 2}, rb[6] = {0, 1, 2, 1, 2, 2};
            for (int f = 0; f < 6; ++f) {
                double s = inv[ra[f]][0] * inv[rb[f]][0] + inv[ra[f]][1] * inv[rb[f]][1] +
                           inv[ra[f]][2] * inv[rb[f]][2];
                double g = scale * s;
                size_t o = ((size_t)e * 6 + f) * n3 + q;
                G64[o] = g;
                G32[o] = (float)g;
            }
        }
        __syncthreads();
    }
}

nb_status build_geometry(nb_mesh *m)
{
    const int N = m->N, n = m->n;
    double xi[kMaxn], wq[kMaxn], D[kMaxn * kMaxn];
    NB_TRY(gll_host(N, xi, wq));
    deriv_host(N, xi, D);
    NB_TRY(upload_deriv_tables(n, D));
    cudaStream_t s = m->ctx->stream;
    double *dxi = nullptr, *dw = nullptr;
    int *dbad = nullptr;
    NB_CUDA(cudaMalloc(&m->kerr, sizeof(int)));
    NB_CUDA(cudaMemsetAsync(m->kerr, 0, sizeof(int), s));
    NB_CUDA(cudaMalloc(&m->D64, sizeof(double) * n * n));
    NB_CUDA(cudaMalloc(&m->D32, sizeof(float) * n * n));
    float D32h[kMaxn * kMaxn];
    for (int t = 0; t < n * n; ++t) D32h[t] = (float)D[t];
    NB_CUDA(cudaMemcpyAsync(m->D64, D, sizeof(double) * n * n, cudaMemcpyHostToDevice, s));
    NB_CUDA(cudaMemcpyAsync(m->D32, D32h, sizeof(float) * n * n, cudaMemcpyHostToDevice, s));
    const size_t ng = (size_t)m->E * 6 * m->n3;
    NB_CUDA(cudaMalloc(&m->G64, sizeof(double) * ng));
    NB_CUDA(cudaMalloc(&m->G32, sizeof(float) * ng));
    NB_CUDA(cudaMalloc(&dxi, sizeof(double) * n * 2 + sizeof(int)));
    dw = dxi + n;
    dbad = (int *)(dxi + 2 * n);
    NB_CUDA(cudaMemcpyAsync(dxi, xi, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    NB_CUDA(cudaMemcpyAsync(dw, wq, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    NB_CUDA(cudaMemsetAsync(dbad, 0, sizeof(int), s));
    const size_t smem = sizeof(double) * 3 * m->n3;
    NB_CUDA(cudaFuncSetAttribute(k_geometry, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    int grid = (int)std::min<int64_t>(m->E, (int64_t)m->ctx->sm_count * 8);
    const int nzg = m->nz_glob > 0 ? m->nz_glob : m->nz;
    int mx = std::max(m->nx, std::max(m->ny, nzg));
    k_geometry<<<grid, 256, smem, s>>>(m->nx, m->ny, m->nz, m->z_off, nzg, n, m->deform / mx, dxi,
                                       dw, m->D64, m->G64, m->G32, dbad);
    NB_CUDA(cudaGetLastError());
    int bad = 0;
    NB_CUDA(cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    NB_CUDA(cudaFree(dxi));
    if (bad) {
        set_error("mesh has %d nodes with a non-positive Jacobian (deform too large)", bad);
        return NB_ERR_MESH;
    }
    return NB_OK;
}

// Global numbering (closed form on the box), multiplicities, mask, and the
// gather-scatter rows: every global node that has more than one local copy or
// lies on the Dirichlet boundary, with its copies in ascending local index.
nb_status build_gs(nb_mesh *m)
{
    const int N = m->N, n = m->n;
    const int64_t Gx = (int64_t)m->nx * N + 1, Gy = (int64_t)m->ny * N + 1,
                  Gz = (int64_t)m->nz * N + 1;
    const int64_t nL = m->nL, nG = m->nG;
    std::vector<int32_t> gid(nL);
    m->mult_host.assign(nG, 0);
    m->mask_host.assign(nG, 1);
    for (int64_t e = 0; e < m->E; ++e) {
        int64_t ex = e % m->nx, ey = (e / m->nx) % m->ny, ez = e / ((int64_t)m->nx * m->ny);
        int64_t base = e * m->n3;
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j) {
                int64_t row = (ex * N) + Gx * ((ey * N + j) + Gy * (ez * N + k));
                int32_t *dst = &gid[base + (k * n + j) * n];
                for (int i = 0; i < n; ++i) {
                    dst[i] = (int32_t)(row + i);
                    m->mult_host[row + i] += 1;
                }
            }
    }
    for (int64_t gz = 0; gz < Gz; ++gz)
        for (int64_t gy = 0; gy < Gy; ++gy) {
            // an interface plane of a slab is not on the Dirichlet boundary
            bool face = (gz == 0 && !m->iface_lo) || (gz == Gz - 1 && !m->iface_hi) || gy == 0 ||
                        gy == Gy - 1;
            uint8_t *mrow = &m->mask_host[Gx * (gy + Gy * gz)];
            for (int64_t gx = 0; gx < Gx; ++gx)
                mrow[gx] = (face || gx == 0 || gx == Gx - 1) ? 0 : 1;
        }
    // rows of the gather-scatter
    std::vector<int32_t> row_of(nG, -1);
    std::vector<int32_t> rgid, roff(1, 0);
    std::vector<uint8_t> rmask;
    for (int64_t g = 0; g < nG; ++g) {
        if (m->mult_host[g] > 1 || m->mask_host[g] == 0) {
            row_of[g] = (int32_t)rgid.size();
            rgid.push_back((int32_t)g);
            rmask.push_back(m->mask_host[g]);
            roff.push_back(roff.back() + m->mult_host[g]);
        }
    }
    const int64_t rows = (int64_t)rgid.size(), copies = roff.back();
    std::vector<int32_t> rloc(copies);
    std::vector<int32_t> fill(roff.begin(), roff.end() - 1);
    std::vector<int32_t> first(nG, -1);
    std::vector<float> c(nL);
    for (int64_t l = 0; l < nL; ++l) {
        int32_t g = gid[l];
        int32_t r = row_of[g];
        if (r >= 0) rloc[fill[r]++] = (int32_t)l;
        if (first[g] < 0) first[g] = (int32_t)l;
        // the global multiplicity of a slab's interface-plane node counts the
        // neighbouring slab's copies too (as many as this slab's)
        const int64_t gzl = g / (Gx * Gy);
        const bool shared = (gzl == 0 && m->iface_lo) || (gzl == Gz - 1 && m->iface_hi);
        c[l] = 1.0f / (float)(m->mult_host[g] * (shared ? 2 : 1));
    }
    cudaStream_t s = m->ctx->stream;
    m->gs_rows = rows;
    m->gs_copies = copies;
    NB_CUDA(cudaMalloc(&m->gid, sizeof(int32_t) * nL));
    NB_CUDA(cudaMalloc(&m->gs_off, sizeof(int32_t) * (rows + 1)));
    NB_CUDA(cudaMalloc(&m->gs_loc, sizeof(int32_t) * std::max<int64_t>(copies, 1)));
    NB_CUDA(cudaMalloc(&m->gs_gid, sizeof(int32_t) * std::max<int64_t>(rows, 1)));
    NB_CUDA(cudaMalloc(&m->gs_mask, std::max<int64_t>(rows, 1)));
    NB_CUDA(cudaMalloc(&m->g_first, sizeof(int32_t) * nG));
    NB_CUDA(cudaMalloc(&m->mask_g, nG));
    NB_CUDA(cudaMalloc(&m->c32, sizeof(float) * nL));
    NB_CUDA(cudaMemcpyAsync(m->gid, gid.data(), sizeof(int32_t) * nL, cudaMemcpyHostToDevice, s));
    NB_CUDA(cudaMemcpyAsync(m->gs_off, roff.data(), sizeof(int32_t) * (rows + 1),
                            cudaMemcpyHostToDevice, s));
    if (copies)
        NB_CUDA(cudaMemcpyAsync(m->gs_loc, rloc.data(), sizeof(int32_t) * copies,
                                cudaMemcpyHostToDevice, s));
    if (rows) {
        NB_CUDA(cudaMemcpyAsync(m->gs_gid, rgid.data(), sizeof(int32_t) * rows,
                                cudaMemcpyHostToDevice, s));
        NB_CUDA(cudaMemcpyAsync(m->gs_mask, rmask.data(), rows, cudaMemcpyHostToDevice, s));
    }
    NB_CUDA(cudaMemcpyAsync(m->g_first, first.data(), sizeof(int32_t) * nG,
                            cudaMemcpyHostToDevice, s));
    NB_CUDA(cudaMemcpyAsync(m->mask_g, m->mask_host.data(), nG, cudaMemcpyHostToDevice, s));
    NB_CUDA(cudaMemcpyAsync(m->c32, c.data(), sizeof(float) * nL, cudaMemcpyHostToDevice, s));
    // the rows by kind (see nb_internal.h); copies stay in ascending order
    std::vector<int32_t> zero;
    std::vector<int2> pair;
    std::vector<int4> quad, oct;
    for (int64_t a = 0; a < rows; ++a) {
        const int32_t *lc = &rloc[roff[a]];
        const int cnt = roff[a + 1] - roff[a];
        if (rmask[a] == 0) {
            for (int q = 0; q < cnt; ++q) zero.push_back(lc[q]);
        } else if (cnt == 2) {
            pair.push_back(make_int2(lc[0], lc[1]));
        } else if (cnt == 4) {
            quad.push_back(make_int4(lc[0], lc[1], lc[2], lc[3]));
        } else if (cnt == 8) {
            oct.push_back(make_int4(lc[0], lc[1], lc[2], lc[3]));
            oct.push_back(make_int4(lc[4], lc[5], lc[6], lc[7]));
        } else {
            set_error("unexpected multiplicity %d of a free node", cnt);
            return NB_ERR_MESH;
        }
    }
    m->n_zero = (int64_t)zero.size();
    m->n_pair = (int64_t)pair.size();
    m->n_quad = (int64_t)quad.size();
    m->n_oct = (int64_t)oct.size() / 2;
    NB_CUDA(cudaMalloc(&m->gs_zero, sizeof(int32_t) * std::max<size_t>(zero.size(), 1)));
    NB_CUDA(cudaMalloc(&m->gs_pair, sizeof(int2) * std::max<size_t>(pair.size(), 1)));
    NB_CUDA(cudaMalloc(&m->gs_quad, sizeof(int4) * std::max<size_t>(quad.size(), 1)));
    NB_CUDA(cudaMalloc(&m->gs_oct, sizeof(int4) * std::max<size_t>(oct.size(), 1)));
    if (!zero.empty())
        NB_CUDA(cudaMemcpyAsync(m->gs_zero, zero.data(), sizeof(int32_t) * zero.size(),
                                cudaMemcpyHostToDevice, s));
    if (!pair.empty())
        NB_CUDA(cudaMemcpyAsync(m->gs_pair, pair.data(), sizeof(int2) * pair.size(),
                                cudaMemcpyHostToDevice, s));
    if (!quad.empty())
        NB_CUDA(cudaMemcpyAsync(m->gs_quad, quad.data(), sizeof(int4) * quad.size(),
                                cudaMemcpyHostToDevice, s));
    if (!oct.empty())
        NB_CUDA(cudaMemcpyAsync(m->gs_oct, oct.data(), sizeof(int4) * oct.size(),
                                cudaMemcpyHostToDevice, s));
    NB_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
    // Jacobi: local diagonal, assembled and masked, inverted
    double *diag = nullptr;
    NB_CUDA(cudaMalloc(&diag, sizeof(double) * nL));
    NB_CUDA(cudaMalloc(&m->dinv64, sizeof(double) * nL));
    NB_CUDA(cudaMalloc(&m->dinv32, sizeof(float) * nL));
    NB_CUDA(cudaMalloc(&m->ones64, sizeof(double) * nL));
    NB_CUDA(cudaMalloc(&m->ones32, sizeof(float) * nL));
    m->gs_ready = true;
    nb_status st = local_diag(m, diag, s);
    if (st == NB_OK) st = dssum(m, NB_FP64, diag, 1, s);
    if (st == NB_OK && (m->iface_lo || m->iface_hi)) {
        // a slab keeps its own part of the diagonal: the interface planes
        // still lack the neighbour's (nb_slab_finish_diag adds it)
        if (cudaMalloc(&m->diag_asm, sizeof(double) * nL) != cudaSuccess) st = NB_ERR_OOM;
        else if (cudaMemcpyAsync(m->diag_asm, diag, sizeof(double) * nL,
                                 cudaMemcpyDeviceToDevice, s) != cudaSuccess) st = NB_ERR_CUDA;
    }
    if (st == NB_OK) st = finish_jacobi(m, diag, s);
    cudaError_t e1 = cudaStreamSynchronize(s);
    cudaFree(diag);
    if (st != NB_OK) { m->gs_ready = false; return st; }
    if (e1 != cudaSuccess) {
        m->gs_ready = false;
        set_error("jacobi set-up: %s", cudaGetErrorString(e1));
        return NB_ERR_CUDA;
    }
    return NB_OK;
}

}  // namespace nb
