// One-level overlapping Schwarz preconditioner with fast-diagonalisation
// local solves (the smoother of Nekbone's multigrid preconditioner; the paper
// names its routines -- h1mg_schwarz, h1mg_fdm, h1mg_extrude, h1mg_do_fast,
// h1mg_tnsr3d_el -- in Section 4.1 without the algorithm; this is the
// textbook method, Fischer 1997, with minimal overlap):
//   z = sum_e R_e^T A_e^-1 R_e r,
// R_e the restriction of the global vector to element e extended by one GLL
// node layer into each neighbour ((n+2)^3 points of the global GLL lattice),
// A_e the separable operator Bz(x)By(x)Ax + Bz(x)Ay(x)Bx + Az(x)By(x)Bx with the
// 1D stiffness / mass matrices assembled over the element and its neighbours
// in each direction on the undeformed box, inverted by fast diagonalisation
// (Ad S = Bd S Lam, S^T Bd S = I; Lynch, Rice and Thomas 1964).
//
// Per application, three kernels: the owner copies of r into a global vector;
// per element, the extended box gathered from it, six tensor contractions and
// the eigenvalue scaling in shared memory, the result stored per element; per
// local node, the sum of the results of the (at most 8) subdomains covering
// its lattice point in a fixed order, masked.  The 1D eigenproblems are
// solved once per mesh on the host (cyclic Jacobi rotations on
// B^-1/2 A B^-1/2, B diagonal) in binary64.
#include <math.h>

#include <algorithm>
#include <vector>

#include "nb_cg_dev.cuh"

namespace nb {

struct SchwarzData {
    int m = 0;           // n + 2 points per direction of an extended element
    float *S = nullptr;  // [3 dirs][4 variants][m][m]
    float *lam = nullptr;  // [3][4][m]
    float *rg = nullptr;   // [nG] owner values of r
    float *zt = nullptr;   // [E][m^3] local solutions
};

// Cyclic Jacobi eigenvalue iteration for a symmetric m x m matrix (Golub and
// Van Loan, Section 8.5): C = Q diag(ev) Q^T, Q in columns.
static void jacobi_eig(int m, std::vector<double> C, std::vector<double> &ev,
                       std::vector<double> &Q)
{
    Q.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                const double v = C[(size_t)i * m + j] * C[(size_t)i * m + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = C[(size_t)p * m + q];
                if (apq == 0.0) continue;
                const double app = C[(size_t)p * m + p], aqq = C[(size_t)q * m + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) /
                                 (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; ++k) {  // C <- J^T C J
                    const double ckp = C[(size_t)k * m + p], ckq = C[(size_t)k * m + q];
                    C[(size_t)k * m + p] = c * ckp - s * ckq;
                    C[(size_t)k * m + q] = s * ckp + c * ckq;
                }
                for (int k = 0; k < m; ++k) {
                    const double cpk = C[(size_t)p * m + k], cqk = C[(size_t)q * m + k];
                    C[(size_t)p * m + k] = c * cpk - s * cqk;
                    C[(size_t)q * m + k] = s * cpk + c * cqk;
                }
                for (int k = 0; k < m; ++k) {
                    const double qkp = Q[(size_t)k * m + p], qkq = Q[(size_t)k * m + q];
                    Q[(size_t)k * m + p] = c * qkp - s * qkq;
                    Q[(size_t)k * m + q] = s * qkp + c * qkq;
                }
            }
    }
    ev.resize(m);
    for (int i = 0; i < m; ++i) ev[i] = C[(size_t)i * m + i];
}

// Extended 1D operators of an element of length L (neighbours of the same
// length on the left / right when the flags are set) on the n+2 nodes
// [x_-1, x_0 .. x_N, x_N+1]; nodes without an unknown (outside the domain,
// the domain's Dirichlet face) are decoupled identity rows.  Out: S (m x m,
// row-major, S^T B S = I) and lam.
static void fdm_1d(int N, const std::vector<double> &K, const std::vector<double> &w, double L,
                   bool left, bool right, std::vector<double> &S, std::vector<double> &lam)
{
    const int n = N + 1, m = n + 2;
    std::vector<double> A((size_t)m * m, 0.0), B(m, 0.0);
    const double sk = 2.0 / L, sm = L / 2.0;
    auto addK = [&](int off, int i0, int cnt) {  // K rows/cols i0.. of an element at offset off
        for (int a = 0; a < cnt; ++a)
            for (int b = 0; b < cnt; ++b)
                A[(size_t)(off + a) * m + off + b] += sk * K[(size_t)(i0 + a) * n + i0 + b];
        for (int a = 0; a < cnt; ++a) B[off + a] += sm * w[i0 + a];
    };
    addK(1, 0, n);
    if (left) addK(0, N - 1, 2);
    if (right) addK(n, 0, 2);
    std::vector<bool> act(m, true);
    if (!left) act[0] = act[1] = false;
    if (!right) act[n] = act[n + 1] = false;
    for (int i = 0; i < m; ++i)
        if (!act[i]) {
            for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = A[(size_t)j * m + i] = 0.0;
            A[(size_t)i * m + i] = 1.0;
            B[i] = 1.0;
        }
    // C = B^-1/2 A B^-1/2 = Q diag(lam) Q^T, S = B^-1/2 Q
    std::vector<double> C((size_t)m * m), Q;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j)
            C[(size_t)i * m + j] = A[(size_t)i * m + j] / sqrt(B[i] * B[j]);
    jacobi_eig(m, C, lam, Q);
    S.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) S[(size_t)i * m + j] = Q[(size_t)i * m + j] / sqrt(B[i]);
}

// r's owner copies into the global vector.
__global__ void k_sw_global(int64_t nL, const float *__restrict__ r, const float *__restrict__ sgn,
                            const int32_t *__restrict__ gid, float *__restrict__ rg)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x)
        if (!signbit(sgn[l])) rg[gid[l]] = r[l];
}

// Variant of the 1D operators of element index e_d of n_d elements.
__device__ __forceinline__ int sw_variant(int e_d, int n_d)
{
    return (e_d == 0 ? 1 : 0) + (e_d == n_d - 1 ? 2 : 0);
}

// One line of a tensor contraction: out[q] = sum_i M[i][q] v[i], M in padded
// rows of P values (16-byte loads, the same row for every thread: broadcast).
template <int m, int P>
__device__ __forceinline__ void sw_line(const float *__restrict__ M, const float (&v)[m],
                                        float (&out)[m])
{
#pragma unroll
    for (int q = 0; q < m; ++q) out[q] = 0.f;
#pragma unroll
    for (int i = 0; i < m; ++i) {
        const float4 *row = reinterpret_cast<const float4 *>(M + i * P);
#pragma unroll
        for (int q4 = 0; q4 < P / 4; ++q4) {
            const float4 s = row[q4];
            if (4 * q4 + 0 < m) out[4 * q4 + 0] += s.x * v[i];
            if (4 * q4 + 1 < m) out[4 * q4 + 1] += s.y * v[i];
            if (4 * q4 + 2 < m) out[4 * q4 + 2] += s.z * v[i];
            if (4 * q4 + 3 < m) out[4 * q4 + 3] += s.w * v[i];
        }
    }
}

// A_e^-1 R_e r for every element: one block per element, one thread per line
// of the extended box (m^2 lines per direction), each contraction done by a
// thread for a whole line held in registers (the 1D matrices in shared
// memory, read as broadcast 16-byte rows).  Phases: a-lines (the gather from
// the global vector, S^T), b-lines (S^T), c-lines (S^T and the eigenvalue
// scaling), a-lines (S), b-lines (S), c-lines (S, stored).  zt[e][c][b][a].
template <int m>
__global__ void __launch_bounds__((m * m + 31) / 32 * 32)
k_sw_local(int64_t E, int nx, int ny, int nz, int N, const float *__restrict__ rg,
           const float *__restrict__ Sall, const float *__restrict__ lall,
           float *__restrict__ zt)
{
    constexpr int m2 = m * m, m3 = m2 * m, P = (m + 3) / 4 * 4;
    __shared__ __align__(16) float t0[m3], t1[m3];
    // per direction: S^T rows (M[i][q] = S[i][q]) and S rows (M[i][q] = S[q][i])
    __shared__ __align__(16) float St[3][m * P], Sf[3][m * P];
    __shared__ float lam[3][m];
    const int gxn = nx * N + 1, gyn = ny * N + 1, gzn = nz * N + 1;
    const int tid = threadIdx.x;
    const bool act = tid < m2;
    const int hi = act ? tid / m : 0, lo = act ? tid % m : 0;
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
        const int var[3] = {sw_variant(ex, nx), sw_variant(ey, ny), sw_variant(ez, nz)};
        __syncthreads();  // the previous element is done with the matrices
        for (int q = tid; q < 3 * m2; q += blockDim.x) {
            const int d = q / m2, r = q % m2, i = r / m, c = r % m;
            const float v = Sall[(d * 4 + var[d]) * m2 + r];  // S[i][c]
            St[d][i * P + c] = v;
            Sf[d][c * P + i] = v;
        }
        for (int q = tid; q < 3 * m; q += blockDim.x)
            lam[q / m][q % m] = lall[(q / m * 4 + var[q / m]) * m + q % m];
        __syncthreads();
        float v[m], o[m];
        // a-lines (c, b) = (hi, lo): the extended box row from the global lattice
        if (act) {
            const int gy = ey * N - 1 + lo, gz = ez * N - 1 + hi;
            const bool okyz = gy >= 0 && gy < gyn && gz >= 0 && gz < gzn;
#pragma unroll
            for (int a = 0; a < m; ++a) {
                const int gx = ex * N - 1 + a;
                v[a] = (okyz && gx >= 0 && gx < gxn) ? rg[((int64_t)gz * gyn + gy) * gxn + gx] : 0.f;
            }
            sw_line<m, P>(St[0], v, o);
#pragma unroll
            for (int a = 0; a < m; ++a) t0[(hi * m + lo) * m + a] = o[a];
        }
        __syncthreads();
        // b-lines (c, a) = (hi, lo)
        if (act) {
#pragma unroll
            for (int j = 0; j < m; ++j) v[j] = t0[(hi * m + j) * m + lo];
            sw_line<m, P>(St[1], v, o);
#pragma unroll
            for (int b = 0; b < m; ++b) t1[(hi * m + b) * m + lo] = o[b];
        }
        __syncthreads();
        // c-lines (b, a) = (hi, lo), then the scaling by 1 / (lx + ly + lz)
        if (act) {
#pragma unroll
            for (int k = 0; k < m; ++k) v[k] = t1[(k * m + hi) * m + lo];
            sw_line<m, P>(St[2], v, o);
            const float lab = lam[0][lo] + lam[1][hi];
#pragma unroll
            for (int c = 0; c < m; ++c) t0[(c * m + hi) * m + lo] = o[c] / (lab + lam[2][c]);
        }
        __syncthreads();
        // back: a-lines with S
        if (act) {
#pragma unroll
            for (int a = 0; a < m; ++a) v[a] = t0[(hi * m + lo) * m + a];
            sw_line<m, P>(Sf[0], v, o);
#pragma unroll
            for (int a = 0; a < m; ++a) t1[(hi * m + lo) * m + a] = o[a];
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int j = 0; j < m; ++j) v[j] = t1[(hi * m + j) * m + lo];
            sw_line<m, P>(Sf[1], v, o);
#pragma unroll
            for (int b = 0; b < m; ++b) t0[(hi * m + b) * m + lo] = o[b];
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int k = 0; k < m; ++k) v[k] = t0[(k * m + hi) * m + lo];
            sw_line<m, P>(Sf[2], v, o);
            float *out = zt + e * m3;
#pragma unroll
            for (int c = 0; c < m; ++c) out[(c * m + hi) * m + lo] = o[c];
        }
    }
}

// z[l] = mask * sum over the subdomains covering l's lattice point of their
// local solutions there, subdomains in ascending element order.
__global__ void k_sw_sum(int64_t nL, int nx, int ny, int nz, int N, int m,
                         const float *__restrict__ zt, const float *__restrict__ sgn,
                         float *__restrict__ z)
{
    const int n = N + 1, n3 = n * n * n, m3 = m * m * m;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / n3;
        const int q = (int)(l - e * n3);
        const int i = q % n, j = (q / n) % n, k = q / (n * n);
        const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
        const int gx = ex * N + i, gy = ey * N + j, gz = ez * N + k;
        float s = 0.f;
        if (sgn[l] != 0.f) {  // masked (Dirichlet) copies stay zero
            // elements e' with e'N - 1 <= g <= e'N + N + 1, per direction
            const int x0 = max(0, (gx - N - 1 + N - 1) / N), x1 = min(nx - 1, (gx + 1) / N);
            const int y0 = max(0, (gy - N - 1 + N - 1) / N), y1 = min(ny - 1, (gy + 1) / N);
            const int z0 = max(0, (gz - N - 1 + N - 1) / N), z1 = min(nz - 1, (gz + 1) / N);
            for (int cz = z0; cz <= z1; ++cz)
                for (int cy = y0; cy <= y1; ++cy)
                    for (int cx = x0; cx <= x1; ++cx) {
                        const int a = gx - (cx * N - 1), b = gy - (cy * N - 1), c = gz - (cz * N - 1);
                        if (a < 0 || a >= m || b < 0 || b >= m || c < 0 || c >= m) continue;
                        const int64_t ee = ((int64_t)cz * ny + cy) * nx + cx;
                        s += zt[ee * m3 + (c * m + b) * m + a];
                    }
        }
        z[l] = s;
    }
}

static nb_status sw_launch_local(int m, int grid, int64_t E, int nx, int ny, int nz, int N,
                                 const float *rg, const float *S, const float *lam, float *zt,
                                 cudaStream_t s)
{
#define NB_SW(MM) k_sw_local<MM><<<grid, (MM * MM + 31) / 32 * 32, 0, s>>>(E, nx, ny, nz, N, rg, S, lam, zt)
    switch (m) {
        case 4: NB_SW(4); break;
        case 5: NB_SW(5); break;
        case 6: NB_SW(6); break;
        case 7: NB_SW(7); break;
        case 8: NB_SW(8); break;
        case 9: NB_SW(9); break;
        case 10: NB_SW(10); break;
        case 11: NB_SW(11); break;
        case 12: NB_SW(12); break;
        case 13: NB_SW(13); break;
        case 14: NB_SW(14); break;
        default:
            set_error("Schwarz preconditioner supports orders N = 1..11");
            return NB_ERR_ARG;
    }
#undef NB_SW
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

void schwarz_free(nb_mesh *m)
{
    SchwarzData *d = (SchwarzData *)m->schwarz;
    if (!d) return;
    cudaFree(d->S);
    cudaFree(d->lam);
    cudaFree(d->rg);
    cudaFree(d->zt);
    delete d;
    m->schwarz = nullptr;
}

// The 1D eigenproblems and the scratch of the mesh (once).
nb_status schwarz_setup(nb_mesh *m)
{
    if (m->schwarz) return NB_OK;
    if (m->N < 1 || m->N > 11) {
        set_error("Schwarz preconditioner supports orders N = 1..11");
        return NB_ERR_ARG;
    }
    const int N = m->N, n = N + 1, mm = n + 2;
    std::vector<double> xi(n), w(n), D((size_t)n * n), K((size_t)n * n, 0.0);
    NB_TRY(gll_host(N, xi.data(), w.data()));
    deriv_host(N, xi.data(), D.data());
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int q = 0; q < n; ++q) s += w[q] * D[(size_t)q * n + i] * D[(size_t)q * n + j];
            K[(size_t)i * n + j] = s;
        }
    std::vector<float> Sh((size_t)3 * 4 * mm * mm), lh((size_t)3 * 4 * mm);
    const int cnt[3] = {m->nx, m->ny, m->nz};
    for (int dir = 0; dir < 3; ++dir)
        for (int v = 0; v < 4; ++v) {
            std::vector<double> S, lam;
            fdm_1d(N, K, w, 1.0 / cnt[dir], !(v & 1), !(v & 2), S, lam);
            for (int q = 0; q < mm * mm; ++q) Sh[((size_t)dir * 4 + v) * mm * mm + q] = (float)S[q];
            for (int q = 0; q < mm; ++q) lh[((size_t)dir * 4 + v) * mm + q] = (float)lam[q];
        }
    SchwarzData *d = new SchwarzData();
    d->m = mm;
    m->schwarz = d;
    const size_t m3 = (size_t)mm * mm * mm;
    cudaError_t e = cudaMalloc(&d->S, sizeof(float) * Sh.size());
    if (e == cudaSuccess) e = cudaMalloc(&d->lam, sizeof(float) * lh.size());
    if (e == cudaSuccess) e = cudaMalloc(&d->rg, sizeof(float) * m->nG);
    if (e == cudaSuccess) e = cudaMalloc(&d->zt, sizeof(float) * m3 * m->E);
    if (e == cudaSuccess)
        e = cudaMemcpy(d->S, Sh.data(), sizeof(float) * Sh.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d->lam, lh.data(), sizeof(float) * lh.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        schwarz_free(m);
        set_error("Schwarz set-up: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA;
    }
    return NB_OK;
}

// z = M r for FP32 L-vectors r (continuous, masked).
nb_status schwarz_apply(nb_mesh *m, const float *r, float *z, cudaStream_t s)
{
    SchwarzData *d = (SchwarzData *)m->schwarz;
    const int g = vec_grid(m->ctx, m->nL);
    k_sw_global<<<g, kVecThreads, 0, s>>>(m->nL, r, m->dinv32, m->gid, d->rg);
    NB_CUDA(cudaGetLastError());
    const int grid = (int)std::min<int64_t>(m->E, (int64_t)m->ctx->sm_count * 12);
    NB_TRY(sw_launch_local(d->m, grid, m->E, m->nx, m->ny, m->nz, m->N, d->rg, d->S, d->lam,
                           d->zt, s));
    k_sw_sum<<<g, kVecThreads, 0, s>>>(m->nL, m->nx, m->ny, m->nz, m->N, d->m, d->zt, m->dinv32, z);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

}  // namespace nb

using namespace nb;

extern "C" nb_status nb_schwarz_apply(nb_mesh *m, const float *r_dev, float *z_dev)
{
    if (!m || !r_dev || !z_dev) {
        set_error("invalid argument: NULL mesh or vector");
        return NB_ERR_ARG;
    }
    if (!m->gs_ready) {
        set_error("call nb_setup_gs first");
        return NB_ERR_STATE;
    }
    NB_CUDA(cudaSetDevice(m->ctx->device));
    NB_TRY(schwarz_setup(m));
    NB_TRY(schwarz_apply(m, r_dev, z_dev, m->ctx->stream));
    NB_CUDA(cudaStreamSynchronize(m->ctx->stream));
    return NB_OK;
}
