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
// Per application, three kernels: the owner copies of r into a global vector
// (inside flexible CG, the update kernel writes them); per element, the
// extended box gathered from it, six tensor contractions (one thread per line)
// and the eigenvalue scaling, the result stored per element; per element
// block, the sum at each node of the results of the (at most 8) subdomains
// covering its lattice point in a fixed order, masked (inside flexible CG with
// the step's dot products).  The 1D eigenproblems are
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
    float *zt = nullptr;   // [E][m][Mp][Mp] local solutions, [c][b][a], rows padded to Mp
    int grid_local = 1;    // blocks of k_sw_local
    int grid_sum[2] = {1, 1};  // blocks of k_sw_sum without / with the coarse
                               // level (at most kMaxPartials / 2)
    // coarse level (two-level form): interior element vertices per direction,
    // the 1D Galerkin eigenproblems Kc s = lam Mc s (S^T Mc S = I), the GLL
    // points for the vertex hats, the y/x-restricted residual and the coarse
    // solution
    bool coarse = false;
    int nc[3] = {0, 0, 0};
    float *Sc = nullptr;    // [3][kCoarseDir^2], S[v][q] row-major per direction
    float *lamc = nullptr;  // [3][kCoarseDir]
    float *xi = nullptr;    // [N + 1]
    float *t2 = nullptr;    // [gz][vy][vx]
    float *rc = nullptr;    // [vz][vy][vx] restricted residual
    float *zc = nullptr;    // [vz][vy][vx]
    // the same coarse level in FP64, for the outer correction of the
    // refinement (schwarz_coarse_correct64)
    double *Sc64 = nullptr, *lamc64 = nullptr, *xi64 = nullptr;
    double *rg64 = nullptr;  // [nG] the FP64 residual on the global lattice
    double *t1 = nullptr;    // [gz][gy][vx]
    double *t2d = nullptr;   // [gz][vy][vx]
    double *ca = nullptr, *cb = nullptr;  // [vz][vy][vx] coarse vectors
};

// Coarse level limits: interior vertices per direction, and in total (two
// buffers of them in one block's shared memory).
constexpr int kCoarseDir = 64;
constexpr int kCoarseTotal = 24576;

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

// Shapes of the local-solve kernel for m = n + 2 points per direction.  A
// phase contracts the outer axis X of a box stored as [X][Y][Z] (strides SX,
// SY, 1) with a 1D matrix M[i][q] (rows padded to Mp = m rounded up to 4) and
// stores the result as [Y][Z][X'], which is the next phase's [X][Y][Z]: three
// phases rotate the axes back.  A thread owns 4 consecutive lines (Z) at one
// Y and all Mp outputs, so every 16-byte matrix row it reads serves 16 FMAs,
// and its 4 inputs at one i are one 16-byte load.  SY / 4 and SX / 4 are odd,
// so the 8 threads of a 16-byte access hit distinct bank groups.
template <int m>
struct SwCfg {
    static constexpr int Mp = (m + 3) / 4 * 4;
    static constexpr int Q = Mp / 4;
    static constexpr int SY = (Q % 2) ? Mp : Mp + 4;
    static constexpr int SX = ((Mp * SY / 4) % 2) ? Mp * SY : Mp * SY + 4;
    static constexpr int BUF = m * SX;             // floats per box buffer
    static constexpr int TPE = m * Q;              // threads per element
    static constexpr int MAT = 24 * m * Mp;        // 3 dirs x 4 variants x (S^T, S) rows
    static constexpr int LAM = 12 * Mp;            // 3 dirs x 4 variants
    static constexpr int EPB0 = (100 * 1024 / 4 - MAT - LAM) / (2 * BUF);
    static constexpr int EPB1 = 256 / TPE;
    static constexpr int EPB = EPB0 < EPB1 ? (EPB0 < 1 ? 1 : EPB0) : EPB1;  // elements per block
    static constexpr int THREADS = EPB * TPE;
    static constexpr size_t SMEM = sizeof(float) * (size_t)(MAT + LAM + 2 * EPB * BUF);
    static constexpr int ZS = m * Mp * Mp;         // floats per element of zt: [c][b][a]
};

// acc[z][q] = sum_i M[i][q] in[i][Y][4 Zq + z]
template <int m>
__device__ __forceinline__ void sw_phase(const float *__restrict__ in, const float *__restrict__ M,
                                         int Y, int Zq, float (&acc)[4][SwCfg<m>::Mp])
{
    using C = SwCfg<m>;
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int q = 0; q < C::Mp; ++q) acc[z][q] = 0.f;
#pragma unroll 4
    for (int i = 0; i < m; ++i) {
        const float4 v = *reinterpret_cast<const float4 *>(in + i * C::SX + Y * C::SY + 4 * Zq);
#pragma unroll
        for (int qq = 0; qq < C::Q; ++qq) {
            const float4 w = *reinterpret_cast<const float4 *>(M + i * C::Mp + 4 * qq);
            acc[0][4 * qq + 0] += v.x * w.x; acc[0][4 * qq + 1] += v.x * w.y;
            acc[0][4 * qq + 2] += v.x * w.z; acc[0][4 * qq + 3] += v.x * w.w;
            acc[1][4 * qq + 0] += v.y * w.x; acc[1][4 * qq + 1] += v.y * w.y;
            acc[1][4 * qq + 2] += v.y * w.z; acc[1][4 * qq + 3] += v.y * w.w;
            acc[2][4 * qq + 0] += v.z * w.x; acc[2][4 * qq + 1] += v.z * w.y;
            acc[2][4 * qq + 2] += v.z * w.z; acc[2][4 * qq + 3] += v.z * w.w;
            acc[3][4 * qq + 0] += v.w * w.x; acc[3][4 * qq + 1] += v.w * w.y;
            acc[3][4 * qq + 2] += v.w * w.z; acc[3][4 * qq + 3] += v.w * w.w;
        }
    }
}

// out[Y][4 Zq + z][q] = acc[z][q] in the rotated layout (strides SX, SY).
template <int m>
__device__ __forceinline__ void sw_store(float *__restrict__ out, const float (&acc)[4][SwCfg<m>::Mp],
                                         int Y, int Zq)
{
    using C = SwCfg<m>;
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
        for (int qq = 0; qq < C::Q; ++qq)
            *reinterpret_cast<float4 *>(out + Y * C::SX + (4 * Zq + z) * C::SY + 4 * qq) =
                make_float4(acc[z][4 * qq], acc[z][4 * qq + 1], acc[z][4 * qq + 2], acc[z][4 * qq + 3]);
}

// A_e^-1 R_e r for every element.  EPB elements per block, TPE threads each;
// the 1D matrices of all variants stay in shared memory for the block's life.
// Per element: the extended box gathered from the global vector as [c][b][a],
// then six phases -- S_z^T, S_y^T, S_x^T with the eigenvalue scaling, S_z,
// S_y, S_x -- the last stored to zt[e][c][b][a] (row stride Mp).
template <int m>
__global__ void __launch_bounds__(SwCfg<m>::THREADS)
k_sw_local(int64_t E, int nx, int ny, int nz, int N, const float *__restrict__ rg,
           const float *__restrict__ Sall, const float *__restrict__ lall,
           float *__restrict__ zt, const CgScalars *sc)
{
    using C = SwCfg<m>;
    constexpr int m2 = m * m, Mp = C::Mp;
    extern __shared__ __align__(16) float sw_smem[];
    float *mat = sw_smem;                 // [(dir * 4 + var) * 2 + (0: S^T, 1: S)][m][Mp]
    float *lam = mat + C::MAT;            // [dir * 4 + var][Mp], padding 1
    const int tid = threadIdx.x;
    const int slot = tid / C::TPE, lt = tid - slot * C::TPE;
    const int Zq = lt / m, Y = lt - Zq * m;
    float *A = lam + C::LAM + slot * 2 * C::BUF, *B = A + C::BUF;
    if (sc && sc->done) return;  // the flexible-CG loop has stopped
    for (int q = tid; q < C::MAT; q += blockDim.x) mat[q] = 0.f;
    __syncthreads();
    for (int q = tid; q < 12 * m2; q += blockDim.x) {
        const int dv = q / m2, r = q - dv * m2, i = r / m, c = r - i * m;
        const float v = Sall[q];  // S[i][c] of direction / variant dv
        mat[(dv * 2 + 0) * m * Mp + i * Mp + c] = v;
        mat[(dv * 2 + 1) * m * Mp + c * Mp + i] = v;
    }
    for (int q = tid; q < C::LAM; q += blockDim.x) {
        const int dv = q / Mp, c = q - dv * Mp;
        lam[q] = c < m ? lall[dv * m + c] : 1.f;
    }
    __syncthreads();
    const int gxn = nx * N + 1, gyn = ny * N + 1, gzn = nz * N + 1;
    for (int64_t e0 = (int64_t)blockIdx.x * C::EPB; e0 < E; e0 += (int64_t)gridDim.x * C::EPB) {
        const int64_t e = e0 + slot;
        const bool ok = e < E;
        const int ex = ok ? (int)(e % nx) : 0, ey = ok ? (int)((e / nx) % ny) : 0;
        const int ez = ok ? (int)(e / ((int64_t)nx * ny)) : 0;
        const int vx = sw_variant(ex, nx), vy = sw_variant(ey, ny), vz = sw_variant(ez, nz);
        if (ok) {  // one row (c, b) of the box per thread and pass: m loads in flight
            const int gx0 = ex * N - 1;
            for (int rr = lt; rr < m2; rr += C::TPE) {
                const int c = rr / m, b = rr - c * m;
                const int gy = ey * N - 1 + b, gz = ez * N - 1 + c;
                const bool row = gy >= 0 && gy < gyn && gz >= 0 && gz < gzn;
                const int64_t r0 = ((int64_t)gz * gyn + gy) * gxn + gx0;
                float v[m];
#pragma unroll
                for (int a = 0; a < m; ++a)
                    v[a] = (row && gx0 + a >= 0 && gx0 + a < gxn) ? rg[r0 + a] : 0.f;
                float *dst = A + c * C::SX + b * C::SY;
#pragma unroll
                for (int a = 0; a < Mp; ++a) dst[a] = a < m ? v[a] : 0.f;
            }
        }
        __syncthreads();
        // phases 0..5: S_z^T, S_y^T, S_x^T (then the eigenvalue scaling), S_z,
        // S_y, S_x; buffers A -> B -> A ...; one copy of the phase code
#pragma unroll 1
        for (int ph = 0; ph < 6; ++ph) {
            const int dir = 2 - ph % 3, var = dir == 0 ? vx : (dir == 1 ? vy : vz);
            const float *in = (ph & 1) ? B : A;
            float *out = (ph & 1) ? A : B;
            if (ok) {
                float acc[4][Mp];
                sw_phase<m>(in, mat + ((dir * 4 + var) * 2 + ph / 3) * m * Mp, Y, Zq, acc);
                if (ph == 2) {  // 1 / (lx[a] + ly[b] + lz[c]) with (Y, Z, X') = (c, b, a)
                    const float *lx = lam + (0 * 4 + vx) * Mp, *ly = lam + (1 * 4 + vy) * Mp;
                    const float lz = lam[(2 * 4 + vz) * Mp + Y];
#pragma unroll
                    for (int z = 0; z < 4; ++z) {
                        const float lyz = lz + ly[4 * Zq + z];
#pragma unroll
                        for (int q = 0; q < Mp; ++q) acc[z][q] = __fdividef(acc[z][q], lyz + lx[q]);
                    }
                }
                if (ph < 5) {
                    sw_store<m>(out, acc, Y, Zq);
                } else {  // zt[e][c][b][a] with (Y, Z, X') = (c, b, a)
                    float *o = zt + e * C::ZS + Y * Mp * Mp;
#pragma unroll
                    for (int z = 0; z < 4; ++z)
                        if (4 * Zq + z < m)
#pragma unroll
                            for (int qq = 0; qq < C::Q; ++qq)
                                *reinterpret_cast<float4 *>(o + (4 * Zq + z) * Mp + 4 * qq) =
                                    make_float4(acc[z][4 * qq], acc[z][4 * qq + 1],
                                                acc[z][4 * qq + 2], acc[z][4 * qq + 3]);
                }
            }
            if (ph < 5) __syncthreads();
        }
    }
}

// z[l] = mask * sum over the subdomains covering l's lattice point of their
// local solutions there, subdomains in ascending element order.  One block
// per element (grid-stride), its threads over the element's n^3 nodes.  With
// DOTS, also the partials of (z, w_prev) (w_prev unassembled) and (r, z), and the last
// block forms the flexible-CG beta = -(z, w_prev) / pap_prev (0 on the first
// step) and rtz = (r, z).
template <int n, bool DOTS, bool COARSE>
__global__ void __launch_bounds__(256)
k_sw_sum(int64_t E, int nx, int ny, int nz, const float *__restrict__ zt,
         const float *__restrict__ sgn, float *__restrict__ z, const float *__restrict__ r,
         const float *__restrict__ wold, CgScalars *sc, double *__restrict__ part,
         const float *__restrict__ zc, const float *__restrict__ xi)
{
    constexpr int N = n - 1, n3 = n * n * n, Mp = SwCfg<n + 2>::Mp, ZS = SwCfg<n + 2>::ZS;
    // subdomains covering a node per direction: 2 for N >= 3 (3 for N = 2, 4 for N = 1)
    constexpr int KD = N >= 3 ? 2 : (N == 2 ? 3 : 4);
    constexpr int QS = (n3 + 255) / 256;  // nodes of an element per thread (256 threads)
    __shared__ double sred[32];
    if (DOTS && sc->done) return;
    // offsets in zt (E * ZS < 2^31, checked at set-up) of the same lattice
    // point in the next element along x, y, z
    const int dX = ZS - N, dY = nx * ZS - N * Mp, dZ = nx * ny * ZS - N * Mp * Mp;
    DotAcc<float> zw, rz;
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
        const int eo = (int)e * ZS;
        // coarse level: the coarse solution at the element's 8 vertices (0 on
        // the boundary: interior vertex (ex + cx - 1, ...) of nx - 1 per row)
        float zv[2][2][2];
#pragma unroll
        for (int cz = 0; cz < 2; ++cz)
#pragma unroll
            for (int cy = 0; cy < 2; ++cy)
#pragma unroll
                for (int cx = 0; cx < 2; ++cx) {
                    const int vx = ex + cx - 1, vy = ey + cy - 1, vz = ez + cz - 1;
                    const bool in = COARSE && vx >= 0 && vx < nx - 1 && vy >= 0 && vy < ny - 1 &&
                                    vz >= 0 && vz < nz - 1;
                    zv[cz][cy][cx] = in ? zc[((int64_t)vz * (ny - 1) + vy) * (nx - 1) + vx] : 0.f;
                }
#pragma unroll
        for (int s = 0; s < QS; ++s) {
            const int q = threadIdx.x + 256 * s;
            if (q >= n3) break;
            const int i = q % n, j = (q / n) % n, k = q / (n * n);
            // subdomain c covers offset g - (c N - 1) in [0, N + 2]: lower
            // neighbours down to e_d - (N + 1 - i) / N, upper up to e_d + (i + 1) / N
            const int lx = min((N + 1 - i) / N, ex), hx = min((i + 1) / N, nx - 1 - ex);
            const int ly = min((N + 1 - j) / N, ey), hy = min((j + 1) / N, ny - 1 - ey);
            const int lz = min((N + 1 - k) / N, ez), hz = min((k + 1) / N, nz - 1 - ez);
            // the own subdomain's [k + 1][j + 1][i + 1], moved to the lowest covering one
            const int p0 = eo + ((k + 1) * Mp + j + 1) * Mp + i + 1 - lx * dX - ly * dY - lz * dZ;
            // all loads issued before the sum, which runs in ascending element order
            float v[KD][KD][KD];
#pragma unroll
            for (int tz = 0; tz < KD; ++tz)
#pragma unroll
                for (int ty = 0; ty < KD; ++ty)
#pragma unroll
                    for (int tx = 0; tx < KD; ++tx) {
                        const bool ok = tz <= lz + hz && ty <= ly + hy && tx <= lx + hx;
                        v[tz][ty][tx] = ok ? zt[p0 + tx * dX + ty * dY + tz * dZ] : 0.f;
                    }
            const int64_t l = e * n3 + q;
            const float sg = sgn[l];
            float sum = 0.f;
#pragma unroll
            for (int tz = 0; tz < KD; ++tz)
#pragma unroll
                for (int ty = 0; ty < KD; ++ty)
#pragma unroll
                    for (int tx = 0; tx < KD; ++tx) sum += v[tz][ty][tx];
            if (COARSE) {  // + R_0^T z_c: trilinear interpolation of the vertex values
                const float ax = 0.5f * (1.f + xi[i]), ay = 0.5f * (1.f + xi[j]),
                            az = 0.5f * (1.f + xi[k]);
                const float y00 = zv[0][0][0] + ax * (zv[0][0][1] - zv[0][0][0]);
                const float y01 = zv[0][1][0] + ax * (zv[0][1][1] - zv[0][1][0]);
                const float y10 = zv[1][0][0] + ax * (zv[1][0][1] - zv[1][0][0]);
                const float y11 = zv[1][1][0] + ax * (zv[1][1][1] - zv[1][1][0]);
                const float z0 = y00 + ay * (y01 - y00), z1 = y10 + ay * (y11 - y10);
                sum += z0 + az * (z1 - z0);
            }
            sum = sg != 0.f ? sum : 0.f;  // masked (Dirichlet) copies are zero
            z[l] = sum;
            if (DOTS) {
                // (z, w_prev) over every copy: w_prev is the unassembled
                // A_L p of the previous step (z continuous); (r, z) over
                // owner copies
                zw.add(sum * wold[l]);
                if (!signbit(sg)) rz.add(r[l] * sum);
            }
        }
    }
    if (!DOTS) return;
    const double tzw = block_sum_acc(zw, sred);
    const double trz = block_sum_acc(rz, sred);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = tzw;
        part[gridDim.x + blockIdx.x] = trz;
    }
    if (last_block(&sc->tick_upd)) {
        double szw, srz;
        sum_partials2(part, part + gridDim.x, gridDim.x, sred, szw, srz);
        if (threadIdx.x == 0) {
            sc->beta = sc->pap_prev > 0.0 ? -szw / sc->pap_prev : 0.0;  // 0: first step
            sc->rtz = srz;
            sc->rp = srz;
            if (!isfinite(sc->beta) || !isfinite(srz) || !(srz > 0.0)) {
                sc->done = 1;
                sc->status = NB_BREAKDOWN;
            }
        }
    }
}

// mode 0: grid of k_sw_sum<n, true> (resident blocks x SMs, one wave) out;
// 1: launch
template <bool DOTS>
static nb_status sw_sum(int mode, int m, int sms, int *grid, int64_t E, int nx, int ny, int nz,
                        const float *zt, const float *sgn, float *z, const float *r,
                        const float *wold, CgScalars *sc, double *part, cudaStream_t s,
                        const float *zc = nullptr, const float *xi = nullptr)
{
#define NB_SWS(NN)                                                                                \
    if (mode == 0) {                                                                              \
        int per_sm[2] = {0, 0};                                                                   \
        NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k_sw_sum<NN, true, false>, \
                                                              256, 0));                           \
        NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k_sw_sum<NN, true, true>, \
                                                              256, 0));                           \
        for (int c = 0; c < 2; ++c)                                                               \
            grid[c] = (int)std::max<int64_t>(1, std::min<int64_t>(E, (int64_t)sms *               \
                                                                      std::max(per_sm[c], 1)));   \
        return NB_OK;                                                                             \
    }                                                                                             \
    if (zc)                                                                                       \
        k_sw_sum<NN, DOTS, true><<<grid[1], 256, 0, s>>>(E, nx, ny, nz, zt, sgn, z, r, wold, sc,  \
                                                         part, zc, xi);                           \
    else                                                                                          \
        k_sw_sum<NN, DOTS, false><<<grid[0], 256, 0, s>>>(E, nx, ny, nz, zt, sgn, z, r, wold, sc, \
                                                          part, zc, xi);                          \
    NB_CUDA(cudaGetLastError());                                                                  \
    return NB_OK
    switch (m - 2) {
        case 2: { NB_SWS(2); }
        case 3: { NB_SWS(3); }
        case 4: { NB_SWS(4); }
        case 5: { NB_SWS(5); }
        case 6: { NB_SWS(6); }
        case 7: { NB_SWS(7); }
        case 8: { NB_SWS(8); }
        case 9: { NB_SWS(9); }
        case 10: { NB_SWS(10); }
        case 11: { NB_SWS(11); }
        case 12: { NB_SWS(12); }
        default:
            set_error("Schwarz preconditioner supports orders N = 1..11");
            return NB_ERR_ARG;
    }
#undef NB_SWS
}

// Coarse restriction, x and y, one block per plane gz: t1[gy][vx] = sum over
// the 2N + 1 nodes of the hat's support of hat(gx) rg[gz][gy][gx] (rows read
// by warps), then t2[gz][vy][vx] = sum over gy of hat(gy) t1[gy][vx].  Every
// interior vertex's hat has the same 2N + 1 weights: (1 + xi_d)/2 for
// d = 0..N, (1 - xi_(d - N))/2 for d = N..2N.  rg holds each global node's
// value once.
__global__ void k_co_rxy(int gxn, int gyn, int N, int ncx, int ncy, const float *__restrict__ xi,
                         const float *__restrict__ rg, float *__restrict__ t2, const CgScalars *sc)
{
    if (sc && sc->done) return;
    extern __shared__ float co_rs[];
    float *hw = co_rs;               // [2N + 1]
    float *t1 = co_rs + 2 * N + 1;   // [gyn][ncx]
    for (int d = threadIdx.x; d <= 2 * N; d += blockDim.x)
        hw[d] = d <= N ? 0.5f * (1.f + xi[d]) : 0.5f * (1.f - xi[d - N]);
    __syncthreads();
    const int gz = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int gy = warp; gy < gyn; gy += nw) {
        const float *row = rg + ((int64_t)gz * gyn + gy) * gxn;
        for (int vx = lane; vx < ncx; vx += 32) {
            float acc = 0.f;
            for (int d = 0; d <= 2 * N; ++d) acc += hw[d] * row[vx * N + d];
            t1[gy * ncx + vx] = acc;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ncy * ncx; t += blockDim.x) {
        const int vx = t % ncx, vy = t / ncx;
        float acc = 0.f;
        for (int d = 0; d <= 2 * N; ++d) acc += hw[d] * t1[(vy * N + d) * ncx + vx];
        t2[((int64_t)gz * ncy + vy) * ncx + vx] = acc;
    }
}

// Coarse restriction, z: rc[vz][vy][vx] = sum over the 2N + 1 planes of the
// hat's support of hat(gz) t2[gz][vy][vx] (one thread per coarse unknown).
__global__ void k_co_rz(int N, int ncxy, int ncz, const float *__restrict__ xi,
                        const float *__restrict__ t2, float *__restrict__ rc, const CgScalars *sc)
{
    if (sc && sc->done) return;
    const int total = ncxy * ncz;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int vxy = t % ncxy, vz = t / ncxy;
        float acc = 0.f;
        for (int d = 0; d <= 2 * N; ++d) {
            const float h = d <= N ? 0.5f * (1.f + xi[d]) : 0.5f * (1.f - xi[d - N]);
            acc += h * t2[(int64_t)(vz * N + d) * ncxy + vxy];
        }
        rc[t] = acc;
    }
}

// One axis of a coarse tensor contraction in shared memory: out = sum over
// the axis of M[a][q] in[..a..] (M row-major [nc][nc]); axis 0 = x (fastest).
__device__ __forceinline__ void co_contract(const float *__restrict__ in, float *__restrict__ out,
                                            const float *__restrict__ M, bool trans, int axis,
                                            int nx, int ny, int nz)
{
    const int total = nx * ny * nz;
    const int na = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const int stride = axis == 0 ? 1 : (axis == 1 ? nx : nx * ny);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int x = t % nx, y = (t / nx) % ny, z = t / (nx * ny);
        const int q = axis == 0 ? x : (axis == 1 ? y : z);
        const int base = t - q * stride;
        float acc = 0.f;
        // trans: out[q] = sum_a M[a][q] in[a] (S^T); else out[q] = sum_a M[q][a] in[a] (S)
        for (int a = 0; a < na; ++a)
            acc += (trans ? M[a * na + q] : M[q * na + a]) * in[base + a * stride];
        out[t] = acc;
    }
}

// Coarse solve in one block: A_0^-1 rc by fast diagonalisation,
// (Sz(x)Sy(x)Sx) diag(1 / (lx + ly + lz)) (Sz(x)Sy(x)Sx)^T, into zc.
__global__ void k_co_solve(int ncx, int ncy, int ncz, const float *__restrict__ Sc,
                           const float *__restrict__ lamc, const float *__restrict__ rc,
                           float *__restrict__ zc, const CgScalars *sc)
{
    if (sc && sc->done) return;
    extern __shared__ __align__(16) float co_smem[];
    const int total = ncx * ncy * ncz;
    float *A = co_smem, *B = co_smem + total;
    const float *Sx = Sc, *Sy = Sc + kCoarseDir * kCoarseDir, *Sz = Sc + 2 * kCoarseDir * kCoarseDir;
    const float *lx = lamc, *ly = lamc + kCoarseDir, *lz = lamc + 2 * kCoarseDir;
    for (int t = threadIdx.x; t < total; t += blockDim.x) A[t] = rc[t];
    __syncthreads();
    co_contract(A, B, Sx, true, 0, ncx, ncy, ncz);
    __syncthreads();
    co_contract(B, A, Sy, true, 1, ncx, ncy, ncz);
    __syncthreads();
    co_contract(A, B, Sz, true, 2, ncx, ncy, ncz);
    __syncthreads();
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int x = t % ncx, y = (t / ncx) % ncy, z = t / (ncx * ncy);
        B[t] = B[t] / (lx[x] + ly[y] + lz[z]);
    }
    __syncthreads();
    co_contract(B, A, Sz, false, 2, ncx, ncy, ncz);
    __syncthreads();
    co_contract(A, B, Sy, false, 1, ncx, ncy, ncz);
    __syncthreads();
    co_contract(B, A, Sx, false, 0, ncx, ncy, ncz);
    __syncthreads();
    for (int t = threadIdx.x; t < total; t += blockDim.x) zc[t] = A[t];
}

// ---------------------------------------------------------------------------
// The coarse level in FP64, applied by the refinement to its FP64 residual
// (schwarz_coarse_correct64): restriction along x, y, z, the coarse solve by
// fast diagonalisation, and the trilinear prolongation to the local nodes.
// One thread per output value throughout.
// ---------------------------------------------------------------------------

// Weight of the hat of an interior vertex at the d-th of the 2N + 1 GLL nodes
// of its support: (1 + xi_d) / 2 on the element below the vertex, (1 - xi_(d-N))
// / 2 on the element above.
__device__ __forceinline__ double hat64(const double *xi, int N, int d)
{
    return d <= N ? 0.5 * (1.0 + xi[d]) : 0.5 * (1.0 - xi[d - N]);
}

// t1[gz][gy][vx] = sum_d hat(d) rg[gz][gy][vx N + d]
__global__ void k_c64_rx(int64_t rows, int gxn, int N, int ncx, const double *__restrict__ xi,
                         const double *__restrict__ rg, double *__restrict__ t1)
{
    const int64_t total = rows * ncx;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int vx = (int)(t % ncx);
        const int64_t row = t / ncx;
        const double *src = rg + row * gxn + (int64_t)vx * N;
        double acc = 0.0;
        for (int d = 0; d <= 2 * N; ++d) acc += hat64(xi, N, d) * src[d];
        t1[t] = acc;
    }
}

// out[o][v][q] = sum_d hat(d) in[o][v N + d][q] (the restriction along the
// middle axis of in[o][g][q], g of length gn)
__global__ void k_c64_rmid(int64_t outer, int gn, int nv, int nq, int N,
                           const double *__restrict__ xi, const double *__restrict__ in,
                           double *__restrict__ out)
{
    const int64_t total = outer * nv * nq;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(t % nq), v = (int)((t / nq) % nv);
        const int64_t o = t / ((int64_t)nq * nv);
        const double *src = in + (o * gn + (int64_t)v * N) * nq + q;
        double acc = 0.0;
        for (int d = 0; d <= 2 * N; ++d) acc += hat64(xi, N, d) * src[(int64_t)d * nq];
        out[t] = acc;
    }
}

// One axis of the coarse fast-diagonalisation solve on [vz][vy][vx]:
// out = S^T in (trans) or S in along the axis (0 = x), S[a][q] row-major
// (kCoarseDir columns); with lam, the result is divided by lx + ly + lz.
__global__ void k_c64_axis(int ncx, int ncy, int ncz, int axis, int trans,
                           const double *__restrict__ S, const double *__restrict__ lam,
                           const double *__restrict__ in, double *__restrict__ out)
{
    const int total = ncx * ncy * ncz;
    const int na = axis == 0 ? ncx : (axis == 1 ? ncy : ncz);
    const int stride = axis == 0 ? 1 : (axis == 1 ? ncx : ncx * ncy);
    const double *M = S + (size_t)axis * kCoarseDir * kCoarseDir;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int x = t % ncx, y = (t / ncx) % ncy, z = t / (ncx * ncy);
        const int q = axis == 0 ? x : (axis == 1 ? y : z);
        const int base = t - q * stride;
        double acc = 0.0;
        for (int a = 0; a < na; ++a)
            acc += (trans ? M[a * na + q] : M[q * na + a]) * in[base + a * stride];
        if (lam) acc /= lam[x] + lam[kCoarseDir + y] + lam[2 * kCoarseDir + z];
        out[t] = acc;
    }
}

// c = R_0^T zc at every local node (trilinear in the element's reference
// coordinates from its 8 vertices; boundary vertices carry 0, so c vanishes
// on the Dirichlet boundary), x += c, and c rounded to FP32 into c32.
__global__ void k_c64_prolong(int64_t nL, int nx, int ny, int N, const double *__restrict__ xi,
                              const double *__restrict__ zc, int ncx, int ncy, int ncz,
                              double *__restrict__ x, float *__restrict__ c32)
{
    const int n = N + 1, n3 = n * n * n;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / n3;
        const int q = (int)(l - e * n3), i = q % n, j = (q / n) % n, k = q / (n * n);
        const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
        const double wx[2] = {0.5 * (1.0 - xi[i]), 0.5 * (1.0 + xi[i])};
        const double wy[2] = {0.5 * (1.0 - xi[j]), 0.5 * (1.0 + xi[j])};
        const double wz[2] = {0.5 * (1.0 - xi[k]), 0.5 * (1.0 + xi[k])};
        double c = 0.0;
        for (int cz = 0; cz < 2; ++cz) {
            const int vz = ez + cz - 1;  // interior vertex index (vertex ez + cz)
            if (vz < 0 || vz >= ncz) continue;
            for (int by = 0; by < 2; ++by) {
                const int vy = ey + by - 1;
                if (vy < 0 || vy >= ncy) continue;
                for (int ax = 0; ax < 2; ++ax) {
                    const int vx = ex + ax - 1;
                    if (vx < 0 || vx >= ncx) continue;
                    c += wz[cz] * wy[by] * wx[ax] * zc[((int64_t)vz * ncy + vy) * ncx + vx];
                }
            }
        }
        x[l] += c;
        c32[l] = (float)c;
    }
}

// r64 -= w32 (the FP32 operator applied to the coarse correction) and the
// partials of (r, c, r), c = 1/multiplicity.
__global__ void k_c64_subnorm(int64_t nL, double *__restrict__ r64, const float *__restrict__ w32,
                              const float *__restrict__ c, double *__restrict__ part)
{
    __shared__ double sred[32];
    double a = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x) {
        const double v = r64[l] - (double)w32[l];
        r64[l] = v;
        a += (double)c[l] * v * v;
    }
    const double t = block_sum(a, sred);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Shared-memory limit and grid (resident blocks x SMs, at most one block
// per EPB elements) of k_sw_local<m>; set once per mesh, outside any capture.
template <int m>
static nb_status sw_local_prepare(int sms, int64_t E, int *grid)
{
    using C = SwCfg<m>;
    NB_CUDA(cudaFuncSetAttribute(k_sw_local<m>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)C::SMEM));
    int per_sm = 0;
    NB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sw_local<m>, C::THREADS,
                                                          C::SMEM));
    const int64_t groups = (E + C::EPB - 1) / C::EPB;
    *grid = (int)std::max<int64_t>(1, std::min<int64_t>(groups, (int64_t)sms * std::max(per_sm, 1)));
    return NB_OK;
}

// mode 0: prepare (grid out), 1: launch with that grid
static nb_status sw_local(int mode, int m, int sms, int *grid, int64_t E, int nx, int ny, int nz,
                          int N, const float *rg, const float *S, const float *lam, float *zt,
                          const CgScalars *sc, cudaStream_t s)
{
#define NB_SW(MM)                                                                                 \
    if (mode == 0) return sw_local_prepare<MM>(sms, E, grid);                                    \
    k_sw_local<MM><<<*grid, SwCfg<MM>::THREADS, SwCfg<MM>::SMEM, s>>>(E, nx, ny, nz, N, rg, S,   \
                                                                     lam, zt, sc);               \
    NB_CUDA(cudaGetLastError());                                                                 \
    return NB_OK
    switch (m) {
        case 4: { NB_SW(4); }
        case 5: { NB_SW(5); }
        case 6: { NB_SW(6); }
        case 7: { NB_SW(7); }
        case 8: { NB_SW(8); }
        case 9: { NB_SW(9); }
        case 10: { NB_SW(10); }
        case 11: { NB_SW(11); }
        case 12: { NB_SW(12); }
        case 13: { NB_SW(13); }
        case 14: { NB_SW(14); }
        default:
            set_error("Schwarz preconditioner supports orders N = 1..11");
            return NB_ERR_ARG;
    }
#undef NB_SW
}

// floats per element of the local solutions for m points per direction
static int64_t sw_zt_stride(int m)
{
    const int Mp = (m + 3) / 4 * 4;
    return (int64_t)m * Mp * Mp;
}

void schwarz_free(nb_mesh *m)
{
    SchwarzData *d = (SchwarzData *)m->schwarz;
    if (!d) return;
    cudaFree(d->S);
    cudaFree(d->lam);
    cudaFree(d->rg);
    cudaFree(d->zt);
    cudaFree(d->Sc);
    cudaFree(d->lamc);
    cudaFree(d->xi);
    cudaFree(d->t2);
    cudaFree(d->rc);
    cudaFree(d->zc);
    cudaFree(d->Sc64);
    cudaFree(d->lamc64);
    cudaFree(d->xi64);
    cudaFree(d->rg64);
    cudaFree(d->t1);
    cudaFree(d->t2d);
    cudaFree(d->ca);
    cudaFree(d->cb);
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
    if (m->E * sw_zt_stride(mm) >= ((int64_t)1 << 31)) {
        set_error("Schwarz preconditioner: at most %lld elements of order %d",
                  (long long)((((int64_t)1 << 31) - 1) / sw_zt_stride(mm)), N);
        return NB_ERR_ARG;
    }
    SchwarzData *d = new SchwarzData();
    d->m = mm;
    m->schwarz = d;
    const size_t m3 = (size_t)sw_zt_stride(mm);
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
    nb_status st = sw_local(0, mm, m->ctx->sm_count, &d->grid_local, m->E, 0, 0, 0, 0, nullptr,
                            nullptr, nullptr, nullptr, nullptr, nullptr);
    if (st == NB_OK)
        st = sw_sum<true>(0, mm, m->ctx->sm_count, d->grid_sum, m->E, 0, 0, 0, nullptr, nullptr,
                          nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (st != NB_OK) schwarz_free(m);
    return st;
}

// Generalised symmetric eigenproblem K s = lam M s of order m (M symmetric
// positive definite): S with S^T M S = I, S^T K S = diag(lam), through the
// Cholesky factor M = C C^T and cyclic Jacobi rotations on C^-1 K C^-T
// (Golub and Van Loan, Section 8.7).  S row-major [i][mode].
static bool gen_eig(int m, const std::vector<double> &K, const std::vector<double> &M,
                    std::vector<double> &S, std::vector<double> &lam)
{
    std::vector<double> C((size_t)m * m, 0.0);
    for (int j = 0; j < m; ++j)
        for (int i = j; i < m; ++i) {
            double v = M[(size_t)i * m + j];
            for (int k = 0; k < j; ++k) v -= C[(size_t)i * m + k] * C[(size_t)j * m + k];
            if (i == j) {
                if (!(v > 0.0)) return false;
                C[(size_t)j * m + j] = sqrt(v);
            } else {
                C[(size_t)i * m + j] = v / C[(size_t)j * m + j];
            }
        }
    // X = C^-1 K (forward substitution, column by column), W = C^-1 X^T
    std::vector<double> X((size_t)m * m), W((size_t)m * m);
    auto fsub = [&](const std::vector<double> &B, std::vector<double> &Y, bool transB) {
        for (int c = 0; c < m; ++c)
            for (int i = 0; i < m; ++i) {
                double v = transB ? B[(size_t)c * m + i] : B[(size_t)i * m + c];
                for (int k = 0; k < i; ++k) v -= C[(size_t)i * m + k] * Y[(size_t)k * m + c];
                Y[(size_t)i * m + c] = v / C[(size_t)i * m + i];
            }
    };
    fsub(K, X, false);
    fsub(X, W, true);
    for (int i = 0; i < m; ++i)  // symmetrise the rounding
        for (int j = 0; j < i; ++j) {
            const double a = 0.5 * (W[(size_t)i * m + j] + W[(size_t)j * m + i]);
            W[(size_t)i * m + j] = W[(size_t)j * m + i] = a;
        }
    std::vector<double> Y;
    jacobi_eig(m, W, lam, Y);  // W = Y diag(lam) Y^T
    // S = C^-T Y (back substitution with C^T, column by column)
    S.assign((size_t)m * m, 0.0);
    for (int c = 0; c < m; ++c)
        for (int i = m - 1; i >= 0; --i) {
            double v = Y[(size_t)i * m + c];
            for (int k = i + 1; k < m; ++k) v -= C[(size_t)k * m + i] * S[(size_t)k * m + c];
            S[(size_t)i * m + c] = v / C[(size_t)i * m + i];
        }
    return true;
}

// The coarse level of the mesh (once): per direction the hats of the n_d - 1
// interior vertices at the n_d N + 1 GLL nodes, the Galerkin 1D stiffness /
// mass Kc = R1 Kf R1^T, Mc = R1 Mf R1^T with Kf, Mf the GLL stiffness / mass
// assembled over the n_d elements of length 1 / n_d, and their generalised
// eigenvectors.  A direction with one element has no interior vertex: no
// coarse space (the correction is zero).
static nb_status schwarz_setup_coarse(nb_mesh *m)
{
    SchwarzData *d = (SchwarzData *)m->schwarz;
    if (d->coarse || d->Sc) return NB_OK;
    const int N = m->N, n = N + 1;
    const int cnt[3] = {m->nx, m->ny, m->nz};
    int64_t total = 1;
    for (int dir = 0; dir < 3; ++dir) {
        d->nc[dir] = cnt[dir] - 1;
        total *= d->nc[dir];
        if (d->nc[dir] > kCoarseDir) {
            set_error("two-level Schwarz: at most %d elements per direction", kCoarseDir + 1);
            return NB_ERR_ARG;
        }
    }
    if (total > kCoarseTotal) {
        set_error("two-level Schwarz: at most %d interior element vertices", kCoarseTotal);
        return NB_ERR_ARG;
    }
    std::vector<double> xi(n), w(n), D((size_t)n * n), K((size_t)n * n, 0.0);
    NB_TRY(gll_host(N, xi.data(), w.data()));
    deriv_host(N, xi.data(), D.data());
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s2 = 0.0;
            for (int q = 0; q < n; ++q) s2 += w[q] * D[(size_t)q * n + i] * D[(size_t)q * n + j];
            K[(size_t)i * n + j] = s2;
        }
    std::vector<float> Sh((size_t)3 * kCoarseDir * kCoarseDir, 0.f), lh((size_t)3 * kCoarseDir, 1.f);
    std::vector<double> Sh64(Sh.size(), 0.0), lh64(lh.size(), 1.0);
    for (int dir = 0; dir < 3 && total > 0; ++dir) {
        const int nd = cnt[dir], nc = nd - 1, ng = nd * N + 1;
        const double L = 1.0 / nd;
        std::vector<double> Kf((size_t)ng * ng, 0.0), Mf((size_t)ng * ng, 0.0), R((size_t)nc * ng, 0.0);
        for (int e = 0; e < nd; ++e)
            for (int i = 0; i < n; ++i) {
                Mf[(size_t)(e * N + i) * ng + e * N + i] += 0.5 * L * w[i];
                for (int j = 0; j < n; ++j)
                    Kf[(size_t)(e * N + i) * ng + e * N + j] += (2.0 / L) * K[(size_t)i * n + j];
            }
        for (int v = 0; v < nc; ++v)
            for (int i = 0; i < n; ++i) {
                R[(size_t)v * ng + v * N + i] = 0.5 * (1.0 + xi[i]);
                R[(size_t)v * ng + (v + 1) * N + i] = 0.5 * (1.0 - xi[i]);
            }
        std::vector<double> Kc((size_t)nc * nc, 0.0), Mc((size_t)nc * nc, 0.0);
        for (int a = 0; a < nc; ++a)
            for (int b = 0; b < nc; ++b) {
                double sk = 0.0, sm = 0.0;
                for (int g = a * N; g <= (a + 2) * N; ++g)
                    for (int h = b * N; h <= (b + 2) * N; ++h) {
                        const double rr = R[(size_t)a * ng + g] * R[(size_t)b * ng + h];
                        sk += rr * Kf[(size_t)g * ng + h];
                        sm += rr * Mf[(size_t)g * ng + h];
                    }
                Kc[(size_t)a * nc + b] = sk;
                Mc[(size_t)a * nc + b] = sm;
            }
        std::vector<double> S, lam;
        if (!gen_eig(nc, Kc, Mc, S, lam)) {
            set_error("two-level Schwarz: coarse mass matrix not positive definite");
            return NB_ERR_ARG;
        }
        for (int a = 0; a < nc; ++a) {
            lh[(size_t)dir * kCoarseDir + a] = (float)lam[a];
            lh64[(size_t)dir * kCoarseDir + a] = lam[a];
            for (int q = 0; q < nc; ++q) {
                Sh[(size_t)dir * kCoarseDir * kCoarseDir + a * nc + q] = (float)S[(size_t)a * nc + q];
                Sh64[(size_t)dir * kCoarseDir * kCoarseDir + a * nc + q] = S[(size_t)a * nc + q];
            }
        }
    }
    std::vector<float> xf(n);
    for (int i = 0; i < n; ++i) xf[i] = (float)xi[i];
    const int64_t gzn = (int64_t)m->nz * N + 1;
    cudaError_t e = cudaMalloc(&d->Sc, sizeof(float) * Sh.size());
    if (e == cudaSuccess) e = cudaMalloc(&d->lamc, sizeof(float) * lh.size());
    if (e == cudaSuccess) e = cudaMalloc(&d->xi, sizeof(float) * n);
    if (e == cudaSuccess)
        e = cudaMalloc(&d->t2, sizeof(float) * std::max<int64_t>(1, gzn * d->nc[1] * d->nc[0]));
    if (e == cudaSuccess) e = cudaMalloc(&d->zc, sizeof(float) * std::max<int64_t>(1, total));
    if (e == cudaSuccess) e = cudaMalloc(&d->rc, sizeof(float) * std::max<int64_t>(1, total));
    if (e == cudaSuccess)
        e = cudaMemcpy(d->Sc, Sh.data(), sizeof(float) * Sh.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d->lamc, lh.data(), sizeof(float) * lh.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d->xi, xf.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    // FP64 copies for the outer coarse correction
    const int64_t gxn = (int64_t)m->nx * N + 1, gyn = (int64_t)m->ny * N + 1;
    if (e == cudaSuccess) e = cudaMalloc(&d->Sc64, sizeof(double) * Sh64.size());
    if (e == cudaSuccess) e = cudaMalloc(&d->lamc64, sizeof(double) * lh64.size());
    if (e == cudaSuccess) e = cudaMalloc(&d->xi64, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d->rg64, sizeof(double) * gxn * gyn * gzn);
    if (e == cudaSuccess)
        e = cudaMalloc(&d->t1, sizeof(double) * std::max<int64_t>(1, gzn * gyn * d->nc[0]));
    if (e == cudaSuccess)
        e = cudaMalloc(&d->t2d, sizeof(double) * std::max<int64_t>(1, gzn * d->nc[1] * d->nc[0]));
    if (e == cudaSuccess) e = cudaMalloc(&d->ca, sizeof(double) * std::max<int64_t>(1, total));
    if (e == cudaSuccess) e = cudaMalloc(&d->cb, sizeof(double) * std::max<int64_t>(1, total));
    if (e == cudaSuccess)
        e = cudaMemcpy(d->Sc64, Sh64.data(), sizeof(double) * Sh64.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d->lamc64, lh64.data(), sizeof(double) * lh64.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d->xi64, xi.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_co_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * sizeof(float) * kCoarseTotal));
    if (e == cudaSuccess)  // the x-restricted plane of k_co_rxy
        e = cudaFuncSetAttribute(k_co_rxy, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float) * (2 * N + 1 + (int64_t)(m->ny * N + 1) *
                                                                      std::max(d->nc[0], 1))));
    if (e != cudaSuccess) {
        set_error("two-level Schwarz set-up: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA;
    }
    d->coarse = total > 0;
    return NB_OK;
}

float *schwarz_rg(nb_mesh *m) { return ((SchwarzData *)m->schwarz)->rg; }

// The owner values of the FP32 L-vector r into the global vector the local
// solves gather from.
nb_status schwarz_gather(nb_mesh *m, const float *r, cudaStream_t s)
{
    SchwarzData *d = (SchwarzData *)m->schwarz;
    k_sw_global<<<vec_grid(m->ctx, m->nL), kVecThreads, 0, s>>>(m->nL, r, m->dinv32, m->gid, d->rg);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// Local solves from the gathered global vector and their masked sum into z;
// with sc, also the flexible-CG dots of z with r and w_prev (partials in
// part, 2 x the sum's grid entries) and beta, rtz in sc.
nb_status schwarz_solve_sum(nb_mesh *m, const float *r, float *z, const float *wold,
                            CgScalars *sc, double *part, cudaStream_t s, bool coarse)
{
    SchwarzData *d = (SchwarzData *)m->schwarz;
    NB_TRY(sw_local(1, d->m, m->ctx->sm_count, &d->grid_local, m->E, m->nx, m->ny, m->nz, m->N,
                    d->rg, d->S, d->lam, d->zt, sc, s));
    const float *zc = nullptr;
    if (coarse && d->coarse) {  // R_0 r (x, y; then z and A_0^-1 in one block)
        const int N = m->N, gxn = m->nx * N + 1, gyn = m->ny * N + 1, gzn = m->nz * N + 1;
        const size_t rs = sizeof(float) * (2 * N + 1 + (size_t)gyn * d->nc[0]);
        k_co_rxy<<<gzn, 256, rs, s>>>(gxn, gyn, N, d->nc[0], d->nc[1], d->xi, d->rg, d->t2, sc);
        NB_CUDA(cudaGetLastError());
        const int total = d->nc[0] * d->nc[1] * d->nc[2];
        k_co_rz<<<(total + 255) / 256, 256, 0, s>>>(N, d->nc[0] * d->nc[1], d->nc[2], d->xi, d->t2,
                                                    d->rc, sc);
        NB_CUDA(cudaGetLastError());
        k_co_solve<<<1, 1024, 2 * sizeof(float) * total, s>>>(d->nc[0], d->nc[1], d->nc[2], d->Sc,
                                                              d->lamc, d->rc, d->zc, sc);
        NB_CUDA(cudaGetLastError());
        zc = d->zc;
    }
    if (sc)
        return sw_sum<true>(1, d->m, 0, d->grid_sum, m->E, m->nx, m->ny, m->nz, d->zt, m->dinv32,
                            z, r, wold, sc, part, s, zc, d->xi);
    return sw_sum<false>(1, d->m, 0, d->grid_sum, m->E, m->nx, m->ny, m->nz, d->zt, m->dinv32, z,
                         r, wold, sc, part, s, zc, d->xi);
}

// Set-up of the coarse level for the two-level form (once per mesh).
nb_status schwarz_coarse_setup(nb_mesh *m)
{
    NB_TRY(schwarz_setup(m));
    return schwarz_setup_coarse(m);
}

// The coarse-grid correction in FP64 inside the refinement's outer step:
// given the FP64 residual r64 = b - A x (continuous, masked), the coarse
// correction c = R_0^T A_0^-1 R_0 r64 is computed in FP64 and added to x; r64
// becomes r64 - A c with A c the FP32 operator (the inner solve's accuracy)
// applied to c rounded to FP32 in c32_tmp, w32_tmp.  *norm_dev receives
// (r, c, r) of the new r64.  The coarse level is the two-level
// preconditioner's; the smooth error the FP32 inner solves leave in x has an
// FP64 residual below what the stopping test resolves, and this correction
// removes it.  No-op (returns false in *applied) without a coarse level.
nb_status schwarz_coarse_correct64(nb_mesh *m, double *r64, double *x, float *c32_tmp,
                                   float *w32_tmp, double *part, double *norm_dev,
                                   bool *applied, cudaStream_t s)
{
    *applied = false;
    NB_TRY(schwarz_coarse_setup(m));
    SchwarzData *d = (SchwarzData *)m->schwarz;
    if (!d->coarse) return NB_OK;
    const int N = m->N, gxn = m->nx * N + 1, gyn = m->ny * N + 1, gzn = m->nz * N + 1;
    const int ncx = d->nc[0], ncy = d->nc[1], ncz = d->nc[2], total = ncx * ncy * ncz;
    auto blocks = [](int64_t cnt) { return (int)std::min<int64_t>((cnt + 255) / 256, 65535); };
    NB_TRY(to_global(m, NB_FP64, r64, d->rg64, s));
    k_c64_rx<<<blocks((int64_t)gzn * gyn * ncx), 256, 0, s>>>((int64_t)gzn * gyn, gxn, N, ncx,
                                                             d->xi64, d->rg64, d->t1);
    k_c64_rmid<<<blocks((int64_t)gzn * ncy * ncx), 256, 0, s>>>(gzn, gyn, ncy, ncx, N, d->xi64,
                                                               d->t1, d->t2d);
    k_c64_rmid<<<blocks(total), 256, 0, s>>>(1, gzn, ncz, ncx * ncy, N, d->xi64, d->t2d, d->ca);
    // A_0^-1 = (Sz Sy Sx) diag(1 / (lx + ly + lz)) (Sz Sy Sx)^T
    const int bt = blocks(total);
    k_c64_axis<<<bt, 256, 0, s>>>(ncx, ncy, ncz, 0, 1, d->Sc64, nullptr, d->ca, d->cb);
    k_c64_axis<<<bt, 256, 0, s>>>(ncx, ncy, ncz, 1, 1, d->Sc64, nullptr, d->cb, d->ca);
    k_c64_axis<<<bt, 256, 0, s>>>(ncx, ncy, ncz, 2, 1, d->Sc64, d->lamc64, d->ca, d->cb);
    k_c64_axis<<<bt, 256, 0, s>>>(ncx, ncy, ncz, 2, 0, d->Sc64, nullptr, d->cb, d->ca);
    k_c64_axis<<<bt, 256, 0, s>>>(ncx, ncy, ncz, 1, 0, d->Sc64, nullptr, d->ca, d->cb);
    k_c64_axis<<<bt, 256, 0, s>>>(ncx, ncy, ncz, 0, 0, d->Sc64, nullptr, d->cb, d->ca);
    const int g = vec_grid(m->ctx, m->nL);
    k_c64_prolong<<<g, kVecThreads, 0, s>>>(m->nL, m->nx, m->ny, N, d->xi64, d->ca, ncx, ncy, ncz,
                                            x, c32_tmp);
    NB_CUDA(cudaGetLastError());
    NB_TRY(ax_local(m, NB_FP32, c32_tmp, w32_tmp, nullptr, nullptr, s));
    NB_TRY(dssum(m, NB_FP32, w32_tmp, 1, s));
    k_c64_subnorm<<<g, kVecThreads, 0, s>>>(m->nL, r64, w32_tmp, m->c32, part);
    NB_CUDA(cudaGetLastError());
    NB_TRY(sum_partials_dev(part, g, norm_dev, s));
    m->launches += 14;
    *applied = true;
    return NB_OK;
}

// z = M r for FP32 L-vectors r (continuous, masked); coarse: two-level form.
nb_status schwarz_apply(nb_mesh *m, const float *r, float *z, cudaStream_t s, bool coarse)
{
    NB_TRY(schwarz_gather(m, r, s));
    return schwarz_solve_sum(m, r, z, nullptr, nullptr, nullptr, s, coarse);
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
    NB_DEVICE_SCOPE(m->ctx->device);
    NB_TRY(schwarz_setup(m));
    NB_TRY(schwarz_apply(m, r_dev, z_dev, m->ctx->stream, false));
    NB_CUDA(cudaStreamSynchronize(m->ctx->stream));
    return NB_OK;
}

extern "C" nb_status nb_schwarz2_apply(nb_mesh *m, const float *r_dev, float *z_dev)
{
    if (!m || !r_dev || !z_dev) {
        set_error("invalid argument: NULL mesh or vector");
        return NB_ERR_ARG;
    }
    if (!m->gs_ready) {
        set_error("call nb_setup_gs first");
        return NB_ERR_STATE;
    }
    NB_DEVICE_SCOPE(m->ctx->device);
    NB_TRY(schwarz_coarse_setup(m));
    NB_TRY(schwarz_apply(m, r_dev, z_dev, m->ctx->stream, true));
    NB_CUDA(cudaStreamSynchronize(m->ctx->stream));
    return NB_OK;
}
