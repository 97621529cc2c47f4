// Emulated reduced precision on the GPU: the CG loop in binary64 with every
// +, -, *, / rounded to t mantissa bits, the study of Section 4.2 (the VPREC
// backend of Section 2 emulates lower precisions by computing each operation
// in the original type and rounding its result).  Rounding: round to nearest,
// ties to even, on the binary64 representation, the binary64 exponent range
// kept.  The operator and the direct-stiffness summation do their operations
// in the oracle's order (per node: the l-loops in turn; per global node: the
// copies in ascending local index); dot products are summed per thread, per
// block in a fixed tree and over blocks in index order.  Not a hot path: one
// block per element, one thread per node, host-launched kernels.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "nb_reduce.cuh"

namespace nb {

__device__ __forceinline__ double vr(double x, int t)
{
    if (t >= 52) return x;
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    if (((b >> 52) & 0x7ffull) == 0x7ffull) return x;
    const int drop = 52 - t;
    const unsigned long long mask = (1ull << drop) - 1ull, half = 1ull << (drop - 1);
    const unsigned long long rem = b & mask;
    b &= ~mask;
    if (rem > half || (rem == half && ((b >> drop) & 1ull))) b += 1ull << drop;
    return __longlong_as_double((long long)b);
}

// Emulated arithmetic of one thread.  mode 0: every result rounded to t
// bits (VPREC).  Monte Carlo Arithmetic (Section 2, the MCA backend; Parker,
// 1997) at virtual precision t: inexact(x) = x + 2^(e_x - t) xi, xi uniform on
// (-1/2, 1/2), 2^(e_x - 1) <= |x| < 2^e_x; mode 1 (random rounding)
// perturbs each result, mode 2 (full MCA) the operands and the result.  Each
// operation is computed correctly rounded in binary64 and never fused with
// another (explicit _rn intrinsics).  Random numbers: SplitMix64 (Steele, Lea
// and Flood, 2014), one stream per thread and launch, keyed by the run's
// seed, the launch's call number and the thread's global index.
struct Emu {
    int mode, t;
    unsigned long long s;

    __device__ Emu(int mode_, int t_, unsigned long long seed, unsigned long long call)
        : mode(mode_), t(t_)
    {
        const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
        s = seed ^ (call * 0xD1B54A32D192ED03ull) ^ (tid * 0x9E3779B97F4A7C15ull);
        next();  // decorrelate neighbouring keys
    }
    __device__ unsigned long long next()
    {
        unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    __device__ double inexact(double x)
    {
        if (x == 0.0 || !isfinite(x)) return x;
        int e;
        frexp(x, &e);
        const double xi = (double)(next() >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        return __dadd_rn(x, ldexp(xi, e - t));
    }
    __device__ double out(double r) { return mode == 0 ? vr(r, t) : inexact(r); }
    __device__ double add(double a, double b)
    {
        if (mode == 2) { a = inexact(a); b = inexact(b); }
        return out(__dadd_rn(a, b));
    }
    __device__ double sub(double a, double b)
    {
        if (mode == 2) { a = inexact(a); b = inexact(b); }
        return out(__dsub_rn(a, b));
    }
    __device__ double mul(double a, double b)
    {
        if (mode == 2) { a = inexact(a); b = inexact(b); }
        return out(__dmul_rn(a, b));
    }
    __device__ double div(double a, double b)
    {
        if (mode == 2) { a = inexact(a); b = inexact(b); }
        return out(__ddiv_rn(a, b));
    }
};

// Parameters of one emulated launch (passed by value).
struct EmuArgs {
    int mode, t;
    unsigned long long seed, call;
};

// w = A_L u per element with every operation emulated (one block per element).
__global__ void k_vp_ax(EmuArgs ea, long long E, int n, const double *__restrict__ Dg,
                        const double *__restrict__ G, const double *__restrict__ u,
                        double *__restrict__ w)
{
    extern __shared__ double vsm[];
    Emu em(ea.mode, ea.t, ea.seed, ea.call);
    const int n2 = n * n, n3 = n2 * n;
    double *D = vsm, *su = D + n2, *wr = su + n3, *ws = wr + n3, *wt = ws + n3;
    for (int q = threadIdx.x; q < n2; q += blockDim.x) D[q] = Dg[q];
    for (long long e = blockIdx.x; e < E; e += gridDim.x) {
        __syncthreads();
        for (int q = threadIdx.x; q < n3; q += blockDim.x) su[q] = u[e * n3 + q];
        __syncthreads();
        const double *Ge = G + e * 6 * n3;
        for (int q = threadIdx.x; q < n3; q += blockDim.x) {
            const int i = q % n, j = (q / n) % n, k = q / n2;
            double ur = 0.0, us = 0.0, ut = 0.0;
            for (int l = 0; l < n; ++l) {
                ur = em.add(ur, em.mul(D[i * n + l], su[(k * n + j) * n + l]));
                us = em.add(us, em.mul(D[j * n + l], su[(k * n + l) * n + i]));
                ut = em.add(ut, em.mul(D[k * n + l], su[(l * n + j) * n + i]));
            }
            const double grr = Ge[q], grs = Ge[n3 + q], grt = Ge[2 * n3 + q];
            const double gss = Ge[3 * n3 + q], gst = Ge[4 * n3 + q], gtt = Ge[5 * n3 + q];
            wr[q] = em.add(em.add(em.mul(grr, ur), em.mul(grs, us)), em.mul(grt, ut));
            ws[q] = em.add(em.add(em.mul(grs, ur), em.mul(gss, us)), em.mul(gst, ut));
            wt[q] = em.add(em.add(em.mul(grt, ur), em.mul(gst, us)), em.mul(gtt, ut));
        }
        __syncthreads();
        for (int q = threadIdx.x; q < n3; q += blockDim.x) {
            const int i = q % n, j = (q / n) % n, k = q / n2;
            double s = 0.0;
            for (int l = 0; l < n; ++l) s = em.add(s, em.mul(D[l * n + i], wr[(k * n + j) * n + l]));
            for (int l = 0; l < n; ++l) s = em.add(s, em.mul(D[l * n + j], ws[(k * n + l) * n + i]));
            for (int l = 0; l < n; ++l) s = em.add(s, em.mul(D[l * n + k], wt[(l * n + j) * n + i]));
            w[e * n3 + q] = s;
        }
    }
}

// Masked direct-stiffness summation with emulated additions, copies in
// ascending local order (single-copy free nodes are unchanged).
__global__ void k_vp_gs(EmuArgs ea, long long rows, const int32_t *__restrict__ off,
                        const int32_t *__restrict__ loc, const uint8_t *__restrict__ mask,
                        double *__restrict__ u)
{
    Emu em(ea.mode, ea.t, ea.seed, ea.call);
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < rows;
         a += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int o = off[a]; o < off[a + 1]; ++o) s = em.add(s, u[loc[o]]);
        if (mask[a] == 0) s = 0.0;
        for (int o = off[a]; o < off[a + 1]; ++o) u[loc[o]] = s;
    }
}

// Block partials of sum a b c with emulated operations (per thread in index
// order, then a fixed tree in shared memory).
__global__ void k_vp_dot(EmuArgs ea, long long n, const double *__restrict__ a,
                         const double *__restrict__ b, const float *__restrict__ c,
                         double *__restrict__ part)
{
    __shared__ double sh[256];
    Emu em(ea.mode, ea.t, ea.seed, ea.call);
    double s = 0.0;
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < n;
         l += (long long)gridDim.x * blockDim.x)
        s = em.add(s, em.mul(em.mul(a[l], b[l]), (double)c[l]));
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] = em.add(sh[threadIdx.x], sh[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// The loop's scalars, one thread.  slot 0: rtz1, 1: rtz2, 2: pap, 3: rtr,
// 4: beta, 5: alpha, 6: |b|, 7: relative residual.  what: 0 rtz (beta),
// 1 pap (alpha), 2 rtr (residual, into hist[it]).
__global__ void k_vp_scalar(EmuArgs ea, int what, int it, int cnt, const double *__restrict__ part,
                            double *sc, double *hist)
{
    Emu em(ea.mode, ea.t, ea.seed, ea.call);
    double s = 0.0;
    for (int q = 0; q < cnt; ++q) s = em.add(s, part[q]);
    if (what == 0) {
        sc[1] = sc[0];
        sc[0] = s;
        sc[4] = it == 0 ? 0.0 : em.div(s, sc[1]);
    } else if (what == 1) {
        sc[2] = s;
        sc[5] = em.div(sc[0], s);
    } else {
        sc[3] = s;
        sc[7] = em.div(sqrt(s), sc[6]);
        hist[it] = sc[7];
    }
}

// z = dinv r (Jacobi; the library's dinv carries an ownership mark in its
// sign bit, |dinv| is the Jacobi factor).
__global__ void k_vp_z(EmuArgs ea, long long n, const double *__restrict__ dinv,
                       const double *__restrict__ r, double *__restrict__ z)
{
    Emu em(ea.mode, ea.t, ea.seed, ea.call);
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < n;
         l += (long long)gridDim.x * blockDim.x)
        z[l] = em.mul(fabs(dinv[l]), r[l]);
}

// p = beta p + z.
__global__ void k_vp_p(EmuArgs ea, long long n, const double *__restrict__ z,
                       double *__restrict__ p, const double *__restrict__ sc)
{
    Emu em(ea.mode, ea.t, ea.seed, ea.call);
    const double beta = sc[4];
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < n;
         l += (long long)gridDim.x * blockDim.x)
        p[l] = em.add(em.mul(beta, p[l]), z[l]);
}

// x += alpha p, r -= alpha w.
__global__ void k_vp_xr(EmuArgs ea, long long n, const double *__restrict__ sc,
                        const double *__restrict__ p, const double *__restrict__ w,
                        double *__restrict__ x, double *__restrict__ r)
{
    Emu em(ea.mode, ea.t, ea.seed, ea.call);
    const double alpha = sc[5];
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < n;
         l += (long long)gridDim.x * blockDim.x) {
        x[l] = em.add(x[l], em.mul(alpha, p[l]));
        r[l] = em.sub(r[l], em.mul(alpha, w[l]));
    }
}

// |b| in binary64 (set-up, not emulated), into sc[6].
__global__ void k_vp_bnorm(int cnt, const double *__restrict__ part, double *sc)
{
    double s = 0.0;
    for (int q = 0; q < cnt; ++q) s += part[q];
    sc[6] = s > 0.0 ? sqrt(s) : 1.0;
}

static int vp_threads(int n3) { return std::min(1024, (n3 + 31) / 32 * 32); }

static nb_status vp_apply(nb_mesh *m, EmuArgs &ea, const double *u, double *w, cudaStream_t s)
{
    const size_t smem = sizeof(double) * ((size_t)m->n * m->n + 4 * (size_t)m->n3);
    NB_CUDA(cudaFuncSetAttribute(k_vp_ax, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (int)std::min<int64_t>(m->E, (int64_t)m->ctx->sm_count * 8);
    k_vp_ax<<<grid, vp_threads(m->n3), smem, s>>>(ea, m->E, m->n, m->D64, m->G64, u, w);
    ++ea.call;
    NB_CUDA(cudaGetLastError());
    if (m->gs_rows > 0) {
        const int g = (int)std::min<int64_t>((m->gs_rows + 255) / 256, (int64_t)m->ctx->sm_count * 8);
        k_vp_gs<<<g, 256, 0, s>>>(ea, m->gs_rows, m->gs_off, m->gs_loc, m->gs_mask, w);
        ++ea.call;
        NB_CUDA(cudaGetLastError());
    }
    return NB_OK;
}

// `iters` emulated CG iterations from x = 0 (see nb_cg_vprec / nb_cg_mca).
static nb_status cg_emulated(nb_mesh *m, int mode, int t, uint64_t seed, int iters, nb_pc pc,
                             const double *b_dev, double *x_dev, double *hist_host,
                             double *relres)
{
    if (!m || !b_dev || !x_dev || t < 1 || t > 52 || iters < 0 ||
        (pc != NB_PC_NONE && pc != NB_PC_JACOBI)) {
        set_error("invalid argument: mesh, vectors, t (1..52), iters or preconditioner");
        return NB_ERR_ARG;
    }
    if (!m->gs_ready) {
        set_error("call nb_setup_gs first");
        return NB_ERR_STATE;
    }
    NB_DEVICE_SCOPE(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    const int64_t n = m->nL;
    const int vb = 256;
    const int vg = (int)std::min<int64_t>((n + vb - 1) / vb, (int64_t)m->ctx->sm_count * 4);
    double *buf = nullptr;
    // r, z, p, w (n each), block partials (vg), scalars (8), history (iters)
    const size_t words = 4 * (size_t)n + vg + 8 + std::max(iters, 1);
    NB_CUDA(cudaMalloc(&buf, sizeof(double) * words));
    double *r = buf, *z = r + n, *p = z + n, *w = p + n, *part = w + n, *sc = part + vg;
    double *hist = sc + 8;
    nb_status st = NB_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && st == NB_OK) {
            set_error("emulated CG: %s", cudaGetErrorString(e));
            st = NB_ERR_CUDA;
        }
    };
    EmuArgs ea = {mode, t, (unsigned long long)seed, 1ull};
    const EmuArgs exact = {0, 52, 0ull, 0ull};  // set-up in binary64
    // x = 0, r = b, p = 0 (the loop starts from zero, as Nekbone's)
    ck(cudaMemsetAsync(x_dev, 0, sizeof(double) * n, s));
    ck(cudaMemcpyAsync(r, b_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    ck(cudaMemsetAsync(p, 0, sizeof(double) * n, s));
    ck(cudaMemsetAsync(sc, 0, sizeof(double) * 8, s));
    k_vp_dot<<<vg, vb, 0, s>>>(exact, n, b_dev, b_dev, m->c32, part);
    k_vp_bnorm<<<1, 1, 0, s>>>(vg, part, sc);
    ck(cudaGetLastError());
    const int jac = pc == NB_PC_JACOBI;
    for (int it = 0; it < iters && st == NB_OK; ++it) {
        // z (Jacobi, or z = r), rtz = (r, c, z), beta, p = beta p + z
        const double *zz = r;
        if (jac) {
            k_vp_z<<<vg, vb, 0, s>>>(ea, n, m->dinv64, r, z);
            ++ea.call;
            zz = z;
        }
        k_vp_dot<<<vg, vb, 0, s>>>(ea, n, r, zz, m->c32, part);
        ++ea.call;
        k_vp_scalar<<<1, 1, 0, s>>>(ea, 0, it, vg, part, sc, hist);
        ++ea.call;
        k_vp_p<<<vg, vb, 0, s>>>(ea, n, zz, p, sc);
        ++ea.call;
        ck(cudaGetLastError());
        if (st != NB_OK) break;
        st = vp_apply(m, ea, p, w, s);
        if (st != NB_OK) break;
        k_vp_dot<<<vg, vb, 0, s>>>(ea, n, w, p, m->c32, part);
        ++ea.call;
        k_vp_scalar<<<1, 1, 0, s>>>(ea, 1, it, vg, part, sc, hist);
        ++ea.call;
        k_vp_xr<<<vg, vb, 0, s>>>(ea, n, sc, p, w, x_dev, r);
        ++ea.call;
        k_vp_dot<<<vg, vb, 0, s>>>(ea, n, r, r, m->c32, part);
        ++ea.call;
        k_vp_scalar<<<1, 1, 0, s>>>(ea, 2, it, vg, part, sc, hist);
        ++ea.call;
        ck(cudaGetLastError());
    }
    std::vector<double> h(std::max(iters, 1));
    if (st == NB_OK) {
        ck(cudaMemcpyAsync(h.data(), hist, sizeof(double) * std::max(iters, 1),
                           cudaMemcpyDeviceToHost, s));
        ck(cudaStreamSynchronize(s));
    }
    cudaStreamSynchronize(s);
    cudaFree(buf);
    if (st != NB_OK) return st;
    if (hist_host) memcpy(hist_host, h.data(), sizeof(double) * iters);
    if (relres) *relres = iters > 0 ? h[iters - 1] : 1.0;
    return NB_OK;
}

}  // namespace nb

using namespace nb;

extern "C" nb_status nb_apply_vprec(nb_mesh *m, int t, const double *u_dev, double *w_dev)
{
    if (!m || !u_dev || !w_dev || t < 1 || t > 52) {
        set_error("invalid argument: mesh, vectors or t (1..52)");
        return NB_ERR_ARG;
    }
    if (!m->gs_ready) {
        set_error("call nb_setup_gs first");
        return NB_ERR_STATE;
    }
    NB_DEVICE_SCOPE(m->ctx->device);
    EmuArgs ea = {0, t, 0ull, 0ull};
    NB_TRY(vp_apply(m, ea, u_dev, w_dev, m->ctx->stream));
    NB_CUDA(cudaStreamSynchronize(m->ctx->stream));
    return NB_OK;
}

extern "C" nb_status nb_cg_vprec(nb_mesh *m, int t, int iters, nb_pc pc, const double *b_dev,
                                 double *x_dev, double *hist_host, double *relres)
{
    return cg_emulated(m, 0, t, 0, iters, pc, b_dev, x_dev, hist_host, relres);
}

extern "C" nb_status nb_cg_mca(nb_mesh *m, int mode, int t, uint64_t seed, int iters, nb_pc pc,
                               const double *b_dev, double *x_dev, double *hist_host,
                               double *relres)
{
    if (mode != 1 && mode != 2) {
        set_error("invalid argument: MCA mode must be 1 (random rounding) or 2 (full MCA)");
        return NB_ERR_ARG;
    }
    return cg_emulated(m, mode, t, seed, iters, pc, b_dev, x_dev, hist_host, relres);
}
