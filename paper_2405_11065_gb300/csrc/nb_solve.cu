// Conjugate-gradient solvers on the device.
//
// The iteration follows Table 1 of the case study: z = solveM(r);
// rtz1 = glsc3(r,c,z); p = beta p + z (add2s1); w = ax(p) with dssum;
// pap = glsc3(w,c,p); x += alpha p, r -= alpha w (add2s2); rtr = glsc3(r,c,r).
// On the GPU the nine lines become two kernels per iteration:
//   1. ax_cg_step: p = dinv*r + beta*p, w_L = A_L p, partials of p.w_L (= pap);
//      its last block sums them: alpha = rtz/pap (breakdown check)
//   2. update with dssum + mask of w folded in: x += alpha p, r -= alpha w,
//      partials of (r,c,dinv r), (r,c,r); its last block sums them: beta,
//      convergence, iteration limit (in FP64, and outside the built orders,
//      a separate dssum kernel and update)
// All scalars live in device memory, so the iteration is captured once in a
// CUDA graph whose while-node repeats it (a one-thread kernel sets the loop
// condition) until converged, at the iteration limit, or on breakdown:
// one graph launch per solve.
//
// Mixed precision (Section 6 runs the CG loop in single precision, set-up in
// double): the reduced-precision solve sits inside FP64 iterative refinement.
// r = b - A x and x += s*d are FP64; the inner PCG runs its operator and
// vectors in FP32 (or with tensor-core contractions), its dot products
// accumulated in FP64.
#include <math.h>

#include <algorithm>

#include "nb_bulk.cuh"
#include "nb_cg_dev.cuh"

namespace nb {

// keep: resume with the previous direction (reliable update); odd: the
// previous inner solve ended after an odd number of steps (nb_learned.cu)
nb_status fcg_learned(nb_mesh *m, nb_prec prec, Workspace &ws, const nb_opts *o, bool keep,
                      bool odd, cudaStream_t s);
nb_status fcg_schwarz(nb_mesh *m, nb_prec prec, Workspace &ws, const nb_opts *o, bool keep,
                      bool odd, cudaStream_t s);
nb_status schwarz_coarse_correct64(nb_mesh *m, double *r64, double *x, float *c32_tmp,
                                   float *w32_tmp, double *part, double *norm_dev,
                                   bool *applied, cudaStream_t s);

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

__global__ void k_cg_setup(CgScalars *sc, double tol, int maxit, double *hist, int hist_cap,
                           int pdl_early)
{
    sc->pdl_early = pdl_early;
    sc->tol = tol;
    sc->maxit = maxit;
    sc->hist = hist;
    sc->hist_cap = hist_cap;
    sc->iter = 0;
    sc->done = 0;
    sc->status = 0;
    sc->beta = 0.0;
    sc->alpha = 0.0;
    sc->loops = 0;
    sc->tick_ax = 0u;
    sc->tick_upd = 0u;
    sc->x_pending = 0;
}

// The weighted dot products glsc3(a, c, b) of the iteration, for continuous
// vectors, equal plain sums over one "owner" copy of every global node.  The
// solver's preconditioner array carries that ownership in its sign bit
// (dinv >= +0 on the owner copy, <= -0 on the others; |dinv| is the Jacobi
// factor), so the iteration reads no weight vector.
template <typename T>
__device__ __forceinline__ bool owner_copy(T d)
{
    return !signbit(d);
}

// p = 0 (unless zero_p == 0: a resumed iteration keeps its direction);
// partials of (r, dinv r) and (r, r) over owner copies.
template <typename T>
__global__ void k_cg_init(int64_t nL, const T *__restrict__ r, const T *__restrict__ dinv,
                          T *__restrict__ p, double *__restrict__ part, int zero_p)
{
    __shared__ double sred[32];
    DotAcc<T> a, b;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x) {
        const T rl = r[l], d = dinv[l];
        if (zero_p) p[l] = T(0);
        if (owner_copy(d)) {
            a.add(rl * (d * rl));
            b.add(rl * rl);
        }
    }
    double ta = block_sum_acc(a, sred);
    double tb = block_sum_acc(b, sred);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ta;
        part[gridDim.x + blockIdx.x] = tb;
    }
}

// bnorm_from_r: the system's right-hand side is the initial residual.
__global__ void k_cg_init_fin(CgScalars *sc, const double *__restrict__ part, int cnt,
                              int bnorm_from_r)
{
    __shared__ double sred[32];
    double rtz = sum_partials(part, cnt, sred);
    double rtr = sum_partials(part + cnt, cnt, sred);
    if (threadIdx.x == 0) {
        sc->rtz = rtz;
        sc->rtz_old = rtz;
        sc->rtr = rtr;
        if (bnorm_from_r) sc->bnorm2 = rtr;
        const double bn = sc->bnorm2 > 0.0 ? sc->bnorm2 : 1.0;
        sc->relres = sqrt(rtr / bn);
        sc->beta = 0.0;
        sc->pap_prev = 0.0;
        if (!(sc->relres >= 0.0) || !isfinite(sc->relres)) {
            sc->done = 1;
            sc->status = NB_BREAKDOWN;
        } else if (sc->relres < sc->tol || rtr == 0.0) {
            sc->done = 1;
        } else if (sc->maxit <= 0) {
            sc->done = 1;
            sc->status = NB_NOT_CONVERGED;
        }
    }
}

// Resumption of the CG iteration after a residual replacement (reliable
// update): r now holds the true residual b - A x (FP64) scaled by 1/s_new,
// while p is still in the units of the previous scale s_old.  With
// c = s_old / s_new the next direction is p = z + beta (c p_old) and
// beta = rtz_new / (rtz_k c^2), rtz_k the last (r, z) before the replaced
// residual (sc->rtz_old after the last update); the ax step applies
// beta_eff = rtz_new / (rtz_k c) to the stored p.  bnorm2 becomes the new
// residual's norm (the segment's tolerance is relative to it).
__global__ void k_cg_resume_fin(CgScalars *sc, const double *__restrict__ part, int cnt, double c)
{
    __shared__ double sred[32];
    const double rtz = sum_partials(part, cnt, sred);
    const double rtr = sum_partials(part + cnt, cnt, sred);
    if (threadIdx.x == 0) {
        const double beta = rtz / (sc->rtz_old * c);
        sc->rtz = rtz;
        sc->rtz_old = rtz;
        sc->rtr = rtr;
        sc->bnorm2 = rtr;
        sc->relres = 1.0;
        sc->beta = beta;
        sc->pap_prev = 0.0;
        if (!isfinite(beta) || !(rtr > 0.0) || !isfinite(rtr)) {
            sc->done = 1;
            sc->status = NB_BREAKDOWN;
        } else if (sc->maxit <= 0) {
            sc->done = 1;
            sc->status = NB_NOT_CONVERGED;
        }
    }
}

// add2s2 twice, then solveM and the two dot products of the next iteration.
template <typename T>
__global__ void k_cg_update(int64_t nL, CgScalars *__restrict__ sc, T *__restrict__ x,
                            T *__restrict__ r, const T *__restrict__ p, const T *__restrict__ w,
                            const T *__restrict__ dinv, double *__restrict__ part)
{
    __shared__ double sred[32];
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    DotAcc<T> a, b;
    auto node = [&](T &xl, T &rv, T pl, T wl, T d) {
        xl = xl + alpha * pl;
        rv = rv - alpha * wl;
        if (owner_copy(d)) {
            a.add(rv * (d * rv));
            b.add(rv * rv);
        }
    };
    int64_t head = 0;
    if constexpr (sizeof(T) == 4) {  // four nodes per 16-byte access (16-byte aligned buffers)
        const int64_t n4 = nL / 4;
        for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4;
             q += (int64_t)gridDim.x * blockDim.x) {
            float4 xv = reinterpret_cast<float4 *>(x)[q];
            float4 rv = reinterpret_cast<float4 *>(r)[q];
            const float4 pv = reinterpret_cast<const float4 *>(p)[q];
            const float4 wv = reinterpret_cast<const float4 *>(w)[q];
            const float4 dv = reinterpret_cast<const float4 *>(dinv)[q];
            node((T &)xv.x, (T &)rv.x, pv.x, wv.x, dv.x);
            node((T &)xv.y, (T &)rv.y, pv.y, wv.y, dv.y);
            node((T &)xv.z, (T &)rv.z, pv.z, wv.z, dv.z);
            node((T &)xv.w, (T &)rv.w, pv.w, wv.w, dv.w);
            reinterpret_cast<float4 *>(x)[q] = xv;
            reinterpret_cast<float4 *>(r)[q] = rv;
        }
        head = n4 * 4;
    }
    for (int64_t l = head + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x) {
        T xl = x[l], rl = r[l];
        node(xl, rl, p[l], w[l], dinv[l]);
        x[l] = xl;
        r[l] = rl;
    }
    double ta = block_sum_acc(a, sred);
    double tb = block_sum_acc(b, sred);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ta;
        part[gridDim.x + blockIdx.x] = tb;
    }
    // the last block to finish: rtz, rtr, beta, convergence (nb_cg_dev.cuh)
    if (last_block(&sc->tick_upd)) cg_finish_iter(sc, part, gridDim.x, sred);
}

// The update with the direct-stiffness summation of w folded in: for each
// local node, w_asm = mask * (sum of w over the node's copies in ascending
// local index), then x += alpha p, r -= alpha w_asm and the partials of
// (r, c, dinv r), (r, c, r) as in k_cg_update.  On the box mesh the copies of
// a node are its mirror nodes in the neighbouring elements: along x the node
// with i = 0 is node i = N of element ex - 1 (offset -(n^3 - N)), i = N is
// node 0 of ex + 1, and likewise along y and z; a node has 1, 2, 4 or 8 of
// them, summed in ascending element order -- the order of the separate
// summation kernel, so the result is bit-identical to dssum + k_cg_update.
// The mask is read from dinv (0 exactly on Dirichlet nodes, also in the
// identity preconditioner's array).  One block per element (grid-stride),
// its threads over the element's nodes.
template <typename T, int n>
__global__ void __launch_bounds__(256)
k_cg_update_gs(int64_t E, int nx, int ny, int nz, CgScalars *__restrict__ sc, T *__restrict__ x,
               T *__restrict__ r, const T *__restrict__ p, const T *__restrict__ w,
               const T *__restrict__ dinv, double *__restrict__ part)
{
    constexpr int N = n - 1, n2 = n * n, n3 = n2 * n;
    __shared__ double sred[32];
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    const int64_t sx = n3 - N, sy = (int64_t)nx * n3 - N * n, sz = (int64_t)nx * ny * n3 - N * n2;
    DotAcc<T> a, b;
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
        for (int q = threadIdx.x; q < n3; q += blockDim.x) {
            const int i = q % n, j = (q / n) % n, k = q / n2;
            const int64_t l = e * n3 + q;
            const int lx = i == 0 && ex > 0, hx = i == N && ex < nx - 1;
            const int ly = j == 0 && ey > 0, hy = j == N && ey < ny - 1;
            const int lz = k == 0 && ez > 0, hz = k == N && ez < nz - 1;
            const T *w0 = w + (l - lx * sx - ly * sy - lz * sz);
            T v[2][2][2];
#pragma unroll
            for (int tz = 0; tz < 2; ++tz)
#pragma unroll
                for (int ty = 0; ty < 2; ++ty)
#pragma unroll
                    for (int tx = 0; tx < 2; ++tx) {
                        const bool ok = tz <= lz + hz && ty <= ly + hy && tx <= lx + hx;
                        v[tz][ty][tx] = ok ? w0[tx * sx + ty * sy + tz * sz] : T(0);
                    }
            const T d = dinv[l];
            T xl = x[l], rl = r[l];
            const T pl = p[l];
            T wl = T(0);
#pragma unroll
            for (int tz = 0; tz < 2; ++tz)
#pragma unroll
                for (int ty = 0; ty < 2; ++ty)
#pragma unroll
                    for (int tx = 0; tx < 2; ++tx) wl += v[tz][ty][tx];
            if (d == T(0)) wl = T(0);  // Dirichlet node
            xl = xl + alpha * pl;
            rl = rl - alpha * wl;
            if (owner_copy(d)) {
                a.add(rl * (d * rl));
                b.add(rl * rl);
            }
            x[l] = xl;
            r[l] = rl;
        }
    }
    double ta = block_sum_acc(a, sred);
    double tb = block_sum_acc(b, sred);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ta;
        part[gridDim.x + blockIdx.x] = tb;
    }
    if (last_block(&sc->tick_upd)) cg_finish_iter(sc, part, gridDim.x, sred);
}

// k_cg_update_gs for even n, two nodes (i0, i0 + 1) of a row per thread with
// 8- / 16-byte accesses.  N is odd, so only the first node of a pair can be
// on the lower x face (i0 = 0) and only the second on the upper one
// (i0 + 1 = N); the y / z copies of both nodes are one vector load each.
// Same sums in the same order as k_cg_update_gs.
template <typename T, int n>
__global__ void __launch_bounds__(256)
k_cg_update_gs2(int64_t E, int nx, int ny, int nz, CgScalars *__restrict__ sc, T *__restrict__ x,
                T *__restrict__ r, const T *__restrict__ p, const T *__restrict__ w,
                const T *__restrict__ dinv, double *__restrict__ part)
{
    static_assert(n % 2 == 0, "pairs of nodes need an even n");
    using V = typename Pair2<T>::type;
    constexpr int N = n - 1, n2 = n * n, n3 = n2 * n, h = n / 2, P = n3 / 2;
    __shared__ double sred[32];
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    const int64_t sx = n3 - N, sy = (int64_t)nx * n3 - N * n, sz = (int64_t)nx * ny * n3 - N * n2;
    DotAcc<T> a, b;
    auto node = [&](T &xl, T &rl, T pl, T wl, T d) {
        if (d == T(0)) wl = T(0);  // Dirichlet node
        xl = xl + alpha * pl;
        rl = rl - alpha * wl;
        if (owner_copy(d)) {
            a.add(rl * (d * rl));
            b.add(rl * rl);
        }
    };
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
        for (int t = threadIdx.x; t < P; t += blockDim.x) {
            const int i0 = 2 * (t % h), j = (t / h) % n, k = t / (h * n);
            const int64_t l = e * n3 + (int64_t)k * n2 + j * n + i0;
            T wa, wb;
            gs_sum_pair<T, n>(w, l, i0, j, k, ex, ey, ez, nx, ny, nz, sx, sy, sz, wa, wb);
            V xv = *reinterpret_cast<V *>(x + l), rv = *reinterpret_cast<V *>(r + l);
            const V pv = *reinterpret_cast<const V *>(p + l);
            const V dv = *reinterpret_cast<const V *>(dinv + l);
            node(xv.x, rv.x, pv.x, wa, dv.x);
            node(xv.y, rv.y, pv.y, wb, dv.y);
            *reinterpret_cast<V *>(x + l) = xv;
            *reinterpret_cast<V *>(r + l) = rv;
        }
    }
    double ta = block_sum_acc(a, sred);
    double tb = block_sum_acc(b, sred);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ta;
        part[gridDim.x + blockIdx.x] = tb;
    }
    if (last_block(&sc->tick_upd)) cg_finish_iter(sc, part, gridDim.x, sred);
}

// k_cg_update_gs2 over node pairs instead of elements: the E n^3 / 2 pairs
// are dealt to the threads of a persistent grid in turn (pair q to thread
// q mod T), so every thread gets the same number of pairs to within one and
// no wave of blocks runs part-empty at the end.  Each thread works on two
// pairs at a time with all their loads issued first; the element of a pair
// and its box coordinates come from multiplications by constants fixed at
// launch (FastDiv).  32-bit indices (E n^3 < 2^31).  Same sums in the same
// order as k_cg_update_gs2, so the result is bit-identical to it.
template <typename T, int n>
__global__ void __launch_bounds__(256)
k_cg_update_pairs(int npairs, int nx, int ny, int nz, FastDiv dnx, FastDiv dny,
                  CgScalars *__restrict__ sc, T *__restrict__ x, T *__restrict__ r,
                  const T *__restrict__ p, const T *__restrict__ w, const T *__restrict__ dinv,
                  double *__restrict__ part)
{
    static_assert(n % 2 == 0, "pairs of nodes need an even n");
    using V = typename Pair2<T>::type;
    constexpr int N = n - 1, n2 = n * n, n3 = n2 * n, h = n / 2, P = n3 / 2;
    __shared__ double sred[32];
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    const int sx = n3 - N, sy = nx * n3 - N * n, sz = nx * ny * n3 - N * n2;
    DotAcc<T> a, b;
    struct Pair {
        int l;
        T wa, wb;
        V xv, rv, pv, dv;
    };
    auto load = [&](int q, Pair &c) {
        const int e = q / P, t = q - e * P;
        const int i0 = 2 * (t % h), j = (t / h) % n, k = t / (h * n);
        const int exy = dnx.div(e), ex = e - exy * nx;
        const int ez = dny.div(exy), ey = exy - ez * ny;
        c.l = e * n3 + k * n2 + j * n + i0;
        gs_sum_pair<T, n, int>(w, c.l, i0, j, k, ex, ey, ez, nx, ny, nz, sx, sy, sz, c.wa, c.wb);
        c.xv = *reinterpret_cast<const V *>(x + c.l);
        c.rv = *reinterpret_cast<const V *>(r + c.l);
        c.pv = *reinterpret_cast<const V *>(p + c.l);
        c.dv = *reinterpret_cast<const V *>(dinv + c.l);
    };
    auto node = [&](T &xl, T &rl, T pl, T wl, T d) {
        if (d == T(0)) wl = T(0);  // Dirichlet node
        xl = xl + alpha * pl;
        rl = rl - alpha * wl;
        if (owner_copy(d)) {
            a.add(rl * (d * rl));
            b.add(rl * rl);
        }
    };
    auto finish = [&](Pair &c) {
        node(c.xv.x, c.rv.x, c.pv.x, c.wa, c.dv.x);
        node(c.xv.y, c.rv.y, c.pv.y, c.wb, c.dv.y);
        *reinterpret_cast<V *>(x + c.l) = c.xv;
        *reinterpret_cast<V *>(r + c.l) = c.rv;
    };
    const int stride = gridDim.x * blockDim.x;
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    for (; q + stride < npairs; q += 2 * stride) {
        Pair c0, c1;
        load(q, c0);
        load(q + stride, c1);
        finish(c0);
        finish(c1);
    }
    if (q < npairs) {
        Pair c0;
        load(q, c0);
        finish(c0);
    }
    double ta = block_sum_acc(a, sred);
    double tb = block_sum_acc(b, sred);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ta;
        part[gridDim.x + blockIdx.x] = tb;
    }
    if (last_block(&sc->tick_upd)) cg_finish_iter(sc, part, gridDim.x, sred);
}

// Flexible CG: rtr from the update's partials, pap_prev, the iteration count,
// the relative residual (history) and the stopping tests (the same step as
// the flexible-CG update kernels of the learned and Schwarz paths).  Called by
// the whole last block.
__device__ __forceinline__ void fcg_finish_iter(CgScalars *sc, const double *part, int cnt,
                                                double *sred)
{
    const double rtr = sum_partials(part, cnt, sred);
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

// The update with the folded summation over contiguous element ranges (FLEX
// 0: Jacobi CG, its (r, dinv r) and (r, r) with beta in the last block; 1:
// flexible CG, (r, r) and the flexible-CG stopping step):
// block b of a persistent grid takes elements [E b / G, E (b + 1) / G), and
// thread t the node pairs t, t + 256, ... of each of them (R rounds).  The
// pair's position in the element -- its local offset and which faces it lies
// on -- is fixed per thread and computed once; per element only the box
// coordinates and the neighbour tests change.  The rounds of one element are
// loaded together before any is used.  With PIPE the next element's loads
// are issued before the current element is finished (more registers, fewer
// resident blocks: it pays where the blocks have few elements).  Same sums in
// the same order as k_cg_update_gs2 (bit-identical).  32-bit indices
// (E n^3 < 2^31).
// XM, the x step of Jacobi CG: 0 x += alpha p every iteration; 1 none (the
// even iteration of a pair: x, p are not read; the last block keeps alpha
// as alpha_x and marks the step pending); 2 x += alpha_x p2 + alpha p (the
// odd iteration: p2 the even iteration's direction, the two additions in
// the order of two single steps, so x is bit-identical to XM = 0).  A pair
// moves 16 + 32 bytes per local node in the update instead of 2 x 28.  The
// odd form with two rounds of pairs and the pipeline is held to three
// resident blocks per SM (80 registers at n = 10; 100 unbounded, i.e. two).
template <typename T, int n, bool PIPE, int FLEX, int XM = 0>
__global__ void __launch_bounds__(256, PIPE && XM == 2 && n * n * n / 2 > 256 ? 3 : 0)
k_cg_update_el(int E, int nx, int ny, int nz, FastDiv dnx, FastDiv dny,
               CgScalars *__restrict__ sc, T *__restrict__ x, T *__restrict__ r,
               const T *__restrict__ p, const T *__restrict__ p2, const T *__restrict__ w,
               const T *__restrict__ dinv, double *__restrict__ part)
{
    static_assert(XM == 0 || FLEX == 0, "deferred x steps are a Jacobi CG form");
    static_assert(n % 2 == 0, "pairs of nodes need an even n");
    using V = typename Pair2<T>::type;
    constexpr int N = n - 1, n2 = n * n, n3 = n2 * n, h = n / 2, P = n3 / 2;
    constexpr int R = (P + 255) / 256;  // rounds of 256 pairs per element
    __shared__ double sred[32];
    const int sx = n3 - N, sy = nx * n3 - N * n, sz = nx * ny * n3 - N * n2;
    // the thread's pair slots: local offset and face flags (bit 0..5: lower x
    // of the first node, upper x of the second, lower / upper y, lower / upper z)
    int loc[R], fl[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int t = threadIdx.x + 256 * q;
        const int i0 = 2 * (t % h), j = (t / h) % n, k = t / (h * n);
        loc[q] = t < P ? k * n2 + j * n + i0 : -1;
        fl[q] = (i0 == 0) | ((i0 + 1 == N) << 1) | ((j == 0) << 2) | ((j == N) << 3) |
                ((k == 0) << 4) | ((k == N) << 5);
    }
    pdl_wait();  // the previous kernel's alpha, w and p (programmatic dependent launch)
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    const T alpha_x = XM == 2 ? (T)sc->alpha_x : T(0);
    DotAcc<T> a, b;
    auto node = [&](T &xl, T &rl, T pl, T p2l, T wl, T d) {
        if (d == T(0)) wl = T(0);  // Dirichlet node
        if (XM == 2) xl = xl + alpha_x * p2l;
        if (XM != 1) xl = xl + alpha * pl;
        rl = rl - alpha * wl;
        if (owner_copy(d)) {
            if (FLEX == 0) a.add(rl * (d * rl));
            b.add(rl * rl);
        }
    };
    const int e0 = (int)((int64_t)E * blockIdx.x / gridDim.x);
    const int e1 = (int)((int64_t)E * (blockIdx.x + 1) / gridDim.x);
    // one element's loads: the summed w of the thread's pairs and x, r, p,
    // (p2,) dinv
    struct Buf {
        T wa[R], wb[R];
        V xv[R], rv[R], pv[R], p2v[R], dv[R];
    };
    auto load = [&](int e, Buf &B) {
        const int exy = dnx.div(e), ex = e - exy * nx;
        const int ez = dny.div(exy), ey = exy - ez * ny;
        // neighbour present below / above in each direction, in the bit layout of fl
        const int nb = (ex > 0) | ((ex < nx - 1) << 1) | ((ey > 0) << 2) | ((ey < ny - 1) << 3) |
                       ((ez > 0) << 4) | ((ez < nz - 1) << 5);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (loc[q] < 0) continue;
            const int l = e * n3 + loc[q], f = fl[q] & nb;
            gs_sum_pair_flags<T, int>(w, l, (f & 1) != 0, (f & 2) != 0, (f >> 2) & 1,
                                      (f >> 3) & 1, (f >> 4) & 1, (f >> 5) & 1, sx, sy, sz,
                                      B.wa[q], B.wb[q]);
            if (XM != 1) {
                B.xv[q] = *reinterpret_cast<const V *>(x + l);
                B.pv[q] = *reinterpret_cast<const V *>(p + l);
            }
            if (XM == 2) B.p2v[q] = *reinterpret_cast<const V *>(p2 + l);
            B.rv[q] = *reinterpret_cast<const V *>(r + l);
            B.dv[q] = *reinterpret_cast<const V *>(dinv + l);
        }
    };
    auto finish = [&](int e, Buf &B) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (loc[q] < 0) continue;
            const int l = e * n3 + loc[q];
            node(B.xv[q].x, B.rv[q].x, B.pv[q].x, B.p2v[q].x, B.wa[q], B.dv[q].x);
            node(B.xv[q].y, B.rv[q].y, B.pv[q].y, B.p2v[q].y, B.wb[q], B.dv[q].y);
            if (XM != 1) *reinterpret_cast<V *>(x + l) = B.xv[q];
            *reinterpret_cast<V *>(r + l) = B.rv[q];
        }
    };
    if constexpr (PIPE) {
        // software pipeline: the next element's loads are in flight while this
        // one is finished (w is read-only here; x and r of different elements)
        Buf A, Bn;
        int e = e0;
        if (e < e1) load(e, A);
        for (; e < e1; e += 2) {
            if (e + 1 < e1) load(e + 1, Bn);
            finish(e, A);
            if (e + 1 >= e1) break;
            if (e + 2 < e1) load(e + 2, A);
            finish(e + 1, Bn);
        }
    } else {
        for (int e = e0; e < e1; ++e) {
            Buf A;
            load(e, A);
            finish(e, A);
        }
    }
    if (sc->pdl_early) pdl_trigger();
    if constexpr (FLEX == 0) {
        double ta = block_sum_acc(a, sred);
        double tb = block_sum_acc(b, sred);
        if (threadIdx.x == 0) {
            part[blockIdx.x] = ta;
            part[gridDim.x + blockIdx.x] = tb;
        }
        if (last_block(&sc->tick_upd)) {
            cg_finish_iter(sc, part, gridDim.x, sred);
            if (XM != 0 && threadIdx.x == 0) {
                if (XM == 1) sc->alpha_x = sc->alpha;
                sc->x_pending = XM == 1;
            }
        }
    } else {
        const double tb = block_sum_acc(b, sred);
        if (threadIdx.x == 0) part[blockIdx.x] = tb;
        if (last_block(&sc->tick_upd)) fcg_finish_iter(sc, part, gridDim.x, sred);
    }
}

// The x step a Jacobi CG solve with deferred x steps still owes when it stops
// after the even iteration of a pair: x += alpha_x p2, and the last direction
// p2 into p (where a resumed solve reads it).  Nothing when none is pending.
template <typename T>
__global__ void k_x_flush(int64_t nL, const CgScalars *__restrict__ sc, T *__restrict__ x,
                          T *__restrict__ p, const T *__restrict__ p2)
{
    if (!sc->x_pending) return;
    const T a = (T)sc->alpha_x;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x) {
        const T pl = p2[l];
        x[l] = x[l] + a * pl;
        p[l] = pl;
    }
}

// k_cg_update_el with the element's contiguous x, r, p and dinv blocks
// streamed by bulk copies (cp.async.bulk) into a two-stage shared-memory ring,
// two elements ahead: each thread first issues the loads of w over the
// copies of its pairs (the only scattered reads), then waits for the ring,
// then updates from shared memory and stores x and r.  Same sums in the same
// order as k_cg_update_el.  Every wait is bounded (one second); a block that
// times out sets *err and the solve's status, drains its copies and stops.
template <int n>
constexpr int upd_tma_vecs()
{
    return 4;  // x, r, p, dinv
}

template <int n>
__global__ void __launch_bounds__(256)
k_cg_update_tma(int E, int nx, int ny, int nz, FastDiv dnx, FastDiv dny,
                CgScalars *__restrict__ sc, float *__restrict__ x, float *__restrict__ r,
                const float *__restrict__ p, const float *__restrict__ w,
                const float *__restrict__ dinv, double *__restrict__ part, int *__restrict__ err)
{
    static_assert(n % 2 == 0, "pairs of nodes need an even n");
    using V = float2;
    constexpr int N = n - 1, n2 = n * n, n3 = n2 * n, h = n / 2, P = n3 / 2;
    constexpr int R = (P + 255) / 256;
    constexpr int NV = upd_tma_vecs<n>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *stage = reinterpret_cast<float *>(smem_raw);  // [2][NV][n3]: x, r, p, dinv
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ double sred[32];
    if (sc->done) return;
    const float alpha = (float)sc->alpha;
    const int sx = n3 - N, sy = nx * n3 - N * n, sz = nx * ny * n3 - N * n2;
    int loc[R], fl[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int t = threadIdx.x + 256 * q;
        const int i0 = 2 * (t % h), j = (t / h) % n, k = t / (h * n);
        loc[q] = t < P ? k * n2 + j * n + i0 : -1;
        fl[q] = (i0 == 0) | ((i0 + 1 == N) << 1) | ((j == 0) << 2) | ((j == N) << 3) |
                ((k == 0) << 4) | ((k == N) << 5);
    }
    DotAcc<float> a, b;
    const int e0 = (int)((int64_t)E * blockIdx.x / gridDim.x);
    const int e1 = (int)((int64_t)E * (blockIdx.x + 1) / gridDim.x);
    const int cnt = e1 - e0;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int t) {  // element e0 + t into stage t & 1
        const int64_t off = (int64_t)(e0 + t) * n3;
        float *dst = stage + (t & 1) * NV * n3;
        constexpr uint32_t bytes = (uint32_t)(n3 * sizeof(float));
        mbar_expect_tx(&bar[t & 1], NV * bytes);
        bulk_g2s(dst + 0 * n3, x + off, bytes, &bar[t & 1]);
        bulk_g2s(dst + 1 * n3, r + off, bytes, &bar[t & 1]);
        bulk_g2s(dst + 2 * n3, p + off, bytes, &bar[t & 1]);
        bulk_g2s(dst + 3 * n3, dinv + off, bytes, &bar[t & 1]);
    };
    if (threadIdx.x == 0) {
        if (cnt > 0) issue(0);
        if (cnt > 1) issue(1);
    }
    int t = 0;
    for (; t < cnt; ++t) {
        const int e = e0 + t;
        const int exy = dnx.div(e), ex = e - exy * nx;
        const int ez = dny.div(exy), ey = exy - ez * ny;
        const int nb = (ex > 0) | ((ex < nx - 1) << 1) | ((ey > 0) << 2) | ((ey < ny - 1) << 3) |
                       ((ez > 0) << 4) | ((ez < nz - 1) << 5);
        float wa[R], wb[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (loc[q] < 0) continue;
            const int f = fl[q] & nb;
            gs_sum_pair_flags<float, int>(w, e * n3 + loc[q], (f & 1) != 0, (f & 2) != 0,
                                          (f >> 2) & 1, (f >> 3) & 1, (f >> 4) & 1, (f >> 5) & 1,
                                          sx, sy, sz, wa[q], wb[q]);
        }
        const bool ok = mbar_wait_bounded(&bar[t & 1], (uint32_t)((t >> 1) & 1));
        if (__syncthreads_or(!ok)) break;
        const float *sg = stage + (t & 1) * NV * n3;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (loc[q] < 0) continue;
            const int lq = loc[q];
            V xv = *reinterpret_cast<const V *>(sg + 0 * n3 + lq);
            V rv = *reinterpret_cast<const V *>(sg + 1 * n3 + lq);
            const V pv = *reinterpret_cast<const V *>(sg + 2 * n3 + lq);
            const V dv = *reinterpret_cast<const V *>(sg + 3 * n3 + lq);
            float wl[2] = {wa[q], wb[q]};
            float *xs[2] = {&xv.x, &xv.y}, *rs[2] = {&rv.x, &rv.y};
            const float ps[2] = {pv.x, pv.y}, ds[2] = {dv.x, dv.y};
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (ds[u] == 0.f) wl[u] = 0.f;  // Dirichlet node
                *xs[u] = *xs[u] + alpha * ps[u];
                *rs[u] = *rs[u] - alpha * wl[u];
                if (owner_copy(ds[u])) {
                    a.add(*rs[u] * (ds[u] * *rs[u]));
                    b.add(*rs[u] * *rs[u]);
                }
            }
            const int64_t l = (int64_t)e * n3 + lq;
            *reinterpret_cast<V *>(x + l) = xv;
            *reinterpret_cast<V *>(r + l) = rv;
        }
        __syncthreads();  // stage t & 1 consumed
        if (threadIdx.x == 0 && t + 2 < cnt) issue(t + 2);
    }
    if (t < cnt) {
        if (threadIdx.x == 0) {
            atomicExch(err, 1);
            sc->status = NB_BREAKDOWN;
            sc->done = 1;
            for (int tt = t; tt < t + 2 && tt < cnt; ++tt)
                mbar_wait_bounded(&bar[tt & 1], (uint32_t)((tt >> 1) & 1));
        }
        __syncthreads();
        return;
    }
    double ta = block_sum_acc(a, sred);
    double tb = block_sum_acc(b, sred);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ta;
        part[gridDim.x + blockIdx.x] = tb;
    }
    if (last_block(&sc->tick_upd)) cg_finish_iter(sc, part, gridDim.x, sred);
}

// Grid of a pair kernel: one wave of its resident blocks (per device, from
// the occupancy of its register count), and no more blocks than pairs need.
// (One cache per kernel: the template parameter is the kernel itself, not its
// type, which kernels of different orders share.)
template <auto kern>
static int update_pairs_grid(int sm_count, int npairs, size_t smem = 0)
{
    static int per_sm_dev[kMaxDevices] = {};
    int &per_sm = device_slot(per_sm_dev);
    if (per_sm == 0) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    const int64_t need = ((int64_t)npairs + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)per_sm * sm_count));
}

// The element-range update pipelines its element loop up to 100 elements per
// SM.  Measured (mixed solves): E=4096 N=9 61.3 against 63.6 ms, N=7 25.5
// against 27.1 ms, E=13824 N=7 108.1 against 110.2 ms; at E=32768 the plain
// loop's higher occupancy wins (N=9 783 against 825 ms).
static bool update_pipelined(const nb_mesh *m) { return m->E <= 100 * (int64_t)m->ctx->sm_count; }

// k_cg_update_gs for n = N + 1 in FP32 (returns false where it is not
// built).  FP64 keeps the separate summation: the folded sum adds every slot,
// zeros included, which costs little on the FP32 pipe but measured slower
// than the separate kernel on the FP64 pipe.
template <int NN, bool PIPE>
static cudaError_t launch_update_el_xm(nb_mesh *m, Workspace &ws, int xm, const float *dinv,
                                       double *part, cudaStream_t s);

// Whether the FP32 Jacobi update is the element-range kernel: even n, by
// choice (variant 1) or by default up to two rounds of 256 node pairs per
// element (n <= 10).
static bool update_el_used(const nb_mesh *m)
{
    const int n = m->n, rounds = (n * n * n / 2 + 255) / 256;
    return n % 2 == 0 && n >= 2 && n <= 16 &&
           (m->update_kind == 1 || (m->update_kind == 0 && rounds <= 2));
}

// xm: the x step form of the element-range kernel (0 where x is updated every
// iteration; 1, 2 the even and odd iteration of a pair with deferred x steps).
static bool launch_update_gs(nb_mesh *m, Workspace &ws, const float *dinv, double *part, int xm,
                             cudaStream_t s)
{
    // one wave: 8 blocks of 256 threads per SM
    const int grid = (int)std::min<int64_t>(m->E, (int64_t)m->ctx->sm_count * 8);
    // even n: the pair kernel over a full persistent grid (at most one pair
    // per thread fewer or more anywhere)
    const int npairs = (int)(m->nL / 2);
    const FastDiv dnx((uint32_t)m->nx), dny((uint32_t)m->ny);
    int pgrid = 0;
#define NB_UGS(K, NN)                                                                           \
    case NN:                                                                                    \
        K<float, NN><<<grid, 256, 0, s>>>(m->E, m->nx, m->ny, m->nz, ws.scal, (float *)ws.x,    \
                                          (float *)ws.r, (const float *)ws.p,                   \
                                          (const float *)ws.w, dinv, part);                     \
        return true;
#define NB_UGP(NN)                                                                              \
    case NN:                                                                                    \
        if (m->update_kind == 3) {                                                              \
            constexpr size_t sm_ = 2 * upd_tma_vecs<NN>() * sizeof(float) * NN * NN * NN;       \
            pgrid = update_pairs_grid<k_cg_update_tma<NN>>(m->ctx->sm_count,                    \
                                      (int)std::min<int64_t>(m->E * 256, npairs), sm_);         \
            pgrid = (int)std::min<int64_t>(pgrid, m->E);                                        \
            k_cg_update_tma<NN><<<pgrid, 256, sm_, s>>>(                                        \
                (int)m->E, m->nx, m->ny, m->nz, dnx, dny, ws.scal, (float *)ws.x,               \
                (float *)ws.r, (const float *)ws.p, (const float *)ws.w, dinv, part, m->kerr);  \
        } else if (update_el_used(m)) {                                                         \
            if (update_pipelined(m))                                                            \
                launch_update_el_xm<NN, true>(m, ws, xm, dinv, part, s);                        \
            else                                                                                \
                launch_update_el_xm<NN, false>(m, ws, xm, dinv, part, s);                       \
        } else {                                                                                \
            pgrid = update_pairs_grid<k_cg_update_pairs<float, NN>>(m->ctx->sm_count, npairs);  \
            k_cg_update_pairs<float, NN><<<pgrid, 256, 0, s>>>(                                 \
                npairs, m->nx, m->ny, m->nz, dnx, dny, ws.scal, (float *)ws.x, (float *)ws.r,   \
                (const float *)ws.p, (const float *)ws.w, dinv, part);                          \
        }                                                                                       \
        return true;
    switch (m->n) {
        NB_UGP(2) NB_UGS(k_cg_update_gs, 3) NB_UGP(4) NB_UGS(k_cg_update_gs, 5) NB_UGP(6)
        NB_UGS(k_cg_update_gs, 7) NB_UGP(8) NB_UGS(k_cg_update_gs, 9) NB_UGP(10)
        NB_UGS(k_cg_update_gs, 11) NB_UGP(12) NB_UGS(k_cg_update_gs, 13) NB_UGP(14)
        NB_UGS(k_cg_update_gs, 15) NB_UGP(16)
        default:
            return false;
    }
#undef NB_UGP
#undef NB_UGS
}

template <int NN, bool PIPE, int FLEX, int XM = 0>
static cudaError_t launch_update_el(nb_mesh *m, CgScalars *sc, float *x, float *r, const float *p,
                                   const float *p2, const float *w, const float *dinv,
                                   double *part, cudaStream_t s)
{
    const int npairs = (int)(m->nL / 2);
    int pgrid = update_pairs_grid<k_cg_update_el<float, NN, PIPE, FLEX, XM>>(
        m->ctx->sm_count, (int)std::min<int64_t>(m->E * 256, npairs));
    pgrid = (int)std::min<int64_t>(pgrid, m->E);
    const FastDiv dnx((uint32_t)m->nx), dny((uint32_t)m->ny);
    return launch_pdl(k_cg_update_el<float, NN, PIPE, FLEX, XM>, pgrid, 256, 0, s, (int)m->E,
                      m->nx, m->ny, m->nz, dnx, dny, sc, x, r, p, p2, w, dinv, part);
}

// The Jacobi update over element ranges with x step form xm (see
// k_cg_update_el).
template <int NN, bool PIPE>
static cudaError_t launch_update_el_xm(nb_mesh *m, Workspace &ws, int xm, const float *dinv,
                                       double *part, cudaStream_t s)
{
    float *x = (float *)ws.x, *r = (float *)ws.r;
    const float *p = (const float *)ws.p, *p2 = (const float *)ws.p2, *w = (const float *)ws.w;
    if (xm == 1) return launch_update_el<NN, PIPE, 0, 1>(m, ws.scal, x, r, p, p2, w, dinv, part, s);
    if (xm == 2) return launch_update_el<NN, PIPE, 0, 2>(m, ws.scal, x, r, p, p2, w, dinv, part, s);
    return launch_update_el<NN, PIPE, 0, 0>(m, ws.scal, x, r, p, nullptr, w, dinv, part, s);
}

// The flexible-CG update over element ranges: x, r with the summation of w
// folded in, (r, r) and the stopping step.  False (nothing launched) where the
// element-range form is not used: odd n, more than two rounds of 256 node
// pairs per element (n > 10), and with rg, the Schwarz path's scatter of the
// new r.  Measured: the learned flexible CG at E=4096, N=7 28.7 against
// 30.3 ms; the Schwarz solve at N=9 39.8 against 39.1 ms with the scatter in
// this kernel, so that path keeps the one-block-per-element kernel.
bool launch_fcg_update_el(nb_mesh *m, Workspace &ws, float *x, float *r, const float *p,
                          const float *w, double *part, float *rg, cudaStream_t s)
{
    if (rg) return false;
    const bool pipe = update_pipelined(m);
    const float *dinv = m->dinv32;
    cudaError_t e = cudaSuccess;
#define NB_FEL(NN)                                                                               \
    case NN:                                                                                     \
        e = pipe ? launch_update_el<NN, true, 1>(m, ws.scal, x, r, p, nullptr, w, dinv, part, s) \
                 : launch_update_el<NN, false, 1>(m, ws.scal, x, r, p, nullptr, w, dinv, part, s);\
        break;
    switch (m->n) {
        NB_FEL(2) NB_FEL(4) NB_FEL(6) NB_FEL(8) NB_FEL(10)
        default:
            return false;
    }
#undef NB_FEL
    (void)e;  // a launch error is reported by the caller's cudaGetLastError
    return true;
}

// The while-node condition of the captured iteration.  It counts executions
// of the loop body itself, so the loop ends after maxit + 1 bodies even if
// no other kernel of the body managed to set `done`.
__global__ void k_cg_cond(CgScalars *sc, cudaGraphConditionalHandle h)
{
    const int loops = sc->loops + 1;
    sc->loops = loops;
    const bool stop = sc->done != 0 || loops > sc->maxit;
    cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// r = b - w (FP64) and partials of (r, c, r).
__global__ void k_residual64(int64_t nL, const double *__restrict__ b, const double *__restrict__ w,
                             const float *__restrict__ c, double *__restrict__ r,
                             double *__restrict__ part)
{
    __shared__ double sred[32];
    double a = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x) {
        const double v = b[l] - (w ? w[l] : 0.0);
        r[l] = v;
        a += (double)c[l] * v * v;
    }
    double t = block_sum(a, sred);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Inner right-hand side: r32 = r64 / s (rounded to FP32), x32 = 0.
__global__ void k_demote(int64_t nL, const double *__restrict__ r64, const double *__restrict__ s2,
                         float *__restrict__ r32, float *__restrict__ x32)
{
    const double inv = 1.0 / sqrt(*s2);
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x) {
        r32[l] = (float)(r64[l] * inv);
        x32[l] = 0.0f;
    }
}

// The FP64 inner solve's start: r = r64, x = 0.
__global__ void k_stage64(int64_t nL, const double *__restrict__ r64, double *__restrict__ r,
                          double *__restrict__ x)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x) {
        r[l] = r64[l];
        x[l] = 0.0;
    }
}

// x += d in FP64.
__global__ void k_add64(int64_t nL, const double *__restrict__ d, double *__restrict__ x)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x)
        x[l] += d[l];
}

// Solution update in FP64: x += s * d.
__global__ void k_promote(int64_t nL, const double *__restrict__ s2, const float *__restrict__ d,
                          double *__restrict__ x)
{
    const double sc = sqrt(*s2);
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nL;
         l += (int64_t)gridDim.x * blockDim.x)
        x[l] += sc * (double)d[l];
}

__global__ void k_fill0(int64_t n, double *__restrict__ x)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x)
        x[l] = 0.0;
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------

nb_status ensure_ws(nb_mesh *m, Workspace &ws, int elt, int hist_cap)
{
    if (ws.x == nullptr) {
        const size_t bytes = (size_t)elt * m->nL;
        ws.nL = m->nL;
        ws.elt = elt;
        NB_CUDA(cudaMalloc(&ws.x, bytes));
        NB_CUDA(cudaMalloc(&ws.r, bytes));
        NB_CUDA(cudaMalloc(&ws.p, bytes));
        NB_CUDA(cudaMalloc(&ws.w, bytes));
        NB_CUDA(cudaMalloc(&ws.z, bytes));
        NB_CUDA(cudaMalloc(&ws.aux, bytes));
        NB_CUDA(cudaMalloc(&ws.part, sizeof(double) * kMaxPartials * 3));
        NB_CUDA(cudaMalloc(&ws.scal, sizeof(CgScalars)));
        NB_CUDA(cudaMallocHost(&ws.scal_host, sizeof(CgScalars)));
        NB_CUDA(cudaMemset(ws.scal, 0, sizeof(CgScalars)));
        NB_CUDA(cudaMemset(ws.r, 0, bytes));
        NB_CUDA(cudaMemset(ws.p, 0, bytes));
        NB_CUDA(cudaMemset(ws.x, 0, bytes));
    }
    if (hist_cap > ws.hist_cap) {
        if (ws.hist) NB_CUDA(cudaFree(ws.hist));
        ws.hist = nullptr;
        NB_CUDA(cudaMalloc(&ws.hist, sizeof(double) * hist_cap));
        ws.hist_cap = hist_cap;
    }
    return NB_OK;
}

static nb_status ensure_fp64_bufs(nb_mesh *m)
{
    if (m->r64 == nullptr) {
        NB_CUDA(cudaMalloc(&m->r64, sizeof(double) * m->nL));
        NB_CUDA(cudaMalloc(&m->w64, sizeof(double) * m->nL));
        NB_CUDA(cudaMalloc(&m->part64, sizeof(double) * kMaxPartials * 2));
    }
    if (m->red_out == nullptr) {
        NB_CUDA(cudaMalloc(&m->red_out, sizeof(double) * 8));
        NB_CUDA(cudaMallocHost(&m->red_host, sizeof(double) * 8));
    }
    return NB_OK;
}

// Kernels of one captured iteration: operator, update with the summation
// folded in (or summation and update), loop condition.
static int cg_body_kernels(const nb_mesh *m, nb_prec prec)
{
    return prec != NB_FP64 && m->n >= 2 && m->n <= 16 ? 3 : 4;
}

// The launches of one iteration (see the file comment): operator (its last
// block computes alpha), gather-scatter, update (its last block computes
// beta and the stopping test), and inside a graph the loop condition.
// use_cond: 1 in a graph, ending the body with the loop condition; 2 in a
// graph, an iteration followed by another one of the same body; 0 launched
// from the host.  In FP32 the operator and the update go out with
// programmatic dependent launch.  xm (FP32, see defer_x): 0 one direction
// buffer, x stepped every iteration; 1 the even iteration of a pair (p read,
// p2 written, no x step); 2 the odd one (p2 read, p written, both x steps).
template <typename T>
static nb_status cg_body(nb_mesh *m, nb_prec prec, Workspace &ws, const T *dinv,
                         cudaGraphConditionalHandle h, int use_cond, int xm, cudaStream_t s)
{
    PdlScope pdl(sizeof(T) == 4);
    int nparts = 0;
    if (xm != 0) {
        float *pa = (float *)ws.p, *pb = (float *)ws.p2;
        NB_TRY(ax_cg_step_from(m, (const float *)ws.r, (const float *)dinv, xm == 1 ? pa : pb,
                               xm == 1 ? pb : pa, (float *)ws.w, ws.scal, ws.part, &nparts, s));
    } else {
        NB_TRY(ax_cg_step(m, prec, ws.r, dinv, ws.p, ws.w, ws.scal, ws.part, &nparts, s));
    }
    double *up = ws.part + kMaxPartials;
    bool folded = false;
    if constexpr (sizeof(T) == 4) folded = launch_update_gs(m, ws, (const float *)dinv, up, xm, s);
    if (!folded && xm != 0) {
        set_error("deferred x steps need the element-range update");
        return NB_ERR_ARG;
    }
    if (!folded) {
        NB_TRY(dssum(m, prec, ws.w, 1, s));
        const int g = vec_grid(m->ctx, m->nL);
        k_cg_update<T><<<g, kVecThreads, 0, s>>>(m->nL, ws.scal, (T *)ws.x, (T *)ws.r,
                                                 (const T *)ws.p, (const T *)ws.w, dinv, up);
    }
    NB_CUDA(cudaGetLastError());
    if (use_cond == 1) {
        k_cg_cond<<<1, 1, 0, s>>>(ws.scal, h);
        NB_CUDA(cudaGetLastError());
    } else if (use_cond == 0) {
        m->launches += cg_body_kernels(m, prec) - 1;
    }
    return NB_OK;
}

// Iterations per captured loop body: two in FP32, so that the second
// operator follows the first update inside the body (a programmatic
// dependent launch); the kernels of an iteration after convergence return at
// once.
template <typename T>
constexpr int cg_body_iters()
{
    return sizeof(T) == 4 ? 2 : 1;
}

// Kernel launches of a graph-run inner solve, from the executed loop bodies.
static int64_t graph_launches(const nb_mesh *m, nb_prec prec, const CgScalars &h)
{
    const int per_iter = cg_body_kernels(m, prec) - 1;  // without the condition
    const int iters = prec == NB_FP64 ? 1 : 2;
    return (int64_t)std::max(h.loops, 1) * (iters * per_iter + 1);
}

// Initial scalars from ws.r: p = 0, rtz, rtr, relres, done.
template <typename T>
static nb_status cg_start(nb_mesh *m, Workspace &ws, const T *dinv, double tol, int maxit,
                          int bnorm_from_r, bool hist, cudaStream_t s)
{
    k_cg_setup<<<1, 1, 0, s>>>(ws.scal, tol, maxit, hist ? ws.hist : nullptr,
                               hist ? ws.hist_cap : 0, pdl_early_for(m->E, m->ctx->sm_count));
    NB_CUDA(cudaGetLastError());
    const int g = vec_grid(m->ctx, m->nL);
    k_cg_init<T><<<g, kVecThreads, 0, s>>>(m->nL, (const T *)ws.r, dinv, (T *)ws.p,
                                           ws.part + kMaxPartials, 1);
    NB_CUDA(cudaGetLastError());
    k_cg_init_fin<<<1, kFinalizeThreads, 0, s>>>(ws.scal, ws.part + kMaxPartials, g, bnorm_from_r);
    NB_CUDA(cudaGetLastError());
    m->launches += 3;
    return NB_OK;
}

// The same after a residual replacement, keeping the search direction p
// (see k_cg_resume_fin; c = s_old / s_new).
template <typename T>
static nb_status cg_resume(nb_mesh *m, Workspace &ws, const T *dinv, double tol, int maxit,
                           bool hist, double c, cudaStream_t s)
{
    k_cg_setup<<<1, 1, 0, s>>>(ws.scal, tol, maxit, hist ? ws.hist : nullptr,
                               hist ? ws.hist_cap : 0, pdl_early_for(m->E, m->ctx->sm_count));
    NB_CUDA(cudaGetLastError());
    const int g = vec_grid(m->ctx, m->nL);
    k_cg_init<T><<<g, kVecThreads, 0, s>>>(m->nL, (const T *)ws.r, dinv, (T *)ws.p,
                                           ws.part + kMaxPartials, 0);
    NB_CUDA(cudaGetLastError());
    k_cg_resume_fin<<<1, kFinalizeThreads, 0, s>>>(ws.scal, ws.part + kMaxPartials, g, c);
    NB_CUDA(cudaGetLastError());
    m->launches += 3;
    return NB_OK;
}

// The loop of cg_iterate: a captured graph with a device-side loop
// condition, or chunks of iterations launched from the host.
template <typename T>
static nb_status cg_loop(nb_mesh *m, nb_prec prec, Workspace &ws, const T *dinv, int key,
                         int use_graph, int maxit, bool defer, cudaStream_t s)
{
    if (use_graph) {
        if (ws.exec == nullptr || ws.graph_key != key || ws.graph_epoch != m->ax_epoch) {
            if (ws.exec) {
                NB_CUDA(cudaGraphExecDestroy(ws.exec));
                ws.exec = nullptr;
            }
            if (ws.graph) {
                NB_CUDA(cudaGraphDestroy(ws.graph));
                ws.graph = nullptr;
            }
            cudaGraph_t g;
            NB_CUDA(cudaGraphCreate(&g, 0));
            cudaGraphConditionalHandle h;
            NB_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t node;
            NB_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            NB_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed));
            nb_status st = NB_OK;
            for (int i = 0; i < cg_body_iters<T>() && st == NB_OK; ++i)
                st = cg_body<T>(m, prec, ws, dinv, h, i + 1 == cg_body_iters<T>() ? 1 : 2,
                                defer ? 1 + i : 0, s);
            cudaGraph_t captured = nullptr;
            cudaError_t ce = cudaStreamEndCapture(s, &captured);
            if (st != NB_OK) {
                cudaGraphDestroy(g);
                return st;
            }
            if (ce != cudaSuccess) {
                cudaGraphDestroy(g);
                set_error("graph capture failed: %s", cudaGetErrorString(ce));
                return NB_ERR_CUDA;
            }
            NB_CUDA(cudaGraphInstantiate(&ws.exec, g, 0));
            ws.graph = g;
            ws.graph_key = key;
            ws.graph_epoch = m->ax_epoch;
        }
        NB_CUDA(cudaGraphLaunch(ws.exec, s));
        return NB_OK;
    }
    // host-driven: launch a chunk of iterations, then look at the flag (an
    // even number: with deferred x steps every chunk is whole pairs)
    const int chunk = 16;
    for (int done_iters = 0; done_iters <= maxit; done_iters += chunk) {
        for (int t = 0; t < chunk; ++t)
            NB_TRY(cg_body<T>(m, prec, ws, dinv, 0, 0, defer ? 1 + (t & 1) : 0, s));
        NB_CUDA(cudaMemcpyAsync(ws.scal_host, ws.scal, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                                s));
        NB_CUDA(cudaStreamSynchronize(s));
        if (ws.scal_host->done) break;
    }
    return NB_OK;
}

// Jacobi CG in FP32 with the pencil operator and the element-range update
// defers the x step over pairs of iterations where the loop's vectors do not
// fit in L2: the operator alternates two direction buffers, so that the even
// iteration's update reads neither x nor p and the odd one applies both steps
// (16 + 32 instead of 2 x 28 bytes per local node in the update).  Measured
// (mixed solves): E=13824 N=9 254.4 against 271.3 ms, E=32768 N=7 290.8
// against 297.2 ms; where x, r, p, w and dinv stay in L2 the sixth vector
// costs more than it saves (E=4096 N=9 61.3 against 59.8 ms), so the rule is
// the six vectors' 24 bytes per local node against the L2 size
// (nb_set_x_deferral overrides it).
static bool defer_x(const nb_mesh *m, nb_prec prec, const Workspace &ws)
{
    if (m->x_defer == 0 || prec != NB_FP32 || ws.elt != 4 || !update_el_used(m) ||
        !ax_cg_step_from_available(m))
        return false;
    return m->x_defer == 1 || (double)24 * m->nL > (double)m->ctx->l2_bytes;
}

// Run iterations until the device scalars say stop.
template <typename T>
static nb_status cg_iterate(nb_mesh *m, nb_prec prec, Workspace &ws, const T *dinv, int key,
                            int use_graph, int maxit, cudaStream_t s)
{
    const bool defer = sizeof(T) == 4 && defer_x(m, prec, ws);
    if (defer && ws.p2 == nullptr) {
        NB_CUDA(cudaMalloc(&ws.p2, (size_t)ws.elt * ws.nL));
        NB_CUDA(cudaMemsetAsync(ws.p2, 0, (size_t)ws.elt * ws.nL, s));
    }
    NB_TRY(cg_loop<T>(m, prec, ws, dinv, key, use_graph, maxit, defer, s));
    if (defer) {
        const int g = vec_grid(m->ctx, m->nL);
        k_x_flush<float><<<g, kVecThreads, 0, s>>>(m->nL, ws.scal, (float *)ws.x, (float *)ws.p,
                                                   (const float *)ws.p2);
        NB_CUDA(cudaGetLastError());
        m->launches += 1;
    }
    return NB_OK;
}

// ||b - A x||_c^2 in FP64 into m->red_out[slot]; r into m->r64.
static nb_status fp64_residual(nb_mesh *m, const double *b, const double *x, int slot,
                               cudaStream_t s)
{
    const double *w = nullptr;
    if (x) {
        NB_TRY(ax_local(m, NB_FP64, x, m->w64, nullptr, nullptr, s));
        NB_TRY(dssum(m, NB_FP64, m->w64, 1, s));
        w = m->w64;
    }
    const int g = vec_grid(m->ctx, m->nL);
    k_residual64<<<g, kVecThreads, 0, s>>>(m->nL, b, w, m->c32, m->r64, m->part64);
    NB_CUDA(cudaGetLastError());
    m->launches += x ? 4 : 2;
    return sum_partials_dev(m->part64, g, m->red_out + slot, s);
}

static void copy_history(const Workspace &ws, int count, int offset, nb_stats *st,
                         cudaStream_t s)
{
    if (!st || !st->history_host || st->history_cap <= offset || count <= 0) return;
    int nmax = std::min(count, std::min(ws.hist_cap, st->history_cap - offset));
    if (nmax <= 0) return;
    cudaMemcpyAsync(st->history_host + offset, ws.hist, sizeof(double) * nmax,
                    cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    st->history_len = offset + nmax;
}

static nb_status solve_fp64(nb_mesh *m, const nb_opts *o, const double *b, double *x,
                            nb_stats *st, cudaStream_t s)
{
    Workspace &ws = m->ws64;
    const int hist_cap = o->record_history ? std::max(o->maxiter, 1) : 0;
    NB_TRY(ensure_ws(m, ws, 8, hist_cap));
    NB_TRY(ensure_fp64_bufs(m));
    const double *dinv = o->pc == NB_PC_NONE ? m->ones64 : m->dinv64;
    // bnorm2 -> scal (through red_out), r = b - A x0
    NB_TRY(fp64_residual(m, b, nullptr, 0, s));  // (b, c, b)
    NB_TRY(fp64_residual(m, b, o->use_x0 ? x : nullptr, 1, s));
    NB_CUDA(cudaMemcpyAsync(ws.r, m->r64, sizeof(double) * m->nL, cudaMemcpyDeviceToDevice, s));
    if (o->use_x0)
        NB_CUDA(cudaMemcpyAsync(ws.x, x, sizeof(double) * m->nL, cudaMemcpyDeviceToDevice, s));
    else
        NB_CUDA(cudaMemsetAsync(ws.x, 0, sizeof(double) * m->nL, s));
    NB_CUDA(cudaMemcpyAsync(&ws.scal->bnorm2, m->red_out, sizeof(double),
                            cudaMemcpyDeviceToDevice, s));
    NB_TRY(cg_start<double>(m, ws, dinv, o->rtol, o->maxiter, 0, o->record_history, s));
    NB_TRY(cg_iterate<double>(m, NB_FP64, ws, dinv, 10 + (int)o->pc, o->use_graph, o->maxiter, s));
    NB_CUDA(cudaMemcpyAsync(x, ws.x, sizeof(double) * m->nL, cudaMemcpyDeviceToDevice, s));
    // true FP64 residual of the result
    NB_TRY(fp64_residual(m, b, x, 1, s));
    NB_CUDA(cudaMemcpyAsync(ws.scal_host, ws.scal, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaMemcpyAsync(m->red_host, m->red_out, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    const CgScalars &h = *ws.scal_host;
    if (!isfinite(m->red_host[0])) {
        set_error("right-hand side has a non-finite entry");
        return NB_ERR_ARG;
    }
    const double bn2 = m->red_host[0] > 0 ? m->red_host[0] : 1.0;
    if (st) {
        if (o->use_graph)
            m->launches += graph_launches(m, NB_FP64, h);
        st->iters = h.iter;
        st->outer_iters = 0;
        st->launches = m->launches;
        st->rel_res = sqrt(m->red_host[1] / bn2);
        st->status = (nb_status)h.status;
        st->history_len = 0;
        st->final_prec = NB_FP64;
    }
    if (o->record_history) copy_history(ws, h.iter, 0, st, s);
    return (nb_status)h.status;
}

// Largest inner tolerance of a reliable-update segment (residual replaced at
// least every 2 decades), and the longest inner solve after which the
// direction is still kept: beyond it (elongated boxes needing thousands of
// iterations per 2 decades) the FP32 recurrence drifts from the true
// residual, a resumed solve stagnates, and restarts are faster.
constexpr double kReliableDrop = 1e-2;
constexpr int kReliableMaxIters = 1000;
constexpr int kReliableShort = 15;

static nb_status solve_refined(nb_mesh *m, const nb_opts *o, const double *b, double *x,
                               nb_stats *st, cudaStream_t s)
{
    Workspace &ws = m->ws32;
    const int hist_cap = o->record_history ? std::max(o->maxiter, 1) : 0;
    NB_TRY(ensure_ws(m, ws, 4, hist_cap));
    NB_TRY(ensure_fp64_bufs(m));
    const float *dinv = o->pc == NB_PC_NONE ? m->ones32 : m->dinv32;
    const int g = vec_grid(m->ctx, m->nL);
    NB_TRY(fp64_residual(m, b, nullptr, 0, s));  // (b, c, b) into red_out[0]
    if (!o->use_x0) {
        k_fill0<<<g, kVecThreads, 0, s>>>(m->nL, x);
        NB_CUDA(cudaGetLastError());
        m->launches += 1;
    }
    int used = 0, outer = 0, stagn = 0, hist_off = 0;
    double prev = INFINITY, rel = INFINITY;
    // reliable update: an inner solve of the same kind as the previous one,
    // which converged, resumes with its direction; s2_prev is the previous
    // residual scale squared, prev_kind 0 none, 1 (P)CG, 2 learned, 3 Schwarz
    int prev_kind = 0, prev_iters = 0;
    bool prev_ok = false;
    double s2_prev = 0.0, prev_end = 1.0, rel_start = 1.0;
    // reliable updates while the solve stays well within FP32's reach; after
    // a long inner solve or a failed resumption, classic restarted refinement
    bool reliable = !o->restart;
    nb_status result = NB_NOT_CONVERGED;
    bool fell_back = false;
    // precision adaptivity: the inner solves' precision, raised one step
    // (tensor-core 16-bit contractions -> FP32 -> FP64) when the FP64
    // residual stops dropping at the current one
    nb_prec inner = o->prec;
    constexpr int kLearnedBudget = 3000;  // flexible-CG iterations per refinement step
    for (outer = 0; outer <= o->max_outer; ++outer) {
        // FP64 residual r = b - A x (skipped product for the zero start)
        NB_TRY(fp64_residual(m, b, (outer == 0 && !o->use_x0) ? nullptr : x, 1, s));
        NB_CUDA(cudaMemcpyAsync(m->red_host, m->red_out, sizeof(double) * 2,
                                cudaMemcpyDeviceToHost, s));
        NB_CUDA(cudaStreamSynchronize(s));
        const double bn2 = m->red_host[0];
        if (!isfinite(bn2)) {
            set_error("right-hand side has a non-finite entry");
            return NB_ERR_ARG;
        }
        if (!(bn2 > 0.0)) {  // b = 0: x = 0 is exact
            rel = 0.0;
            result = NB_OK;
            break;
        }
        rel = sqrt(m->red_host[1] / bn2);
        if (!isfinite(rel)) { result = NB_BREAKDOWN; break; }
        if (rel < o->rtol) { result = NB_OK; break; }
        if (outer == o->max_outer || used >= o->maxiter) { result = NB_NOT_CONVERGED; break; }
        if (rel > 0.5 * prev) {
            if ((o->pc == NB_PC_LEARNED || o->pc == NB_PC_SCHWARZ || o->pc == NB_PC_SCHWARZ2) &&
                !fell_back) {
                fell_back = true;  // the learned steps stopped paying: Jacobi-PCG takes over
                stagn = 0;
            } else if (inner != NB_FP64 && ++stagn >= 2) {
                // two steps without progress: the inner precision cannot
                // resolve the correction any more (its operator error times
                // the condition number is near one); raise it one step, and
                // restart the inner solves in the new precision
                inner = inner == NB_FP32 ? NB_FP64 : NB_FP32;
                stagn = 0;
                reliable = false;
                prev_ok = false;
            } else if (inner == NB_FP64 && ++stagn >= 3) {
                result = NB_STAGNATED;
                break;
            }
        } else {
            stagn = 0;
        }
        prev = rel;
        // two-level Schwarz: the coarse-grid correction in FP64 on the FP64
        // residual (x += R_0^T A_0^-1 R_0 r, r -= A that); the FP32 inner solves
        // leave errors of FP32 size in the smoothest modes, whose residual the
        // stopping test does not resolve
        double rel_in = rel;
        if (o->pc == NB_PC_SCHWARZ2 && !fell_back && inner == NB_FP32) {
            bool applied = false;
            NB_TRY(schwarz_coarse_correct64(m, m->r64, x, (float *)ws.x, (float *)ws.r, m->part64,
                                            m->red_out + 1, &applied, s));
            if (applied) {
                NB_CUDA(cudaMemcpyAsync(m->red_host + 1, m->red_out + 1, sizeof(double),
                                        cudaMemcpyDeviceToHost, s));
                NB_CUDA(cudaStreamSynchronize(s));
                rel_in = sqrt(m->red_host[1] / bn2);
                if (!isfinite(rel_in)) { result = NB_BREAKDOWN; break; }
                if (rel_in == 0.0) { rel = 0.0; result = NB_OK; break; }  // x is exact
            }
        }
        const int remaining = o->maxiter - used;
        if (inner == NB_FP64) {
            // the precision raised to FP64: PCG in FP64 on A d = r64 to the
            // step's tolerance, then x += d
            Workspace &w64 = m->ws64;
            NB_TRY(ensure_ws(m, w64, 8, 0));
            const double *dinv64 = o->pc == NB_PC_NONE ? m->ones64 : m->dinv64;
            const double tau64 = std::min(0.5, std::max(o->inner_rtol, 0.5 * o->rtol / rel_in));
            k_stage64<<<g, kVecThreads, 0, s>>>(m->nL, m->r64, (double *)w64.r, (double *)w64.x);
            NB_CUDA(cudaGetLastError());
            NB_TRY(cg_start<double>(m, w64, dinv64, tau64, remaining, 1, false, s));
            NB_TRY(cg_iterate<double>(m, NB_FP64, w64, dinv64, 10 + (int)NB_PC_JACOBI,
                                      o->use_graph, remaining, s));
            k_add64<<<g, kVecThreads, 0, s>>>(m->nL, (const double *)w64.x, x);
            NB_CUDA(cudaGetLastError());
            NB_CUDA(cudaMemcpyAsync(w64.scal_host, w64.scal, sizeof(CgScalars),
                                    cudaMemcpyDeviceToHost, s));
            NB_CUDA(cudaStreamSynchronize(s));
            const int it64 = w64.scal_host->iter;
            m->launches += 2 + (o->use_graph ? graph_launches(m, NB_FP64, *w64.scal_host) : 0);
            used += it64;
            prev_kind = 0;
            prev_ok = false;
            if (w64.scal_host->status == NB_BREAKDOWN && it64 == 0) { result = NB_BREAKDOWN; break; }
            continue;
        }
        // inner solve on r32 = r64/||r64||, from zero
        k_demote<<<g, kVecThreads, 0, s>>>(m->nL, m->r64, m->red_out + 1, (float *)ws.r,
                                           (float *)ws.x);
        NB_CUDA(cudaGetLastError());
        const bool schwarz = o->pc == NB_PC_SCHWARZ || o->pc == NB_PC_SCHWARZ2;
        const bool use_learned = (o->pc == NB_PC_LEARNED || schwarz) && !fell_back;
        // the inner solve only has to close the remaining gap to rtol (with a
        // factor 2 of margin), and never less than inner_rtol per step.  With
        // the direction kept (reliable update) the residual is replaced at
        // least every 2 decades: the FP32 recurrence then stays close to the
        // true residual, and the iteration count stays that of FP64 PCG
        // (941 against 936 at E=4096, N=9; 6061 with replacements every 5
        // decades, where the recurrence drifts)
        const int kind = !use_learned ? 1 : (schwarz ? 2 + (int)o->pc : 2);
        const bool keep_dir = reliable;
        // resume only where the FP32 recurrence agreed with the true residual:
        // the FP64 residual dropped to at most 100x what the recurrence
        // claimed (else it drifted and the kept direction would mislead the
        // next solve: restart)
        const bool agreed = outer > 0 && rel / rel_start <= 100.0 * prev_end;
        const bool resume = keep_dir && prev_ok && prev_kind == kind && agreed;
        // a resumed solve that needs more than eight times the previous
        // solve's iterations (plus 200) stops, and the next step restarts (the
        // second solve, after the first 2 decades, typically takes 4x the first)
        const int cap = resume ? 8 * prev_iters + 200 : remaining;
        const bool odd = (prev_iters & 1) != 0;
        // with the Schwarz preconditioners, after a short inner solve (the
        // recurrence has little room to drift) the next one may close
        // inner_rtol again, which saves FP64 residuals (measured there: the
        // two-level solve needs 4 refinement steps instead of 5)
        const bool short_prev = resume && schwarz && prev_iters < kReliableShort;
        const double step_rtol =
            keep_dir && !short_prev ? std::max(o->inner_rtol, kReliableDrop) : o->inner_rtol;
        const double tau = std::min(0.5, std::max(step_rtol, 0.5 * o->rtol / rel_in));
        if (use_learned && schwarz) {
            // flexible CG with the Schwarz preconditioner (nb_schwarz.cu)
            k_cg_setup<<<1, 1, 0, s>>>(ws.scal, tau, std::min(remaining, cap),
                                       o->record_history ? ws.hist : nullptr,
                                       o->record_history ? ws.hist_cap : 0,
                                       pdl_early_for(m->E, m->ctx->sm_count));
            NB_CUDA(cudaGetLastError());
            NB_TRY(fcg_schwarz(m, inner, ws, o, resume, odd, s));
        } else if (use_learned) {
            // flexible CG with the learned preconditioner (nb_learned.cu), on a
            // bounded budget; Jacobi-PCG takes over if it fails
            k_cg_setup<<<1, 1, 0, s>>>(ws.scal, tau,
                                       std::min(std::min(remaining, cap), kLearnedBudget),
                                       o->record_history ? ws.hist : nullptr,
                                       o->record_history ? ws.hist_cap : 0,
                                       pdl_early_for(m->E, m->ctx->sm_count));
            NB_CUDA(cudaGetLastError());
            NB_TRY(fcg_learned(m, inner, ws, o, resume, odd, s));
        } else {
            if (resume)
                NB_TRY(cg_resume<float>(m, ws, dinv, tau, std::min(remaining, cap), o->record_history,
                                        sqrt(s2_prev / m->red_host[1]), s));
            else
                NB_TRY(cg_start<float>(m, ws, dinv, tau, remaining, 1, o->record_history, s));
            NB_TRY(cg_iterate<float>(m, inner, ws, dinv, 20 * (int)inner + (int)o->pc,
                                     o->use_graph, remaining, s));
        }
        s2_prev = m->red_host[1];
        k_promote<<<g, kVecThreads, 0, s>>>(m->nL, m->red_out + 1, (const float *)ws.x, x);
        NB_CUDA(cudaGetLastError());
        m->launches += 2;  // demote + promote
        NB_CUDA(cudaMemcpyAsync(ws.scal_host, ws.scal, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                                s));
        NB_CUDA(cudaStreamSynchronize(s));
        const int it = ws.scal_host->iter;
        if (o->use_graph && !use_learned) m->launches += graph_launches(m, inner, *ws.scal_host);
        if (o->record_history) {
            copy_history(ws, it, hist_off, st, s);
            hist_off += it;
        }
        used += it;
        // an inner solve of more than kReliableMaxIters iterations (an
        // ill-conditioned problem: the FP32 recurrence drifts over it) or a
        // resumed one that hit its cap ends the reliable updates of this solve
        if (it > kReliableMaxIters || (resume && it >= cap)) reliable = false;
        prev_kind = kind;
        prev_ok = ws.scal_host->status == 0 && it > 0;
        prev_iters = it;
        prev_end = ws.scal_host->relres;  // the recurrence's drop over this solve
        rel_start = rel_in;
        const bool capped = resume && it >= cap && ws.scal_host->status == NB_NOT_CONVERGED;
        if (use_learned && ws.scal_host->status != 0 && !capped) {
            fell_back = true;  // the learned step failed: Jacobi-PCG from here on
            prev = INFINITY;
            stagn = 0;
            continue;
        }
        if (ws.scal_host->status == NB_BREAKDOWN && it == 0) { result = NB_BREAKDOWN; break; }
    }
    if (result == NB_OK && fell_back) result = NB_FELL_BACK;
    if (st) {
        st->iters = used;
        st->outer_iters = outer;
        st->launches = m->launches;
        st->rel_res = rel;
        st->status = result;
        st->final_prec = inner;
        if (o->record_history) st->history_len = std::min(hist_off, st->history_cap);
    }
    return result;
}

// ---------------------------------------------------------------------------
// The CG iteration in split phases, for drivers that combine several meshes
// (the slabs of a partitioned box): each call does one step of Table 1 on
// this mesh and returns its partial dot products; the caller sums them over
// the meshes and passes alpha and beta back.
// ---------------------------------------------------------------------------

__global__ void k_split_scalars(CgScalars *sc, double alpha, double beta)
{
    sc->alpha = alpha;
    sc->beta = beta;
    sc->rtz = 1.0;
    sc->rtz_old = 1.0;
    sc->bnorm2 = 1.0;
    sc->tol = 0.0;
    sc->maxit = 0x7fffffff;
    sc->iter = 0;
    sc->done = 0;
    sc->status = 0;
    sc->hist = nullptr;
    sc->hist_cap = 0;
}

static nb_status split_scalars(nb_mesh *m)
{
    if (!m->scal_split) {
        NB_CUDA(cudaMalloc(&m->scal_split, sizeof(CgScalars)));
        NB_CUDA(cudaMemset(m->scal_split, 0, sizeof(CgScalars)));
    }
    NB_TRY(ensure_fp64_bufs(m));
    return NB_OK;
}

nb_status split_step(nb_mesh *m, nb_prec prec, double beta, const void *r, void *p, void *w,
                     double *pap, cudaStream_t s)
{
    NB_TRY(split_scalars(m));
    k_split_scalars<<<1, 1, 0, s>>>(m->scal_split, 0.0, beta);
    NB_CUDA(cudaGetLastError());
    const void *dinv = prec == NB_FP64 ? (const void *)m->dinv64 : (const void *)m->dinv32;
    int nparts = 0;
    NB_TRY(ax_cg_step(m, prec, r, dinv, p, w, m->scal_split, m->part64, &nparts, s));
    NB_CUDA(cudaMemcpyAsync(m->red_host, &m->scal_split->pap, sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    *pap = m->red_host[0];
    return NB_OK;
}

nb_status split_update(nb_mesh *m, nb_prec prec, double alpha, void *x, void *r, const void *p,
                       const void *w, double out[2], cudaStream_t s)
{
    NB_TRY(split_scalars(m));
    k_split_scalars<<<1, 1, 0, s>>>(m->scal_split, alpha, 0.0);
    NB_CUDA(cudaGetLastError());
    const int g = vec_grid(m->ctx, m->nL);
    if (prec == NB_FP64)
        k_cg_update<double><<<g, kVecThreads, 0, s>>>(m->nL, m->scal_split, (double *)x,
                                                      (double *)r, (const double *)p,
                                                      (const double *)w, m->dinv64, m->part64);
    else
        k_cg_update<float><<<g, kVecThreads, 0, s>>>(m->nL, m->scal_split, (float *)x,
                                                     (float *)r, (const float *)p,
                                                     (const float *)w, m->dinv32, m->part64);
    NB_CUDA(cudaGetLastError());
    NB_CUDA(cudaMemcpyAsync(m->red_host, &m->scal_split->rtz, sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaMemcpyAsync(m->red_host + 1, &m->scal_split->rtr, sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    out[0] = m->red_host[0];
    out[1] = m->red_host[1];
    return NB_OK;
}

nb_status split_dots(nb_mesh *m, nb_prec prec, const void *r, double out[2], cudaStream_t s)
{
    NB_TRY(split_scalars(m));
    const int g = vec_grid(m->ctx, m->nL);
    if (prec == NB_FP64)
        k_cg_init<double><<<g, kVecThreads, 0, s>>>(m->nL, (const double *)r, m->dinv64, nullptr,
                                                    m->part64, 0);
    else
        k_cg_init<float><<<g, kVecThreads, 0, s>>>(m->nL, (const float *)r, m->dinv32, nullptr,
                                                   m->part64, 0);
    NB_CUDA(cudaGetLastError());
    NB_TRY(sum_partials_dev(m->part64, g, m->red_out, s));
    NB_TRY(sum_partials_dev(m->part64 + g, g, m->red_out + 1, s));
    NB_CUDA(cudaMemcpyAsync(m->red_host, m->red_out, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                            s));
    NB_CUDA(cudaStreamSynchronize(s));
    out[0] = m->red_host[0];
    out[1] = m->red_host[1];
    return NB_OK;
}

nb_status solve(nb_mesh *m, const nb_opts *o, const double *b, double *x, nb_stats *st)
{
    cudaStream_t s = m->ctx->stream;
    cudaEvent_t e0, e1;
    NB_CUDA(cudaEventCreate(&e0));
    NB_CUDA(cudaEventCreate(&e1));
    NB_CUDA(cudaEventRecord(e0, s));
    m->launches = 0;
    nb_status r = o->prec == NB_FP64 ? solve_fp64(m, o, b, x, st, s)
                                      : solve_refined(m, o, b, x, st, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) st->seconds = ms * 1e-3;
    return r;
}

}  // namespace nb
