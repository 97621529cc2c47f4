// Batched solves: many independent Poisson problems of different element
// count and order in one solve.
//
// Layout.  The problems' L-vectors are concatenated with the problems grouped
// by order, so every order's elements form one contiguous range; geometric
// factors and the Jacobi arrays follow the same order, and the gather-scatter
// rows of all problems form one list (local indices offset into the batch).
// Per-element tables give each element's problem and L offset.
//
// Iteration.  Table 1's loop for all problems at once: the operator (one
// launch per order present), the per-problem alpha (one warp per problem sums
// its elements' partials in element order), the gather-scatter, the update
// (one block per element), the per-problem beta and stopping tests, and the
// loop condition "some problem is still running".  The iteration is one CUDA
// graph with a while node, launched for K iterations at a time.
//
// Active lists.  Every kernel walks device lists of the elements (per order,
// and over all orders) and of the gather-scatter row chunks of the problems
// still running; between graph launches the host reads the problems' flags
// and rebuilds the lists once a quarter of the listed elements belong to
// problems that have stopped, so a batch whose stragglers run for thousands
// of iterations pays for the stragglers only.  Problems that stopped within
// a launch are skipped by every kernel.  The FP64 refinement around the loop
// runs per problem (own scale, own inner tolerance) with the running problems
// advanced together.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "nb_cg_dev.cuh"

namespace nb {

nb_status bax_f32(int n, int mchoice, bool pupd, int sm_count, long long E, long long e_first,
                  const int32_t *list, const int *cnt, const float *G, const float *u, float *w,
                  const float *r, const float *dinv, float *p, const int32_t *elem_prob,
                  const BScal *bs, double *part_e, cudaStream_t s);
nb_status bax_f64(int n, int mchoice, bool pupd, int sm_count, long long E, long long e_first,
                  const int32_t *list, const int *cnt, const double *G, const double *u,
                  double *w, const double *r, const double *dinv, double *p,
                  const int32_t *elem_prob, const BScal *bs, double *part_e, cudaStream_t s);

nb_status bax_tma_f32(int n, int sm_count, long long E, long long e_first, const int32_t *list,
                      const int *cnt, const float *G, float *w, const float *r, const float *dinv,
                      float *p, const int32_t *elem_prob, BScal *bs, double *part_e, int *err,
                      cudaStream_t s);
bool bax_tma_available_f32(int n);

constexpr int kRowChunk = 2048;  // gather-scatter rows per list entry

struct BatchGroup {
    int n = 0;
    int64_t e0 = 0, e1 = 0;  // element range
    int64_t l0 = 0;          // L offset of the first element
    int variant = 1;         // FP32 step: 0, 1 elements-per-block choices, 2 bulk copy (autotuned)
};

struct BatchWs {
    void *x = nullptr, *r = nullptr, *p = nullptr, *w = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace nb

struct nb_batch {
    nb_ctx *ctx = nullptr;
    int nprob = 0;
    std::vector<nb_mesh *> meshes;  // caller order
    std::vector<int> order;         // internal index -> caller index
    std::vector<int> rank;          // caller index -> internal index
    std::vector<int64_t> l_off, g_off;  // caller order
    int64_t nL = 0, nG = 0, E = 0, rows = 0;
    std::vector<nb::BatchGroup> groups;
    std::vector<int64_t> prob_e0_host;  // internal order, nprob + 1
    std::vector<int64_t> prob_row0_host;  // internal order, nprob + 1: gather-scatter rows
    std::vector<int> prob_group;        // internal order: index into groups
    float *G32 = nullptr;
    double *G64 = nullptr;
    float *dinv32 = nullptr;
    double *dinv64 = nullptr;
    int32_t *gs_off = nullptr, *gs_loc = nullptr;
    uint8_t *gs_mask = nullptr;
    int32_t *elem_prob = nullptr;  // [E] internal problem index
    int64_t *elem_l0 = nullptr;    // [E + 1]
    int64_t *prob_e0 = nullptr;    // [nprob + 1]
    int4 *prob_dim = nullptr;      // [nprob] (nx, ny, nz, n) of each problem's box
    nb::BScal *bs = nullptr;       // [nprob]
    nb::BScal *bs_host = nullptr;  // pinned
    int *loops = nullptr;          // graph loop counter
    int *loops_host = nullptr;     // pinned mirror
    int *kerr = nullptr;           // device flag: a bulk-copy wait timed out
    double *part_e = nullptr;      // [2 E]
    double *red = nullptr;         // [4 nprob]: |r|^2, |b|^2, tau, active
    double *red_host = nullptr;    // pinned
    double *r64 = nullptr, *w64 = nullptr;
    nb::BatchWs ws32, ws64;
    // active lists (device, one allocation; pinned mirror): counts
    // [groups: elements per order, all elements, row chunks], then per order
    // the element list in the order's slot [e0, e1), the list over all
    // orders, and the row chunks (first row, end row, problem, 0)
    int *act = nullptr;
    int *act_host = nullptr;
    int64_t act_words = 0, act_e_off = 0, act_all_off = 0, act_ch_off = 0, max_chunks = 0;
    std::vector<char> act_run;  // problems the lists currently hold
    int64_t act_elems = 0;
};

namespace nb {

// ---------------------------------------------------------------------------
// kernels (per-element loops: one block per element, grid-stride)
// ---------------------------------------------------------------------------

// Sum of a[lo..hi) by one warp in a fixed order (lane-strided, then a fixed
// shuffle tree), returned on lane 0.
__device__ __forceinline__ double warp_range_sum(const double *a, int64_t lo, int64_t hi)
{
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    for (int64_t e = lo + lane; e < hi; e += 32) v += a[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over a warp by a fixed shuffle tree, on lane 0.
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Element lists: batch element indices with their count on the device; a
// null list stands for every element.
__device__ __forceinline__ int64_t list_len(const int *cnt, int64_t E)
{
    return cnt ? (int64_t)*cnt : E;
}
__device__ __forceinline__ int64_t list_at(const int32_t *list, int64_t i)
{
    return list ? (int64_t)list[i] : i;
}

__global__ void k_bsetup(int nprob, BScal *bs, double tol, int maxit, const double *red,
                         int use_red)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    BScal b = {};
    b.tol = use_red ? red[2 * nprob + p] : tol;
    b.maxit = maxit;
    b.done = use_red ? (red[3 * nprob + p] == 0.0) : 0;
    bs[p] = b;
}

// Bodies of one graph launch: loops[0] counts them, loops[1] + 1 is the cap.
__global__ void k_bchunk(int *loops, int cap)
{
    loops[0] = 0;
    loops[1] = cap;
}

// p = 0 and owner-copy partials of (r, dinv r), (r, r) per listed element
// (one warp per element).
template <typename T>
__global__ void k_binit(int64_t E, const int32_t *__restrict__ list, const int *__restrict__ cnt,
                        const int64_t *__restrict__ el0, const T *__restrict__ r,
                        const T *__restrict__ dinv, T *__restrict__ p, double *__restrict__ part)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t ne = list_len(cnt, E);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < ne;
         i += nwarps) {
        const int64_t e = list_at(list, i);
        DotAcc<T> a, b;
        for (int64_t l = el0[e] + lane; l < el0[e + 1]; l += 32) {
            const T rl = r[l], d = dinv[l];
            p[l] = T(0);
            if (!signbit(d)) {
                a.add(rl * (d * rl));
                b.add(rl * rl);
            }
        }
        const double ta = warp_sum(a.value());
        const double tb = warp_sum(b.value());
        if (lane == 0) {
            part[e] = ta;
            part[E + e] = tb;
        }
    }
}

__global__ void k_bfin_init(int nprob, const int64_t *__restrict__ pe0, const double *part,
                            int64_t E, BScal *bs, int bnorm_from_r, const double *bnorm2)
{
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= nprob) return;
    const double rtz = warp_range_sum(part, pe0[p], pe0[p + 1]);
    const double rtr = warp_range_sum(part + E, pe0[p], pe0[p + 1]);
    if ((threadIdx.x & 31) == 0) {
        BScal &b = bs[p];
        b.rtz = b.rtz_old = rtz;
        b.rtr = rtr;
        if (bnorm_from_r) b.bnorm2 = rtr;
        else if (bnorm2) b.bnorm2 = bnorm2[p];
        const double bn = b.bnorm2 > 0.0 ? b.bnorm2 : 1.0;
        b.relres = sqrt(rtr / bn);
        b.beta = 0.0;
        if (b.done) return;
        if (!isfinite(b.relres)) {
            b.done = 1;
            b.status = NB_BREAKDOWN;
        } else if (b.relres < b.tol || rtr == 0.0) {
            b.done = 1;
        } else if (b.maxit <= 0) {
            b.done = 1;
            b.status = NB_NOT_CONVERGED;
        }
    }
}

__global__ void k_bfin_alpha(int nprob, const int64_t *__restrict__ pe0, const double *part,
                             BScal *bs)
{
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= nprob) return;
    if (bs[p].done) return;  // uniform over the warp
    const double pap = warp_range_sum(part, pe0[p], pe0[p + 1]);
    if ((threadIdx.x & 31) == 0) {
        BScal &b = bs[p];
        b.pap = pap;
        const double alpha = b.rtz / pap;
        if (!(pap > 0.0) || !isfinite(alpha)) {
            b.alpha = 0.0;
            b.done = 1;
            b.status = NB_BREAKDOWN;
        } else {
            b.alpha = alpha;
        }
    }
}

// Masked direct-stiffness summation over the listed row chunks, copies
// summed in ascending local order (as k_gs); chunks of problems that have
// stopped are skipped when bs is given.
template <typename T>
__global__ void k_bgs(const int4 *__restrict__ ch, const int *__restrict__ cnt,
                      const int32_t *__restrict__ off, const int32_t *__restrict__ loc,
                      const uint8_t *__restrict__ rmask, const BScal *__restrict__ bs,
                      T *__restrict__ u)
{
    const int nc = *cnt;
    for (int c = blockIdx.x; c < nc; c += gridDim.x) {
        const int4 q = ch[c];
        if (bs && bs[q.z].done) continue;  // uniform over the block
        for (int a = q.x + threadIdx.x; a < q.y; a += blockDim.x) {
            const int o0 = off[a], o1 = off[a + 1];
            T s = T(0);
            for (int o = o0; o < o1; ++o) s += u[loc[o]];
            if (rmask[a] == 0) s = T(0);
            for (int o = o0; o < o1; ++o) u[loc[o]] = s;
        }
    }
}

// x += alpha_q p, r -= alpha_q w and the owner-copy partials of (r, dinv r),
// (r, r) per listed element: one warp per element (lane-strided, coalesced),
// the partials summed by a fixed shuffle tree.
template <typename T>
__global__ void k_bupdate(int64_t E, const int32_t *__restrict__ list, const int *__restrict__ cnt,
                          const int64_t *__restrict__ el0,
                          const int32_t *__restrict__ eprob, const BScal *__restrict__ bs,
                          T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p,
                          const T *__restrict__ w, const T *__restrict__ dinv,
                          double *__restrict__ part)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t ne = list_len(cnt, E);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < ne;
         i += nwarps) {
        const int64_t e = list_at(list, i);
        const BScal &b = bs[eprob[e]];
        if (b.done) continue;  // uniform over the warp
        const T alpha = (T)b.alpha;
        DotAcc<T> a, c;
        for (int64_t l = el0[e] + lane; l < el0[e + 1]; l += 32) {
            x[l] = x[l] + alpha * p[l];
            const T rl = r[l] - alpha * w[l];
            r[l] = rl;
            const T d = dinv[l];
            if (!signbit(d)) {
                a.add(rl * (d * rl));
                c.add(rl * rl);
            }
        }
        const double ta = warp_sum(a.value());
        const double tc = warp_sum(c.value());
        if (lane == 0) {
            part[e] = ta;
            part[E + e] = tc;
        }
    }
}

// k_bupdate with the direct-stiffness summation of w folded in (FP32): per
// node, w_asm = mask * the sum of w over the node's copies -- its mirror nodes
// in the neighbouring elements of the problem's box (i = 0 of element ex is
// i = N of ex - 1, and so on per direction) -- in ascending local index, the
// order of k_bgs, so the result is bit-identical to k_bgs + k_bupdate.  The
// mask is dinv == 0 (Dirichlet).  A warp per active element.
__global__ void k_bupdate_gs(int64_t E, const int32_t *__restrict__ list, const int *__restrict__ cnt,
                             const int64_t *__restrict__ el0, const int32_t *__restrict__ eprob,
                             const int64_t *__restrict__ pe0, const int4 *__restrict__ pdim,
                             const BScal *__restrict__ bs, float *__restrict__ x,
                             float *__restrict__ r, const float *__restrict__ p,
                             const float *__restrict__ w, const float *__restrict__ dinv,
                             double *__restrict__ part)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t ne = list_len(cnt, E);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < ne;
         i += nwarps) {
        const int64_t e = list_at(list, i);
        const int pr = eprob[e];
        const BScal &b = bs[pr];
        if (b.done) continue;  // uniform over the warp
        const float alpha = (float)b.alpha;
        const int4 dm = pdim[pr];
        const int nx = dm.x, ny = dm.y, nz = dm.z, n = dm.w, N = n - 1, n2 = n * n, n3 = n2 * n;
        // batch local indices are below 2^31 (checked at set-up)
        const int el = (int)(e - pe0[pr]);
        const int ex = el % nx, ey = (el / nx) % ny, ez = el / (nx * ny);
        const int sx = n3 - N, sy = nx * n3 - N * n, sz = nx * ny * n3 - N * n2;
        DotAcc<float> a, c;
        const int l0 = (int)el0[e];
        for (int q = lane; q < n3; q += 32) {
            const int l = l0 + q;
            const int ii = q % n, jj = (q / n) % n, kk = q / n2;
            const int lx = ii == 0 && ex > 0, hx = ii == N && ex < nx - 1;
            const int ly = jj == 0 && ey > 0, hy = jj == N && ey < ny - 1;
            const int lz = kk == 0 && ez > 0, hz = kk == N && ez < nz - 1;
            const int w0 = l - lx * sx - ly * sy - lz * sz;
            float v[2][2][2];
#pragma unroll
            for (int tz = 0; tz < 2; ++tz)
#pragma unroll
                for (int ty = 0; ty < 2; ++ty)
#pragma unroll
                    for (int tx = 0; tx < 2; ++tx) {
                        const bool ok = tz <= lz + hz && ty <= ly + hy && tx <= lx + hx;
                        v[tz][ty][tx] = ok ? w[w0 + tx * sx + ty * sy + tz * sz] : 0.f;
                    }
            float wl = 0.f;
#pragma unroll
            for (int tz = 0; tz < 2; ++tz)
#pragma unroll
                for (int ty = 0; ty < 2; ++ty)
#pragma unroll
                    for (int tx = 0; tx < 2; ++tx) wl += v[tz][ty][tx];
            const float d = dinv[l];
            if (d == 0.f) wl = 0.f;  // Dirichlet node
            x[l] = x[l] + alpha * p[l];
            const float rl = r[l] - alpha * wl;
            r[l] = rl;
            if (!signbit(d)) {
                a.add(rl * (d * rl));
                c.add(rl * rl);
            }
        }
        const double ta = warp_sum(a.value());
        const double tc = warp_sum(c.value());
        if (lane == 0) {
            part[e] = ta;
            part[E + e] = tc;
        }
    }
}

__global__ void k_bfin_iter(int nprob, const int64_t *__restrict__ pe0, const double *part,
                            int64_t E, BScal *bs)
{
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= nprob) return;
    if (bs[p].done) return;
    const double rtz = warp_range_sum(part, pe0[p], pe0[p + 1]);
    const double rtr = warp_range_sum(part + E, pe0[p], pe0[p + 1]);
    if ((threadIdx.x & 31) == 0) {
        BScal &b = bs[p];
        b.rtz_old = b.rtz;
        b.rtz = rtz;
        b.rtr = rtr;
        b.beta = rtz / b.rtz_old;
        b.iter += 1;
        const double bn = b.bnorm2 > 0.0 ? b.bnorm2 : 1.0;
        b.relres = sqrt(rtr / bn);
        if (!isfinite(b.relres) || !isfinite(b.beta)) {
            b.done = 1;
            b.status = NB_BREAKDOWN;
        } else if (b.relres < b.tol) {
            b.done = 1;
        } else if (b.iter >= b.maxit) {
            b.done = 1;
            b.status = NB_NOT_CONVERGED;
        }
    }
}

// Loop condition: some problem still running, and at most maxit + 1 bodies.
__global__ void k_bcond(int nprob, const BScal *bs, int *loops, cudaGraphConditionalHandle h)
{
    int running = 0;
    for (int p = threadIdx.x; p < nprob; p += blockDim.x) running |= (bs[p].done == 0);
    running = __syncthreads_or(running);
    if (threadIdx.x == 0) {
        const int l = loops[0] + 1;
        loops[0] = l;
        cudaGraphSetConditional(h, (running && l <= loops[1]) ? 1u : 0u);
    }
}

// r = b - w (w may be NULL) and owner-copy partials of (r, r) and (b, b)
// per listed element.
__global__ void k_bresid(int64_t E, const int32_t *__restrict__ list, const int *__restrict__ cnt,
                         const int64_t *__restrict__ el0, const double *__restrict__ b,
                         const double *__restrict__ w, const double *__restrict__ dinv,
                         double *__restrict__ r, double *__restrict__ part)
{
    __shared__ double sred[32];
    const int64_t ne = list_len(cnt, E);
    for (int64_t i = blockIdx.x; i < ne; i += gridDim.x) {
        const int64_t e = list_at(list, i);
        double a = 0.0, c = 0.0;
        for (int64_t l = el0[e] + threadIdx.x; l < el0[e + 1]; l += blockDim.x) {
            const double bl = b[l];
            const double v = bl - (w ? w[l] : 0.0);
            r[l] = v;
            if (!signbit(dinv[l])) {
                a += v * v;
                c += bl * bl;
            }
        }
        const double ta = block_sum(a, sred);
        const double tc = block_sum(c, sred);
        if (threadIdx.x == 0) {
            part[e] = ta;
            part[E + e] = tc;
        }
    }
}

__global__ void k_bsum2(int nprob, const int64_t *__restrict__ pe0, const double *part, int64_t E,
                        double *out)
{
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= nprob) return;
    const double a = warp_range_sum(part, pe0[p], pe0[p + 1]);
    const double c = warp_range_sum(part + E, pe0[p], pe0[p + 1]);
    if ((threadIdx.x & 31) == 0) {
        out[p] = a;
        out[nprob + p] = c;
    }
}

// Inner right-hand side per problem: r32 = r64 / |r64| for running problems
// (zero otherwise), x32 = 0.  red[3 nprob + p] = 1 marks a running problem.
__global__ void k_bdemote(int64_t E, const int32_t *__restrict__ list, const int *__restrict__ cnt,
                          const int64_t *__restrict__ el0,
                          const int32_t *__restrict__ eprob, int nprob, const double *red,
                          const double *__restrict__ r64, float *__restrict__ r32,
                          float *__restrict__ x32)
{
    const int64_t ne = list_len(cnt, E);
    for (int64_t i = blockIdx.x; i < ne; i += gridDim.x) {
        const int64_t e = list_at(list, i);
        const int p = eprob[e];
        const bool act = red[3 * nprob + p] != 0.0;
        const double inv = act ? 1.0 / sqrt(red[p]) : 0.0;
        for (int64_t l = el0[e] + threadIdx.x; l < el0[e + 1]; l += blockDim.x) {
            r32[l] = (float)(r64[l] * inv);
            x32[l] = 0.0f;
        }
    }
}

__global__ void k_bpromote(int64_t E, const int32_t *__restrict__ list,
                           const int *__restrict__ cnt, const int64_t *__restrict__ el0,
                           const int32_t *__restrict__ eprob, int nprob, const double *red,
                           const float *__restrict__ x32, double *__restrict__ x)
{
    const int64_t ne = list_len(cnt, E);
    for (int64_t i = blockIdx.x; i < ne; i += gridDim.x) {
        const int64_t e = list_at(list, i);
        const int p = eprob[e];
        if (red[3 * nprob + p] == 0.0) continue;
        const double s = sqrt(red[p]);
        for (int64_t l = el0[e] + threadIdx.x; l < el0[e + 1]; l += blockDim.x)
            x[l] += s * (double)x32[l];
    }
}

__global__ void k_bcopy(int64_t n, const double *__restrict__ a, double *__restrict__ b)
{
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x)
        b[l] = a[l];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static int elem_grid(const nb_batch *B) { return (int)std::min<int64_t>(B->E, B->ctx->sm_count * 16); }
// one warp per element, 8 per block of 256 threads
static int warp_elem_grid(const nb_batch *B)
{
    return (int)std::min<int64_t>((B->E + 7) / 8, B->ctx->sm_count * 16);
}
static int warp_grid(int nprob) { return (nprob * 32 + 255) / 256; }
static int chunk_grid(const nb_batch *B)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>(B->max_chunks, B->ctx->sm_count * 8));
}

// device views of the active lists
static const int *cnt_group(const nb_batch *B, int g) { return B->act + g; }
static const int32_t *list_group(const nb_batch *B, int g)
{
    return B->act + B->act_e_off + B->groups[g].e0;
}
static const int *cnt_all(const nb_batch *B) { return B->act + B->groups.size(); }
static const int32_t *list_all(const nb_batch *B) { return B->act + B->act_all_off; }
static const int *cnt_chunks(const nb_batch *B) { return B->act + B->groups.size() + 1; }
static const int4 *list_chunks(const nb_batch *B)
{
    return reinterpret_cast<const int4 *>(B->act + B->act_ch_off);
}

// Make the lists hold the elements and row chunks of the problems marked in
// run (internal order).  One host-to-device copy; nothing is done if the
// lists already hold that set.
static nb_status set_active(nb_batch *B, const std::vector<char> &run, cudaStream_t s)
{
    if (run == B->act_run) return NB_OK;
    NB_CUDA(cudaStreamSynchronize(s));  // the pinned mirror of the last upload is free again
    int *h = B->act_host;
    const int ng = (int)B->groups.size();
    int32_t *le = h + B->act_e_off, *la = h + B->act_all_off;
    int4 *ch = reinterpret_cast<int4 *>(h + B->act_ch_off);
    std::fill(h, h + ng + 2, 0);
    int nall = 0, nch = 0;
    for (int q = 0; q < B->nprob; ++q) {
        if (!run[q]) continue;
        const int g = B->prob_group[q];
        for (int64_t e = B->prob_e0_host[q]; e < B->prob_e0_host[q + 1]; ++e) {
            le[B->groups[g].e0 + h[g]++] = (int32_t)e;
            la[nall++] = (int32_t)e;
        }
        const int64_t r1 = B->prob_row0_host[q + 1];
        for (int64_t r = B->prob_row0_host[q]; r < r1; r += kRowChunk)
            ch[nch++] = make_int4((int)r, (int)std::min<int64_t>(r + kRowChunk, r1), q, 0);
    }
    h[ng] = nall;
    h[ng + 1] = nch;
    NB_CUDA(cudaMemcpyAsync(B->act, h, sizeof(int) * B->act_words, cudaMemcpyHostToDevice, s));
    B->act_run = run;
    B->act_elems = nall;
    return NB_OK;
}

// The operator on one order's listed elements (variant: see BatchGroup).
template <typename T>
static nb_status bax_group(nb_batch *B, int gi, int variant, bool pupd, const T *u, T *w,
                           const T *r, const T *dinv, T *p, double *part, cudaStream_t s)
{
    const BatchGroup &g = B->groups[gi];
    const int64_t E = g.e1 - g.e0;
    const size_t lo = (size_t)g.l0, go = (size_t)g.l0 * 6;
    auto off = [&](const T *v) { return v ? v + lo : nullptr; };
    if (sizeof(T) == 4 && pupd && variant == 2)
        return bax_tma_f32(g.n, B->ctx->sm_count, E, g.e0, list_group(B, gi), cnt_group(B, gi),
                           (const float *)B->G32 + go, (float *)(w + lo), (const float *)off(r),
                           (const float *)off(dinv), (float *)(p + lo), B->elem_prob, B->bs,
                           part, B->kerr, s);
    const int mchoice = variant == 0 ? 0 : 1;
    if (sizeof(T) == 4)
        return bax_f32(g.n, mchoice, pupd, B->ctx->sm_count, E, g.e0, list_group(B, gi),
                       cnt_group(B, gi), (const float *)B->G32 + go, (const float *)off(u),
                       (float *)(w + lo), (const float *)off(r), (const float *)off(dinv),
                       p ? (float *)(p + lo) : nullptr, B->elem_prob, B->bs, part, s);
    return bax_f64(g.n, mchoice, pupd, B->ctx->sm_count, E, g.e0, list_group(B, gi),
                   cnt_group(B, gi), (const double *)B->G64 + go, (const double *)off(u),
                   (double *)(w + lo), (const double *)off(r), (const double *)off(dinv),
                   p ? (double *)(p + lo) : nullptr, B->elem_prob, B->bs, part, s);
}

template <typename T>
static nb_status bax_all(nb_batch *B, bool pupd, const T *u, T *w, const T *r, const T *dinv,
                         T *p, double *part, cudaStream_t s)
{
    for (int gi = 0; gi < (int)B->groups.size(); ++gi)
        NB_TRY(bax_group<T>(B, gi, B->groups[gi].variant, pupd, u, w, r, dinv, p, part, s));
    return NB_OK;
}

template <typename T>
static nb_status batch_body(nb_batch *B, BatchWs &ws, const T *dinv, int use_cond,
                            cudaGraphConditionalHandle h, cudaStream_t s)
{
    NB_TRY(bax_all<T>(B, true, nullptr, (T *)ws.w, (const T *)ws.r, dinv, (T *)ws.p, B->part_e, s));
    k_bfin_alpha<<<warp_grid(B->nprob), 256, 0, s>>>(B->nprob, B->prob_e0, B->part_e, B->bs);
    NB_CUDA(cudaGetLastError());
    if constexpr (sizeof(T) == 4) {  // summation folded into the update
        k_bupdate_gs<<<warp_elem_grid(B), 256, 0, s>>>(
            B->E, list_all(B), cnt_all(B), B->elem_l0, B->elem_prob, B->prob_e0, B->prob_dim,
            B->bs, (float *)ws.x, (float *)ws.r, (const float *)ws.p, (const float *)ws.w,
            (const float *)dinv, B->part_e);
    } else {
        k_bgs<T><<<chunk_grid(B), 256, 0, s>>>(list_chunks(B), cnt_chunks(B), B->gs_off,
                                               B->gs_loc, B->gs_mask, B->bs, (T *)ws.w);
        NB_CUDA(cudaGetLastError());
        k_bupdate<T><<<warp_elem_grid(B), 256, 0, s>>>(B->E, list_all(B), cnt_all(B),
                                                  B->elem_l0, B->elem_prob, B->bs, (T *)ws.x,
                                                  (T *)ws.r, (const T *)ws.p, (const T *)ws.w,
                                                  dinv, B->part_e);
    }
    NB_CUDA(cudaGetLastError());
    k_bfin_iter<<<warp_grid(B->nprob), 256, 0, s>>>(B->nprob, B->prob_e0, B->part_e, B->E, B->bs);
    NB_CUDA(cudaGetLastError());
    if (use_cond) {
        k_bcond<<<1, 256, 0, s>>>(B->nprob, B->bs, B->loops, h);
        NB_CUDA(cudaGetLastError());
    }
    return NB_OK;
}

static nb_status ensure_bws(nb_batch *B, BatchWs &ws, size_t elt)
{
    if (ws.x) return NB_OK;
    const size_t bytes = elt * B->nL;
    NB_CUDA(cudaMalloc(&ws.x, bytes));
    NB_CUDA(cudaMalloc(&ws.r, bytes));
    NB_CUDA(cudaMalloc(&ws.p, bytes));
    NB_CUDA(cudaMalloc(&ws.w, bytes));
    NB_CUDA(cudaMemset(ws.p, 0, bytes));
    NB_CUDA(cudaMemset(ws.w, 0, bytes));
    return NB_OK;
}

// Run the batched PCG on ws (r holds the residuals of the current x) for the
// problems in the active lists until every one has stopped.  Tolerances from
// red (per problem) if use_red; relative to |r0| if bnorm_from_r, else to
// bnorm2[p].  The loop runs up to K iterations per graph launch (K doubling
// up to 512 while no list is rebuilt); the kernels launched are added to
// *launches.
template <typename T>
static nb_status batch_cg(nb_batch *B, BatchWs &ws, const T *dinv, double tol, int maxit,
                          int use_red, int use_graph, int bnorm_from_r, const double *bnorm2,
                          cudaStream_t s, int64_t *launches)
{
    // operator per order, alpha, (summation,) update, beta, (condition)
    const int64_t per_body =
        (int64_t)B->groups.size() + (sizeof(T) == 4 ? 3 : 4) + (use_graph ? 1 : 0);
    *launches += 3;
    k_bsetup<<<(B->nprob + 255) / 256, 256, 0, s>>>(B->nprob, B->bs, tol, maxit, B->red, use_red);
    NB_CUDA(cudaGetLastError());
    k_binit<T><<<warp_elem_grid(B), 256, 0, s>>>(B->E, list_all(B), cnt_all(B), B->elem_l0,
                                            (const T *)ws.r, dinv, (T *)ws.p, B->part_e);
    NB_CUDA(cudaGetLastError());
    k_bfin_init<<<warp_grid(B->nprob), 256, 0, s>>>(B->nprob, B->prob_e0, B->part_e, B->E, B->bs,
                                                    bnorm_from_r, bnorm2);
    NB_CUDA(cudaGetLastError());
    if (use_graph && !ws.exec) {
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
        nb_status st = batch_body<T>(B, ws, dinv, 1, h, s);
        cudaGraph_t captured = nullptr;
        cudaError_t ce = cudaStreamEndCapture(s, &captured);
        if (st != NB_OK || ce != cudaSuccess) {
            cudaGraphDestroy(g);
            if (st != NB_OK) return st;
            set_error("batch graph capture failed: %s", cudaGetErrorString(ce));
            return NB_ERR_CUDA;
        }
        NB_CUDA(cudaGraphInstantiate(&ws.exec, g, 0));
        ws.graph = g;
    }
    std::vector<char> run(B->nprob);
    int K = 32;
    int64_t done_bodies = 0;
    for (;;) {
        if (use_graph) {
            k_bchunk<<<1, 1, 0, s>>>(B->loops, K - 1);  // the first body runs unconditionally
            NB_CUDA(cudaGetLastError());
            NB_CUDA(cudaGraphLaunch(ws.exec, s));
            NB_CUDA(cudaMemcpyAsync(B->loops_host, B->loops, sizeof(int), cudaMemcpyDeviceToHost,
                                    s));
        } else {
            for (int t = 0; t < K; ++t) NB_TRY(batch_body<T>(B, ws, dinv, 0, 0, s));
        }
        NB_CUDA(cudaMemcpyAsync(B->bs_host, B->bs, sizeof(BScal) * B->nprob,
                                cudaMemcpyDeviceToHost, s));
        NB_CUDA(cudaStreamSynchronize(s));
        const int ran = use_graph ? B->loops_host[0] : K;
        done_bodies += ran;
        *launches += (use_graph ? 1 : 0) + ran * per_body;
        int64_t live = 0;
        for (int q = 0; q < B->nprob; ++q) {
            run[q] = B->bs_host[q].done == 0 && B->act_run[q];
            if (run[q]) live += B->prob_e0_host[q + 1] - B->prob_e0_host[q];
        }
        if (live == 0 || done_bodies > (int64_t)maxit) break;
        if (4 * live < 3 * B->act_elems) {
            NB_TRY(set_active(B, run, s));
            K = 32;
        } else {
            K = std::min(2 * K, 512);
        }
    }
    return NB_OK;
}

// |b - A x|^2 and |b|^2 per listed problem into red[0..2 nprob); x may be
// NULL (x = 0).
static nb_status batch_residual(nb_batch *B, const double *b, const double *x, cudaStream_t s)
{
    const double *w = nullptr;
    if (x) {
        NB_TRY(bax_all<double>(B, false, x, B->w64, nullptr, nullptr, nullptr, nullptr, s));
        k_bgs<double><<<chunk_grid(B), 256, 0, s>>>(list_chunks(B), cnt_chunks(B), B->gs_off,
                                                    B->gs_loc, B->gs_mask, nullptr, B->w64);
        NB_CUDA(cudaGetLastError());
        w = B->w64;
    }
    k_bresid<<<elem_grid(B), 256, 0, s>>>(B->E, list_all(B), cnt_all(B), B->elem_l0, b, w,
                                          B->dinv64, B->r64, B->part_e);
    NB_CUDA(cudaGetLastError());
    k_bsum2<<<warp_grid(B->nprob), 256, 0, s>>>(B->nprob, B->prob_e0, B->part_e, B->E, B->red);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

static void free_bws(BatchWs &ws)
{
    if (ws.exec) cudaGraphExecDestroy(ws.exec);
    if (ws.graph) cudaGraphDestroy(ws.graph);
    cudaFree(ws.x);
    cudaFree(ws.r);
    cudaFree(ws.p);
    cudaFree(ws.w);
    ws = BatchWs();
}

}  // namespace nb

using namespace nb;

extern "C" nb_status nb_batch_destroy(nb_batch *B)
{
    if (!B) return NB_OK;
    ::nb::DeviceGuard nb_device_guard_(B->ctx->device);
    cudaStreamSynchronize(B->ctx->stream);
    for (nb_mesh *m : B->meshes) nb_mesh_destroy(m);
    free_bws(B->ws32);
    free_bws(B->ws64);
    void *bufs[] = {B->G32, B->G64, B->dinv32, B->dinv64, B->gs_off, B->gs_loc, B->gs_mask,
                    B->elem_prob, B->elem_l0, B->prob_e0, B->prob_dim, B->bs, B->loops,
                    B->part_e, B->red, B->r64, B->w64, B->act, B->kerr};
    for (void *b : bufs) cudaFree(b);
    if (B->bs_host) cudaFreeHost(B->bs_host);
    if (B->red_host) cudaFreeHost(B->red_host);
    if (B->act_host) cudaFreeHost(B->act_host);
    if (B->loops_host) cudaFreeHost(B->loops_host);
    nb_ctx *ctx = B->ctx;
    delete B;
    ctx_release(ctx);
    return NB_OK;
}

extern "C" nb_status nb_batch_create(nb_ctx *ctx, int nprob, const int *nx, const int *ny,
                                     const int *nz, const int *N, const double *deform,
                                     nb_batch **out)
{
    if (!ctx || !out || nprob < 1 || !nx || !ny || !nz || !N || !deform) {
        set_error("invalid argument: batch description");
        return NB_ERR_ARG;
    }
    *out = nullptr;
    NB_DEVICE_SCOPE(ctx->device);
    nb_batch *B = new nb_batch();
    B->ctx = ctx;
    ctx_retain(ctx);
    B->nprob = nprob;
    B->meshes.assign(nprob, nullptr);
    nb_status st = NB_OK;
    for (int p = 0; p < nprob && st == NB_OK; ++p) {
        st = nb_setup_mesh(ctx, nx[p], ny[p], nz[p], N[p], deform[p], &B->meshes[p]);
        if (st == NB_OK) st = nb_setup_gs(B->meshes[p]);
    }
    if (st != NB_OK) {
        nb_batch_destroy(B);
        return st;
    }
    // internal order: grouped by order, stable
    B->order.resize(nprob);
    std::iota(B->order.begin(), B->order.end(), 0);
    std::stable_sort(B->order.begin(), B->order.end(),
                     [&](int a, int b) { return N[a] < N[b]; });
    B->rank.resize(nprob);
    for (int q = 0; q < nprob; ++q) B->rank[B->order[q]] = q;
    B->l_off.assign(nprob, 0);
    B->g_off.assign(nprob, 0);
    int64_t gacc = 0;
    for (int p = 0; p < nprob; ++p) {
        B->g_off[p] = gacc;
        gacc += B->meshes[p]->nG;
    }
    B->nG = gacc;
    std::vector<int32_t> eprob;
    std::vector<int64_t> el0(1, 0);
    B->prob_e0_host.assign(1, 0);
    int64_t lacc = 0;
    for (int q = 0; q < nprob; ++q) {
        nb_mesh *m = B->meshes[B->order[q]];
        B->l_off[B->order[q]] = lacc;
        if (B->groups.empty() || B->groups.back().n != m->n) {
            BatchGroup g;
            g.n = m->n;
            g.e0 = g.e1 = (int64_t)eprob.size();
            g.l0 = lacc;
            B->groups.push_back(g);
        }
        B->prob_group.push_back((int)B->groups.size() - 1);
        for (int64_t e = 0; e < m->E; ++e) {
            eprob.push_back(q);
            el0.push_back(el0.back() + m->n3);
        }
        B->groups.back().e1 = (int64_t)eprob.size();
        B->prob_e0_host.push_back((int64_t)eprob.size());
        lacc += m->nL;
    }
    B->nL = lacc;
    B->E = (int64_t)eprob.size();
    if (B->nL >= ((int64_t)1 << 31)) {
        nb_batch_destroy(B);
        set_error("batch too large for 32-bit local indices");
        return NB_ERR_ARG;
    }
    // gather-scatter rows with batch local indices
    std::vector<int32_t> off(1, 0), loc;
    std::vector<uint8_t> rmask;
    B->prob_row0_host.assign(1, 0);
    for (int q = 0; q < nprob && st == NB_OK; ++q) {
        nb_mesh *m = B->meshes[B->order[q]];
        std::vector<int32_t> o(m->gs_rows + 1), l(std::max<int64_t>(m->gs_copies, 1));
        std::vector<uint8_t> mk(std::max<int64_t>(m->gs_rows, 1));
        st = nb_get_maps(m, nullptr, nullptr, nullptr, nullptr, o.data(), l.data(), mk.data());
        const int32_t base = (int32_t)B->l_off[B->order[q]];
        const int32_t obase = off.back();
        for (int64_t a = 0; a < m->gs_rows; ++a) {
            off.push_back(obase + o[a + 1]);
            rmask.push_back(mk[a]);
        }
        for (int64_t c = 0; c < m->gs_copies; ++c) loc.push_back(base + l[c]);
        B->prob_row0_host.push_back((int64_t)rmask.size());
        B->max_chunks += (m->gs_rows + kRowChunk - 1) / kRowChunk;
    }
    if (st != NB_OK) {
        nb_batch_destroy(B);
        return st;
    }
    B->rows = (int64_t)rmask.size();
    cudaStream_t s = ctx->stream;
    auto fail = [&](nb_status e) {
        nb_batch_destroy(B);
        return e;
    };
#define NB_BCUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            set_error("batch set-up: %s", cudaGetErrorString(e_));                             \
            return fail(e_ == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA);           \
        }                                                                                      \
    } while (0)
    NB_BCUDA(cudaMalloc(&B->G32, sizeof(float) * 6 * B->nL));
    NB_BCUDA(cudaMalloc(&B->G64, sizeof(double) * 6 * B->nL));
    NB_BCUDA(cudaMalloc(&B->dinv32, sizeof(float) * B->nL));
    NB_BCUDA(cudaMalloc(&B->dinv64, sizeof(double) * B->nL));
    NB_BCUDA(cudaMalloc(&B->gs_off, sizeof(int32_t) * off.size()));
    NB_BCUDA(cudaMalloc(&B->gs_loc, sizeof(int32_t) * std::max<size_t>(loc.size(), 1)));
    NB_BCUDA(cudaMalloc(&B->gs_mask, std::max<size_t>(rmask.size(), 1)));
    NB_BCUDA(cudaMalloc(&B->elem_prob, sizeof(int32_t) * B->E));
    NB_BCUDA(cudaMalloc(&B->elem_l0, sizeof(int64_t) * (B->E + 1)));
    NB_BCUDA(cudaMalloc(&B->prob_e0, sizeof(int64_t) * (nprob + 1)));
    NB_BCUDA(cudaMalloc(&B->prob_dim, sizeof(int4) * nprob));
    NB_BCUDA(cudaMalloc(&B->bs, sizeof(BScal) * nprob));
    NB_BCUDA(cudaMemset(B->bs, 0, sizeof(BScal) * nprob));
    NB_BCUDA(cudaMallocHost(&B->bs_host, sizeof(BScal) * nprob));
    NB_BCUDA(cudaMalloc(&B->loops, 2 * sizeof(int)));
    NB_BCUDA(cudaMallocHost(&B->loops_host, 2 * sizeof(int)));
    NB_BCUDA(cudaMalloc(&B->kerr, sizeof(int)));
    NB_BCUDA(cudaMemset(B->kerr, 0, sizeof(int)));
    for (BatchGroup &g : B->groups) g.variant = bax_tma_available_f32(g.n) ? 2 : 1;
    NB_BCUDA(cudaMalloc(&B->part_e, sizeof(double) * 2 * B->E));
    NB_BCUDA(cudaMalloc(&B->red, sizeof(double) * 4 * nprob));
    NB_BCUDA(cudaMallocHost(&B->red_host, sizeof(double) * 4 * nprob));
    {
        const int64_t nc = ((int64_t)B->groups.size() + 2 + 3) / 4 * 4;
        B->act_e_off = nc;
        B->act_all_off = nc + B->E;
        B->act_ch_off = (nc + 2 * B->E + 3) / 4 * 4;  // int4 chunks on a 16-byte boundary
        B->act_words = B->act_ch_off + 4 * std::max<int64_t>(B->max_chunks, 1);
        NB_BCUDA(cudaMalloc(&B->act, sizeof(int) * B->act_words));
        NB_BCUDA(cudaMallocHost(&B->act_host, sizeof(int) * B->act_words));
        NB_BCUDA(cudaMemset(B->act, 0, sizeof(int) * B->act_words));
    }
    NB_BCUDA(cudaMalloc(&B->r64, sizeof(double) * B->nL));
    NB_BCUDA(cudaMalloc(&B->w64, sizeof(double) * B->nL));
    NB_BCUDA(cudaMemset(B->w64, 0, sizeof(double) * B->nL));
    for (int q = 0; q < nprob; ++q) {
        nb_mesh *m = B->meshes[B->order[q]];
        const size_t lo = (size_t)B->l_off[B->order[q]];
        NB_BCUDA(cudaMemcpyAsync(B->G32 + 6 * lo, m->G32, sizeof(float) * 6 * m->nL,
                                 cudaMemcpyDeviceToDevice, s));
        NB_BCUDA(cudaMemcpyAsync(B->G64 + 6 * lo, m->G64, sizeof(double) * 6 * m->nL,
                                 cudaMemcpyDeviceToDevice, s));
        NB_BCUDA(cudaMemcpyAsync(B->dinv32 + lo, m->dinv32, sizeof(float) * m->nL,
                                 cudaMemcpyDeviceToDevice, s));
        NB_BCUDA(cudaMemcpyAsync(B->dinv64 + lo, m->dinv64, sizeof(double) * m->nL,
                                 cudaMemcpyDeviceToDevice, s));
    }
    NB_BCUDA(cudaMemcpyAsync(B->gs_off, off.data(), sizeof(int32_t) * off.size(),
                             cudaMemcpyHostToDevice, s));
    if (!loc.empty())
        NB_BCUDA(cudaMemcpyAsync(B->gs_loc, loc.data(), sizeof(int32_t) * loc.size(),
                                 cudaMemcpyHostToDevice, s));
    if (!rmask.empty())
        NB_BCUDA(cudaMemcpyAsync(B->gs_mask, rmask.data(), rmask.size(), cudaMemcpyHostToDevice, s));
    NB_BCUDA(cudaMemcpyAsync(B->elem_prob, eprob.data(), sizeof(int32_t) * B->E,
                             cudaMemcpyHostToDevice, s));
    NB_BCUDA(cudaMemcpyAsync(B->elem_l0, el0.data(), sizeof(int64_t) * (B->E + 1),
                             cudaMemcpyHostToDevice, s));
    NB_BCUDA(cudaMemcpyAsync(B->prob_e0, B->prob_e0_host.data(), sizeof(int64_t) * (nprob + 1),
                             cudaMemcpyHostToDevice, s));
    std::vector<int4> dims(nprob);
    for (int q = 0; q < nprob; ++q) {
        const nb_mesh *m = B->meshes[B->order[q]];
        dims[q] = make_int4(m->nx, m->ny, m->nz, m->n);
    }
    NB_BCUDA(cudaMemcpyAsync(B->prob_dim, dims.data(), sizeof(int4) * nprob,
                             cudaMemcpyHostToDevice, s));
    NB_BCUDA(cudaStreamSynchronize(s));
#undef NB_BCUDA
    *out = B;
    return NB_OK;
}

extern "C" nb_status nb_batch_layout(const nb_batch *B, int64_t *l_off, int64_t *g_off,
                                     int64_t totals[2])
{
    if (!B) {
        set_error("invalid argument: batch is NULL");
        return NB_ERR_ARG;
    }
    for (int p = 0; p < B->nprob; ++p) {
        if (l_off) l_off[p] = B->l_off[p];
        if (g_off) g_off[p] = B->g_off[p];
    }
    if (totals) {
        totals[0] = B->nL;
        totals[1] = B->nG;
    }
    return NB_OK;
}

extern "C" nb_mesh *nb_batch_mesh(nb_batch *B, int p)
{
    if (!B || p < 0 || p >= B->nprob) return nullptr;
    return B->meshes[p];
}

extern "C" nb_status nb_batch_to_local(nb_batch *B, const double *ug, double *uL)
{
    if (!B || !ug || !uL) {
        set_error("invalid argument: NULL batch or vector");
        return NB_ERR_ARG;
    }
    NB_DEVICE_SCOPE(B->ctx->device);
    for (int p = 0; p < B->nprob; ++p)
        NB_TRY(to_local(B->meshes[p], NB_FP64, ug + B->g_off[p], uL + B->l_off[p], 1,
                        B->ctx->stream));
    NB_CUDA(cudaStreamSynchronize(B->ctx->stream));
    return NB_OK;
}

extern "C" nb_status nb_batch_autotune(nb_batch *B, int reps, void *flush, size_t flush_bytes)
{
    if (!B || reps < 1) {
        set_error("invalid argument: batch or reps");
        return NB_ERR_ARG;
    }
    NB_DEVICE_SCOPE(B->ctx->device);
    cudaStream_t s = B->ctx->stream;
    NB_TRY(ensure_bws(B, B->ws32, sizeof(float)));
    NB_TRY(set_active(B, std::vector<char>(B->nprob, 1), s));
    // every problem running with beta = 0: the step the solver launches
    NB_CUDA(cudaMemsetAsync(B->bs, 0, sizeof(BScal) * B->nprob, s));
    cudaEvent_t e0, e1;
    NB_CUDA(cudaEventCreate(&e0));
    NB_CUDA(cudaEventCreate(&e1));
    for (int gi = 0; gi < (int)B->groups.size(); ++gi) {
        BatchGroup &g = B->groups[gi];
        double best = 1e300;
        int bestv = g.variant;
        const int nv = bax_tma_available_f32(g.n) ? 3 : 2;
        for (int v = 0; v < nv; ++v) {
            double tot = 0.0;
            for (int r = 0; r <= reps; ++r) {  // the first launch is a warm-up
                if (flush && flush_bytes) NB_TRY(l2_flush(B->ctx, flush, flush_bytes, r, s));
                cudaEventRecord(e0, s);
                NB_TRY(bax_group<float>(B, gi, v, true, nullptr, (float *)B->ws32.w,
                                        (const float *)B->ws32.r, B->dinv32, (float *)B->ws32.p,
                                        B->part_e, s));
                cudaEventRecord(e1, s);
                NB_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) tot += ms;
            }
            if (tot < best) {
                best = tot;
                bestv = v;
            }
        }
        g.variant = bestv;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // graphs captured with the old choice are rebuilt on the next solve
    free_bws(B->ws32);
    return NB_OK;
}

extern "C" nb_status nb_batch_solve(nb_batch *B, const nb_opts *o, const double *b, double *x,
                                    nb_stats *stats, nb_stats *total)
{
    if (!B || !o || !b || !x) {
        set_error("invalid argument: NULL batch, options or vector");
        return NB_ERR_ARG;
    }
    if (o->prec != NB_FP64 && o->prec != NB_FP32) {
        set_error("batched solves support NB_FP64 and NB_FP32");
        return NB_ERR_ARG;
    }
    if (o->pc != NB_PC_JACOBI && o->pc != NB_PC_NONE) {
        set_error("batched solves support the Jacobi and identity preconditioners");
        return NB_ERR_ARG;
    }
    if (o->pc == NB_PC_NONE) {
        set_error("batched solves use the Jacobi preconditioner");
        return NB_ERR_ARG;
    }
    if (!(o->rtol > 0.0 && o->rtol < 1.0) || o->maxiter < 0 || o->max_outer < 0) {
        set_error("invalid argument: rtol, maxiter or max_outer");
        return NB_ERR_ARG;
    }
    NB_DEVICE_SCOPE(B->ctx->device);
    cudaStream_t s = B->ctx->stream;
    const int np = B->nprob;
    cudaEvent_t t0, t1;
    NB_CUDA(cudaEventCreate(&t0));
    NB_CUDA(cudaEventCreate(&t1));
    NB_CUDA(cudaEventRecord(t0, s));
    std::vector<int> iters(np, 0), outer_p(np, 0), status(np, NB_NOT_CONVERGED);
    std::vector<double> rel(np, INFINITY);
    int batched_iters = 0, outer = 0;
    int64_t launches = 0;
    const int ngroups = (int)B->groups.size();
    const std::vector<char> all(np, 1);
    if (o->prec == NB_FP64) {
        // plain FP64 PCG of every problem, in place on x
        NB_TRY(ensure_bws(B, B->ws64, sizeof(double)));
        NB_TRY(set_active(B, all, s));
        NB_TRY(batch_residual(B, b, o->use_x0 ? x : nullptr, s));
        launches += 2 + (o->use_x0 ? ngroups + 1 : 0);
        if (o->use_x0) {
            k_bcopy<<<B->ctx->sm_count * 4, 256, 0, s>>>(B->nL, x, (double *)B->ws64.x);
            ++launches;
        } else {
            NB_CUDA(cudaMemsetAsync(B->ws64.x, 0, sizeof(double) * B->nL, s));
        }
        k_bcopy<<<B->ctx->sm_count * 4, 256, 0, s>>>(B->nL, B->r64, (double *)B->ws64.r);
        NB_CUDA(cudaGetLastError());
        ++launches;
        // tolerance relative to |b| (red[nprob + p] from the residual pass)
        NB_TRY(batch_cg<double>(B, B->ws64, B->dinv64, o->rtol, o->maxiter, 0, o->use_graph, 0,
                                B->red + np, s, &launches));
        NB_CUDA(cudaMemcpyAsync(B->bs_host, B->bs, sizeof(BScal) * np, cudaMemcpyDeviceToHost, s));
        k_bcopy<<<B->ctx->sm_count * 4, 256, 0, s>>>(B->nL, (double *)B->ws64.x, x);
        NB_TRY(set_active(B, all, s));  // the final residual of every problem
        NB_TRY(batch_residual(B, b, x, s));
        launches += 1 + ngroups + 3;
        NB_CUDA(cudaMemcpyAsync(B->red_host, B->red, sizeof(double) * 2 * np,
                                cudaMemcpyDeviceToHost, s));
        NB_CUDA(cudaStreamSynchronize(s));
        for (int q = 0; q < np; ++q) {
            const int p = B->order[q];
            iters[p] = B->bs_host[q].iter;
            batched_iters = std::max(batched_iters, iters[p]);
            const double bn = B->red_host[np + q];
            rel[p] = bn > 0.0 ? sqrt(B->red_host[q] / bn) : 0.0;
            status[p] = B->bs_host[q].status;
            if (status[p] == 0 && !(rel[p] < o->rtol * 1.5)) status[p] = NB_NOT_CONVERGED;
        }
    } else {
        NB_TRY(ensure_bws(B, B->ws32, sizeof(float)));
        if (!o->use_x0) NB_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * B->nL, s));
        std::vector<double> bn2(np, 0.0), prev(np, INFINITY);
        std::vector<int> stagn(np, 0);
        std::vector<char> running(np, 1);
        int used = 0;
        std::vector<char> run_q(np, 1);  // running problems, internal order
        for (outer = 0; outer <= o->max_outer; ++outer) {
            for (int q = 0; q < np; ++q) run_q[q] = running[B->order[q]];
            NB_TRY(set_active(B, run_q, s));
            NB_TRY(batch_residual(B, b, (outer == 0 && !o->use_x0) ? nullptr : x, s));
            NB_CUDA(cudaMemcpyAsync(B->red_host, B->red, sizeof(double) * 2 * np,
                                    cudaMemcpyDeviceToHost, s));
            NB_CUDA(cudaStreamSynchronize(s));
            launches += 2 + ((outer == 0 && !o->use_x0) ? 0 : ngroups + 1);
            bool any = false;
            for (int q = 0; q < np; ++q) {
                const int p = B->order[q];
                if (!running[p]) {
                    B->red_host[3 * np + q] = 0.0;
                    continue;
                }
                if (outer == 0) bn2[p] = B->red_host[np + q];
                if (!isfinite(bn2[p])) {
                    set_error("right-hand side of problem %d has a non-finite entry", p);
                    return NB_ERR_ARG;
                }
                rel[p] = bn2[p] > 0.0 ? sqrt(B->red_host[q] / bn2[p]) : 0.0;
                outer_p[p] = outer;
                bool stop = false;
                if (!isfinite(rel[p])) {
                    status[p] = NB_BREAKDOWN;
                    stop = true;
                } else if (rel[p] < o->rtol) {
                    status[p] = NB_OK;
                    stop = true;
                } else if (outer == o->max_outer || used >= o->maxiter) {
                    status[p] = NB_NOT_CONVERGED;
                    stop = true;
                } else if (rel[p] > 0.5 * prev[p] && ++stagn[p] >= 3) {
                    status[p] = NB_STAGNATED;
                    stop = true;
                }
                if (!(rel[p] > 0.5 * prev[p])) stagn[p] = 0;
                prev[p] = rel[p];
                running[p] = !stop;
                B->red_host[3 * np + q] = stop ? 0.0 : 1.0;
                B->red_host[2 * np + q] =
                    std::min(0.5, std::max(o->inner_rtol, 0.5 * o->rtol / std::max(rel[p], 1e-300)));
                any |= !stop;
            }
            if (!any) break;
            for (int q = 0; q < np; ++q) run_q[q] = running[B->order[q]];
            NB_TRY(set_active(B, run_q, s));
            NB_CUDA(cudaMemcpyAsync(B->red + 2 * np, B->red_host + 2 * np, sizeof(double) * 2 * np,
                                    cudaMemcpyHostToDevice, s));
            k_bdemote<<<elem_grid(B), 256, 0, s>>>(B->E, list_all(B), cnt_all(B), B->elem_l0,
                                                    B->elem_prob, np, B->red, B->r64,
                                                    (float *)B->ws32.r, (float *)B->ws32.x);
            NB_CUDA(cudaGetLastError());
            NB_TRY(batch_cg<float>(B, B->ws32, B->dinv32, 0.0, o->maxiter - used, 1, o->use_graph,
                                   1, nullptr, s, &launches));
            NB_TRY(set_active(B, run_q, s));  // every problem of this step is promoted
            k_bpromote<<<elem_grid(B), 256, 0, s>>>(B->E, list_all(B), cnt_all(B), B->elem_l0,
                                                     B->elem_prob, np, B->red,
                                                     (const float *)B->ws32.x, x);
            NB_CUDA(cudaGetLastError());
            NB_CUDA(cudaMemcpyAsync(B->bs_host, B->bs, sizeof(BScal) * np, cudaMemcpyDeviceToHost, s));
            NB_CUDA(cudaStreamSynchronize(s));
            int most = 0;
            for (int q = 0; q < np; ++q) {
                iters[B->order[q]] += B->bs_host[q].iter;
                most = std::max(most, B->bs_host[q].iter);
            }
            used += most;
            batched_iters += most;
            launches += 2;  // demote and promote
        }
    }
    NB_CUDA(cudaEventRecord(t1, s));
    NB_CUDA(cudaEventSynchronize(t1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    int kerr = 0;
    NB_CUDA(cudaMemcpy(&kerr, B->kerr, sizeof(int), cudaMemcpyDeviceToHost));
    if (kerr) {
        cudaMemset(B->kerr, 0, sizeof(int));
        set_error("a bulk copy of the batched operator did not complete within one second");
        return NB_ERR_CUDA;
    }
    nb_status worst = NB_OK;
    double worst_rel = 0.0;
    for (int p = 0; p < np; ++p) {
        if (stats) {
            stats[p].iters = iters[p];
            stats[p].outer_iters = outer_p[p];
            stats[p].rel_res = rel[p];
            stats[p].seconds = ms * 1e-3;
            stats[p].status = (nb_status)status[p];
            stats[p].history_len = 0;
            stats[p].launches = 0;
        }
        if (status[p] > worst) worst = (nb_status)status[p];
        worst_rel = std::max(worst_rel, rel[p]);
    }
    if (total) {
        total->iters = batched_iters;
        total->outer_iters = outer;
        total->rel_res = worst_rel;
        total->seconds = ms * 1e-3;
        total->status = worst;
        total->history_len = 0;
        total->launches = launches;
    }
    return worst;
}
