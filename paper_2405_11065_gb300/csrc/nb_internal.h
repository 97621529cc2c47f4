// Internal declarations shared by the translation units of the library.
// Not part of the public C ABI (include/nekbone_gb300.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/nekbone_gb300.h"

namespace nb {

constexpr int kMaxN = 15;          // highest polynomial order supported
constexpr int kMaxn = kMaxN + 1;   // GLL points per direction
constexpr int kFinalizeThreads = 512;
constexpr int kMaxPartials = 1 << 16;
constexpr int kMaxDevices = 64;    // devices with their own launch-shape caches

// The entry of a per-device cache for the calling thread's current device
// (a scratch entry, never kept, beyond kMaxDevices).  Launch shapes that
// depend on occupancy, and the shared-memory attribute set with them, are
// per device.
inline int &device_slot(int (&slots)[kMaxDevices])
{
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) {
        static thread_local int spare;
        spare = 0;
        return spare;
    }
    return slots[d];
}

// Makes `device` current for the lifetime of the guard and restores the
// caller's current device afterwards, so that a library call leaves the
// calling thread's device as it found it.
class DeviceGuard {
  public:
    explicit DeviceGuard(int device)
    {
        if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
        if (prev_ != device) err_ = cudaSetDevice(device);
        else prev_ = -1;  // nothing to restore
    }
    ~DeviceGuard()
    {
        if (prev_ >= 0 && err_ == cudaSuccess) cudaSetDevice(prev_);
    }
    cudaError_t error() const { return err_; }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;

  private:
    int prev_ = -1;
    cudaError_t err_ = cudaSuccess;
};

void set_error(const char *fmt, ...);

#define NB_CUDA(call)                                                               \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            ::nb::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,              \
                            cudaGetErrorString(e_));                                \
            return e_ == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA;      \
        }                                                                           \
    } while (0)

// Enter `device` for the rest of the enclosing scope (see DeviceGuard).
#define NB_DEVICE_SCOPE(device)                   \
    ::nb::DeviceGuard nb_device_guard_(device);   \
    NB_CUDA(nb_device_guard_.error())

#define NB_TRY(expr)                     \
    do {                                 \
        nb_status s_ = (expr);           \
        if (s_ < 0) return s_;           \
    } while (0)

// Programmatic dependent launch.  Inside a PdlScope the CG loops launch
// their kernels that support it with the programmatic-serialization
// attribute: such a kernel may start while the previous kernel of the stream
// finishes (its last block's reductions, the launch latency) and runs its
// independent prologue -- barrier set-up, bulk copies of constant data,
// tensor-memory allocation -- before it waits (griddepcontrol.wait, pdl_wait)
// for the previous kernel's completion.  Only kernels that wait before their
// first dependent read are launched through launch_pdl.
extern thread_local bool g_pdl;

class PdlScope {
  public:
    explicit PdlScope(bool on) : prev_(g_pdl) { g_pdl = on; }
    ~PdlScope() { g_pdl = prev_; }
    PdlScope(const PdlScope &) = delete;
    PdlScope &operator=(const PdlScope &) = delete;

  private:
    bool prev_;
};

// Whether the CG loop's kernels should let their successor launch as soon as
// their main work is done, rather than as their blocks exit.  Measured: the
// early start hides the last block's scalar step where blocks have few
// elements (E = 4096, N = 9: 62.5 against 63.5 ms per solve); on larger meshes
// the successor's early blocks take SM slots from the persistent grids of the
// previous kernel's last wave (E = 32768, N = 7: 376 against 297 ms).
inline int pdl_early_for(int64_t E, int sm_count) { return E <= 32 * (int64_t)sm_count ? 1 : 0; }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = g_pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Division by a divisor fixed at launch time (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994): for
// 0 <= x < 2^31, x / d = (umulhi(x, m) + x) >> l with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1.
struct FastDiv {
    uint32_t m = 1, l = 0, d = 1;
    FastDiv() = default;
    explicit FastDiv(uint32_t div) : d(div)
    {
        while ((1ull << l) < div) ++l;
        m = (uint32_t)(((1ull << 32) * ((1ull << l) - div)) / div + 1);
    }
#ifdef __CUDACC__
    __device__ __forceinline__ int div(int x) const
    {
        return (int)((__umulhi((uint32_t)x, m) + (uint32_t)x) >> l);
    }
#endif
};

// Device-resident scalars of one CG solve.  Every kernel of the iteration
// reads alpha/beta from here, so a captured graph needs no host values.
struct CgScalars {
    double rtz;       // (r, c, z) of the current iteration
    double rtz_old;   // of the previous iteration
    double pap;       // (w, c, p)
    double rtr;       // (r, c, r)
    double alpha, beta;
    double bnorm2;    // (b, c, b) of the system being solved
    double relres;    // sqrt(rtr / bnorm2)
    double tol;       // relative tolerance
    double fcg_zw;    // flexible CG: (z, c, w_prev)
    double pap_prev;  // flexible CG: previous (p, c, A p)
    double rp;        // flexible CG: (r, c, p)
    double alpha_x;   // alpha of the iteration whose x step is deferred
    int x_pending;    // 1: x still lacks alpha_x times the other direction buffer
    int iter;         // iterations done
    int maxit;        // iteration limit
    int done;         // 1 when the loop must stop
    int status;       // 0 running/converged, NB_NOT_CONVERGED, NB_BREAKDOWN
    int hist_cap;     // capacity of hist
    int loops;        // executions of the graph's loop body (hard stop at maxit + 1)
    int pdl_early;    // 1: the loop's kernels let the next one launch after their main
                      // work (programmatic dependent launch; small meshes, see pdl_early_for)
    double *hist;     // device history (relres per iteration) or nullptr
    unsigned int tick_ax;   // blocks of the operator kernel done (last block finalises)
    unsigned int tick_upd;  // blocks of the update kernel done
};

// Per-problem scalars of a batched CG solve (one entry per problem, in the
// batch's internal order).
struct BScal {
    double rtz, rtz_old, pap, rtr, alpha, beta, bnorm2, relres, tol;
    int iter, maxit, done, status;
};

// A preallocated set of vectors for one solve precision.
struct Workspace {
    size_t nL = 0;
    int elt = 0;                  // bytes per value (4 or 8)
    void *x = nullptr, *r = nullptr, *p = nullptr, *w = nullptr, *z = nullptr;
    void *aux = nullptr;          // flexible CG: previous A p
    void *p2 = nullptr;           // Jacobi CG with deferred x steps: the second direction
    double *part = nullptr;       // per-block partial sums (kMaxPartials * 3)
    CgScalars *scal = nullptr;    // device scalars
    CgScalars *scal_host = nullptr;  // pinned mirror
    double *hist = nullptr;       // device history buffer
    int hist_cap = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_key = -1;           // which configuration the graph holds
    int graph_epoch = -1;         // the mesh's ax_epoch at its capture
    cudaGraph_t graph2 = nullptr;       // flexible-CG iteration graph
    cudaGraphExec_t exec2 = nullptr;
    intptr_t graph2_key = 0;            // the model it was captured with
    int graph2_epoch = -1;              // the mesh's ax_epoch at its capture
};

// Launch shape of the ax kernel for one (precision, order).
struct AxConfig {
    int variant = -1;          // kernel variant id chosen by the autotuner (-1: default)
    int grid = 0;              // blocks (persistent grid)
    int threads = 0;
};

}  // namespace nb

struct nb_ctx {
    int device = 0;
    int sm_count = 0;
    int l2_bytes = 0;  // L2 cache size
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    // references: the caller's (dropped by nb_destroy) and one per mesh,
    // batch and model built on the context, so that those can be destroyed
    // after the context (in any order, e.g. by a garbage collector)
    std::atomic<int> refs{1};
};

namespace nb {
void ctx_retain(nb_ctx *c);
void ctx_release(nb_ctx *c);
}  // namespace nb

struct nb_mesh {
    nb_ctx *ctx = nullptr;
    int nx = 0, ny = 0, nz = 0, N = 0, n = 0, n3 = 0;
    double deform = 0.0;
    // z-slab of a larger box (nb_setup_slab): elements ez + z_off of a box of
    // nz_glob elements along z; an interface plane below / above (shared with
    // the neighbouring slab, not Dirichlet; the copies of the lower one are
    // not owners).  A whole box: z_off = 0, nz_glob = nz, no interfaces.
    int z_off = 0, nz_glob = 0;
    bool iface_lo = false, iface_hi = false;
    double *diag_asm = nullptr;  // [nL] slab-local assembled diagonal (slabs only)
    nb::CgScalars *scal_split = nullptr;  // scalars of the split-phase CG calls
    int64_t E = 0, nL = 0, nG = 0;
    bool gs_ready = false;
    // geometry
    double *D64 = nullptr;     // n*n, D[i][l] = l_l'(xi_i)
    float *D32 = nullptr;
    double *G64 = nullptr;     // [E][6][n3]
    float *G32 = nullptr;
    // numbering and gather-scatter
    int32_t *gid = nullptr;    // [nL]
    int64_t gs_rows = 0, gs_copies = 0;
    int32_t *gs_off = nullptr;   // [rows+1]
    int32_t *gs_loc = nullptr;   // [copies]
    int32_t *gs_gid = nullptr;   // [rows]
    uint8_t *gs_mask = nullptr;  // [rows]
    int32_t *g_first = nullptr;  // [nG] first local copy of each global node
    // the same rows split by kind, for the masked summation of the solver:
    // copies of Dirichlet nodes (set to zero, nothing read), and free shared
    // nodes with 2, 4 or 8 copies (ascending local indices, one vector load)
    int32_t *gs_zero = nullptr;  // [n_zero]
    int2 *gs_pair = nullptr;     // [n_pair]
    int4 *gs_quad = nullptr;     // [n_quad]
    int4 *gs_oct = nullptr;      // [2 n_oct]
    int64_t n_zero = 0, n_pair = 0, n_quad = 0, n_oct = 0;
    uint8_t *mask_g = nullptr;   // [nG]
    // weights and preconditioner
    float *c32 = nullptr;      // [nL] 1/multiplicity (exact in float)
    double *dinv64 = nullptr;  // [nL]
    float *dinv32 = nullptr;
    double *ones64 = nullptr;  // [nL] identity preconditioner (mask)
    float *ones32 = nullptr;
    // host copies of the small maps
    std::vector<int32_t> mult_host;  // [nG]
    std::vector<uint8_t> mask_host;  // [nG]
    // solve workspaces
    nb::Workspace ws64, ws32;
    double *r64 = nullptr, *w64 = nullptr, *x64 = nullptr, *b64 = nullptr, *g64 = nullptr;
    double *part64 = nullptr;
    double *red_out = nullptr;       // device scalar for glsc3/norms
    double *red_host = nullptr;      // pinned mirror
    nb::AxConfig ax_cfg[4];
    int update_kind = 0;       // FP32 update with the folded summation, even n:
                               // 1 element ranges (k_cg_update_el), 2 node pairs
                               // (k_cg_update_pairs), 3 element ranges with
                               // bulk-copied vectors (k_cg_update_tma), 0 element
                               // ranges where an element takes at most two rounds
                               // of 256 pairs, else node pairs (measured fastest)
    int x_defer = -1;          // deferred x steps: -1 by size, 0 never, 1 where possible
    int ax_epoch = 0;          // bumped whenever an operator variant choice changes:
                               // captured iteration graphs of an older epoch are stale
    int *kerr = nullptr;             // device flag: a pipelined kernel's wait timed out
    int64_t launches = 0;            // kernels issued by the current solve
    // learned preconditioner (optional)
    void *learned = nullptr;
    // Schwarz preconditioner data (built on first use)
    void *schwarz = nullptr;
};

namespace nb {

// ---- setup (nb_setup.cu)
nb_status gll_host(int N, double *xi, double *w);
void deriv_host(int N, const double *xi, double *D);
nb_status build_geometry(nb_mesh *m);
nb_status build_gs(nb_mesh *m);
nb_status slab_free(nb_mesh *m);

// ---- operator (nb_ax.cu)
nb_status upload_deriv_tables(int n, const double *D64);
// w = A_L u on all elements; if pap_part != nullptr also per-block partials
// of sum(u*w) (FP64); pupd: if non-null, u is first formed as
// u = dinv*r + beta*u_old (CG direction update, see ax_cg_step).
nb_status ax_local(nb_mesh *m, nb_prec prec, const void *u, void *w, double *pap_part,
                   int *nparts, cudaStream_t s);
nb_status ax_cg_step(nb_mesh *m, nb_prec prec, const void *r, const void *dinv, void *p,
                     void *w, CgScalars *scal, double *pap_part, int *nparts,
                     cudaStream_t s);
// The same step in FP32 with the previous direction read from p_prev and the
// new one written to p (two buffers that the iteration alternates); only
// where the pencil operator is the FP32 variant in use.
bool ax_cg_step_from_available(const nb_mesh *m);
nb_status ax_cg_step_from(nb_mesh *m, const float *r, const float *dinv, const float *p_prev,
                          float *p, float *w, CgScalars *scal, double *pap_part, int *nparts,
                          cudaStream_t s);
int ax_variant_count(const nb_mesh *m, nb_prec prec);
nb_status l2_flush(const nb_ctx *ctx, void *buf, size_t bytes, int pattern, cudaStream_t s);
// ---- slabs and the split-phase CG (nb_slab.cu, nb_solve.cu)
nb_status slab_face(nb_mesh *m, nb_prec prec, int side, const void *u, void *face, cudaStream_t s);
nb_status slab_face_add(nb_mesh *m, nb_prec prec, int side, void *u, const void *face,
                        cudaStream_t s);
nb_status slab_diag_face(nb_mesh *m, int side, double *face, cudaStream_t s);
nb_status slab_finish_diag(nb_mesh *m, const double *face_lo, const double *face_hi,
                           cudaStream_t s);
nb_status split_step(nb_mesh *m, nb_prec prec, double beta, const void *r, void *p, void *w,
                     double *pap, cudaStream_t s);
nb_status split_update(nb_mesh *m, nb_prec prec, double alpha, void *x, void *r, const void *p,
                       const void *w, double out[2], cudaStream_t s);
nb_status split_dots(nb_mesh *m, nb_prec prec, const void *r, double out[2], cudaStream_t s);
const char *ax_variant_name(const nb_mesh *m, nb_prec prec, int v);
int ax_variant_in_use(const nb_mesh *m, nb_prec prec);

// ---- gather-scatter and vectors (nb_vec.cu)
nb_status dssum(nb_mesh *m, nb_prec prec, void *u, int masked, cudaStream_t s);
nb_status gs_rows_launch(const nb_ctx *ctx, int64_t rows, const int32_t *off, const int32_t *loc,
                         const uint8_t *rmask, nb_prec prec, void *u, int masked, cudaStream_t s);
nb_status to_local(nb_mesh *m, nb_prec prec, const void *ug, void *uL, int masked,
                   cudaStream_t s);
nb_status to_global(nb_mesh *m, nb_prec prec, const void *uL, void *ug, cudaStream_t s);
nb_status glsc3_dev(nb_mesh *m, nb_prec prec, const void *a, const void *b, double *part,
                    double *out_dev, cudaStream_t s);
nb_status sum_partials_dev(const double *part, int cnt, double *out_dev, cudaStream_t s);
nb_status local_diag(nb_mesh *m, double *diag, cudaStream_t s);
nb_status finish_jacobi(nb_mesh *m, double *diag, cudaStream_t s);

// ---- solvers (nb_solve.cu)
nb_status ensure_ws(nb_mesh *m, Workspace &ws, int elt, int hist_cap);
nb_status solve(nb_mesh *m, const nb_opts *o, const double *b, double *x, nb_stats *st);

}  // namespace nb
