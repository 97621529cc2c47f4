/*
 * nekbone_gb300.h -- C ABI of the GB300 (sm_103a) spectral-element Poisson
 * conjugate-gradient library.
 *
 * The method is the conjugate-gradient (CG) solve of the Nekbone mini-app as
 * profiled in the mixed-precision case study (Section 4.1, Table 1): each
 * iteration applies the preconditioner (solveM), three weighted dot products
 * (glsc3), two kinds of vector updates (add2s1, add2s2) and the matrix-free
 * spectral-element operator ax, whose "accumulations before and after"
 * (Table 1, note b) are the direct-stiffness summation over shared nodes.
 * Section 6 of the paper runs that loop in single precision with the set-up
 * kept in double; this library adds FP64 iterative refinement around an FP32
 * (or tensor-core) inner solve.
 *
 * Conventions for every function below:
 *  - Return value: NB_OK (0) on success; a negative nb_status on an error (no
 *    output is valid); a positive nb_status is a solver outcome with a valid
 *    solution (not converged, stagnated, breakdown, fell back).
 *    nb_last_error() returns a message for the last error of the calling
 *    thread.
 *  - "_dev" pointers are CUDA device pointers on the context's device; "_host"
 *    pointers are ordinary host memory.  The caller owns every buffer it
 *    passes and must keep it alive until the call returns (device work is
 *    complete when a call returns unless stated otherwise).  The library owns
 *    what it allocates and frees it in the matching *_destroy call.
 *  - All work is issued on the context's stream (set at nb_create or with
 *    nb_set_stream).  Functions synchronise that stream before returning.
 *  - Vector layout: an "L-vector" holds E*(N+1)^3 values, element-major,
 *    [e][k][j][i] with i fastest; a "G-vector" holds one value per unique
 *    (global) node, index gx + (nx*N+1)*(gy + (ny*N+1)*gz).
 *  - Element e of an nx*ny*nz box is (ex, ey, ez) with e = ex + nx*(ey + ny*ez).
 *  - The precision argument selects the value type of vector arguments:
 *    NB_FP64 -> double; NB_FP32, NB_TC_F16, NB_TC_BF16 -> float.
 *  - The library validates sizes and pointers on the host, never aborts and
 *    bounds every device loop by an iteration limit.
 */
#ifndef NEKBONE_GB300_H
#define NEKBONE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nb_ctx nb_ctx;   /* device, stream, error state */
typedef struct nb_mesh nb_mesh; /* device geometry, numbering, gather-scatter, workspaces */

typedef enum {
    NB_OK = 0,
    NB_ERR_ARG = -1,        /* invalid argument (size, pointer, enum, NaN input) */
    NB_ERR_CUDA = -2,       /* a CUDA runtime call failed */
    NB_ERR_OOM = -3,        /* device allocation failed */
    NB_ERR_MESH = -4,       /* invalid mesh: non-positive Jacobian, bad order */
    NB_ERR_STATE = -5,      /* call out of order (e.g. solve before setup_gs) */
    NB_NOT_CONVERGED = 1,   /* iteration limit reached; x holds the last iterate */
    NB_STAGNATED = 2,       /* refinement stopped reducing the residual */
    NB_BREAKDOWN = 3,       /* p^T A p <= 0 or a non-finite scalar */
    NB_FELL_BACK = 4        /* learned preconditioner abandoned for Jacobi */
} nb_status;

typedef enum {
    NB_FP64 = 0,      /* operator and vectors in double */
    NB_FP32 = 1,      /* operator and vectors in float, dots accumulated in double */
    NB_TC_F16 = 2,    /* float vectors, derivative contractions on FP16 tensor cores */
    NB_TC_BF16 = 3    /* float vectors, derivative contractions on BF16 tensor cores */
} nb_prec;

typedef enum {
    NB_PC_NONE = 0,    /* solveM is a copy (the paper's no-multigrid case) */
    NB_PC_JACOBI = 1,  /* z = diag(A)^-1 r */
    NB_PC_LEARNED = 2, /* per-element network inside flexible CG */
    NB_PC_SCHWARZ = 3, /* overlapping Schwarz, fast-diagonalisation local solves
                          (the smoother of Nekbone's multigrid solveM); FP32
                          refinement steps, even n, orders N <= 11 */
    NB_PC_SCHWARZ2 = 4 /* the same plus the coarse-grid level (two-level
                          additive Schwarz, trilinear coarse space on the
                          element vertices); at most 65 elements per direction
                          and 24576 interior vertices */
} nb_pc;

typedef struct {
    nb_prec prec;       /* NB_FP64: plain FP64 PCG.  Others: FP64 iterative
                           refinement around an inner solve in that precision */
    nb_pc pc;           /* preconditioner */
    double rtol;        /* stop when ||b - A x||_c / ||b||_c < rtol (FP64) */
    int maxiter;        /* iteration limit (inner iterations summed) */
    double inner_rtol;  /* relative tolerance of each inner solve (refinement) */
    int max_outer;      /* refinement step limit */
    int use_graph;      /* 1: the iteration is a CUDA graph with a device-side
                           while loop; 0: host-launched kernels */
    int record_history; /* 1: keep the recursive residual of each iteration */
    int use_x0;         /* 1: x_dev holds the initial guess; 0: start from zero */
    int restart;        /* refinement: 1 restarts
                           each inner CG from p = 0 (classic iterative refinement,
                           each inner solve to inner_rtol); 0 (default) keeps the
                           search direction across the FP64 residual replacement
                           (reliable update), replacing the residual each time it
                           has dropped by max(inner_rtol, 1e-2), as long as the
                           inner solves stay below 1000 iterations and resumed
                           ones converge (else it falls back to restarts).  The
                           same holds for the flexible CG of the learned (fused
                           form) and Schwarz preconditioners, except that with
                           the Schwarz preconditioners an inner solve that follows
                           one of fewer than 15 iterations closes inner_rtol
                           itself; the batch always restarts. */
} nb_opts;

typedef struct {
    int iters;              /* CG iterations (inner iterations summed) */
    int outer_iters;        /* refinement steps (0 for plain FP64 PCG) */
    double rel_res;         /* final relative residual ||b - A x||/||b|| in FP64 */
    double seconds;         /* wall time of the solve on the device */
    nb_status status;
    int history_len;        /* entries written to history_host */
    double *history_host;   /* caller-provided, history_cap entries, or NULL */
    int history_cap;
    int64_t launches;       /* kernels launched by the solve (graph nodes included) */
    nb_prec final_prec;     /* precision of the last inner solve: opts.prec, or a higher one
                               when the refinement raised it (precision adaptivity: after
                               two refinement steps in which the FP64 residual did not
                               halve, the inner solves go from the tensor-core precisions
                               to NB_FP32, and from NB_FP32 to FP64 PCG; NB_STAGNATED only
                               when FP64 inner solves stall too) */
} nb_stats;

/* Library version string. */
const char *nb_version(void);

/* Message of the last error on the calling thread ("" if none). */
const char *nb_last_error(void);

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to issue work on, or NULL for a stream owned by the context; that stream is
 * a blocking stream, so it is ordered with work on the legacy default stream.
 * The solver captures CUDA graphs on the context's stream, so it must not be
 * the legacy default stream itself (pass NULL instead).
 * Errors: NB_ERR_ARG (bad device), NB_ERR_CUDA. */
nb_status nb_create(nb_ctx **ctx, int device, void *cuda_stream);

/* Replace the stream used by later calls (NULL: the context's own stream). */
nb_status nb_set_stream(nb_ctx *ctx, void *cuda_stream);

nb_status nb_destroy(nb_ctx *ctx);

/* Build the box mesh of nx*ny*nz hexahedral elements of order N (1 <= N <= 15)
 * on the unit cube, nodes at the Gauss-Lobatto-Legendre points, displaced by
 * a*sin(pi x)sin(pi y)sin(pi z) in each coordinate with a = deform/max(nx,ny,nz),
 * and compute on the device the six geometric factors per node (FP64 and FP32
 * copies).  The paper keeps this initialisation in double (Section 6, step 3).
 * Errors: NB_ERR_ARG (sizes), NB_ERR_MESH (a non-positive Jacobian),
 * NB_ERR_OOM. */
nb_status nb_setup_mesh(nb_ctx *ctx, int nx, int ny, int nz, int N,
                        double deform, nb_mesh **out);

/* Build the global numbering, multiplicities, Dirichlet mask (homogeneous on
 * the box boundary), the gather-scatter lists of shared or masked nodes, the
 * dot-product weights c = 1/multiplicity and the Jacobi inverse diagonal.
 * Must follow nb_setup_mesh.  Errors: NB_ERR_STATE, NB_ERR_OOM, NB_ERR_CUDA. */
nb_status nb_setup_gs(nb_mesh *mesh);

nb_status nb_mesh_destroy(nb_mesh *mesh);

/* Sizes: out[0]=E, out[1]=N, out[2]=n_local, out[3]=n_global,
 * out[4]=number of gather-scatter rows (shared or masked global nodes),
 * out[5]=total local copies in those rows, out[6..8]=nx,ny,nz. */
nb_status nb_mesh_sizes(const nb_mesh *mesh, int64_t out[9]);

/* Copy the index maps to host buffers for inspection (any may be NULL):
 * gid[n_local] global node of each local node; mult[n_global];
 * mask[n_global] (1 free, 0 Dirichlet); gs_row_gid[rows] global node of each
 * gather-scatter row (ascending); gs_off[rows+1] row offsets; gs_loc[copies]
 * local copies of each row in ascending order; gs_mask[rows]. */
nb_status nb_get_maps(const nb_mesh *mesh, int32_t *gid, int32_t *mult,
                      uint8_t *mask, int32_t *gs_row_gid, int32_t *gs_off,
                      int32_t *gs_loc, uint8_t *gs_mask);

/* Copy geometry to host buffers (any may be NULL): G[E][6][n^3] in FP64,
 * order (rr, rs, rt, ss, st, tt); dinv[n_local] Jacobi inverse diagonal
 * (0 on Dirichlet nodes); c[n_local] = 1/multiplicity. */
nb_status nb_get_geom(const nb_mesh *mesh, double *G, double *dinv, double *c);

/* u_L = Q u_G: copy each global value to all its local copies; masked != 0
 * also zeroes Dirichlet nodes.  Both vectors in the precision's type. */
nb_status nb_to_local(nb_mesh *mesh, nb_prec prec, const void *ug_dev,
                      void *uL_dev, int masked);

/* u_G = value of a continuous L-vector at each global node (first copy). */
nb_status nb_to_global(nb_mesh *mesh, nb_prec prec, const void *uL_dev,
                       void *ug_dev);

/* Matrix-free operator ax (Table 1 line 5): w_L = A_L u_L element by element,
 * A_e = D^T G D over the n^3 GLL nodes with six geometric factors per node
 * (local_grad3, geometric factors, local_grad3_t).  assemble != 0 follows
 * with the direct-stiffness summation and the Dirichlet mask (dssum), giving
 * the assembled operator on continuous vectors.  u_dev and w_dev must not
 * overlap.  prec: NB_FP64 (double), NB_FP32 (float), NB_TC_F16/NB_TC_BF16
 * (float vectors; derivative contractions on tensor cores, FP32 accumulate). */
nb_status nb_ax(nb_mesh *mesh, nb_prec prec, int assemble, const void *u_dev,
                void *w_dev);

/* Direct-stiffness summation in place (gather-scatter over shared nodes, sum
 * in ascending local index), then the Dirichlet mask if masked != 0.
 * Deterministic: the same input gives bit-identical output. */
nb_status nb_dssum(nb_mesh *mesh, nb_prec prec, void *u_dev, int masked);

/* glsc3 (Table 1 lines 3, 6, 9): *out_host = sum_l a_l b_l c_l with
 * c = 1/multiplicity; products in the precision's type, accumulated in FP64
 * in a fixed order (deterministic). */
nb_status nb_glsc3(nb_mesh *mesh, nb_prec prec, const void *a_dev,
                   const void *b_dev, double *out_host);

/* Fill opts with defaults: FP32 inner solve with FP64 refinement, Jacobi,
 * rtol 1e-10, maxiter 10000, inner_rtol 1e-4, max_outer 30, use_graph 1,
 * record_history 0, use_x0 0. */
void nb_default_opts(nb_opts *opts);

/* Solve A x = b for the assembled, masked operator.  b_dev and x_dev are FP64
 * L-vectors; b must be continuous and zero on Dirichlet nodes; with use_x0 = 1
 * x_dev holds the initial guess on entry (continuous, masked); it holds the
 * solution on exit.
 * NB_FP64: preconditioned CG in the order of Table 1, all in FP64.
 * With use_x0 = 0 the initial guess is zero and x_dev is only written.
 * Other precisions: FP64 iterative refinement -- r = b - A x in FP64, an inner
 * PCG (or flexible CG with NB_PC_LEARNED) in the reduced precision with FP64
 * dot-product accumulation, then x += correction in FP64 -- until the FP64
 * residual meets rtol.  stats may be NULL.
 * Returns NB_OK, a positive outcome, or a negative error. */
nb_status nb_solve(nb_mesh *mesh, const nb_opts *opts, const double *b_dev,
                   double *x_dev, nb_stats *stats);

/* nb_solve with host G-vectors: bg_host[n_global] right-hand side (masked on
 * the device), xg_host[n_global] solution (initial guess zero).  Copies
 * host->device and device->host inside the call. */
nb_status nb_solve_host(nb_mesh *mesh, const nb_opts *opts,
                        const double *bg_host, double *xg_host, nb_stats *stats);

/* Measure the operator kernel: `reps` launches on the context's stream, each
 * bracketed by CUDA events, with `flush_bytes` of `flush_dev` overwritten and
 * then read back between launches (outside the events) to evict the L2 cache
 * and write its dirty lines back, so every launch starts on a clean cache
 * holding none of its data; flush_dev may be NULL (flush_bytes should exceed
 * the L2 size).  cg_step = 0 times ax (u -> w, the nb_ax kernel); cg_step = 1 times
 * the fused CG-step kernel of the solver (p = dinv*r + beta*p, w = A_L p,
 * partial p.w) on the mesh's solve workspace.  variant: -1 for the current
 * choice, else a kernel variant index (see nb_autotune).  *ms_out = mean
 * milliseconds per launch.  Errors: NB_ERR_ARG, NB_ERR_STATE, NB_ERR_CUDA. */
nb_status nb_time_ax(nb_mesh *mesh, nb_prec prec, int cg_step, int variant, int reps,
                     void *flush_dev, size_t flush_bytes, double *ms_out);

/* Number of operator kernel variants available for (mesh order, prec). */
int nb_ax_variants(const nb_mesh *mesh, nb_prec prec);

/* Select operator variant `variant` (0 <= variant < nb_ax_variants) for
 * later operator applications and solves in precision prec on this mesh,
 * or -1 for the built-in default; the choice nb_autotune would otherwise
 * make by timing.  Errors: NB_ERR_ARG (index out of range, bad prec). */
nb_status nb_set_ax_variant(nb_mesh *mesh, nb_prec prec, int variant);

/* Kernel of the FP32 iteration's update with the folded direct-stiffness
 * summation (x += alpha p, r -= alpha dssum(w), the next dots), for even
 * N + 1: 0 the built-in choice (1 up to N = 9, else 2), 1 contiguous element
 * ranges per block with the pair positions fixed per thread, 2 node pairs
 * dealt round-robin over a persistent grid, 3 element ranges with x, r, p
 * and dinv streamed by bulk copies into a two-stage shared-memory ring.  All
 * sum in the same order (bit-identical results).  Errors: NB_ERR_ARG. */
nb_status nb_set_update_variant(nb_mesh *mesh, int variant);

/* Deferred x steps of the FP32 Jacobi iteration, where the update is variant
 * 1 and the operator the pencil kernel: the iteration alternates two
 * direction buffers, the first iteration of each pair skips x += alpha p and
 * the second applies both steps in the same order (same bits).  mode -1 the
 * built-in rule (where x, r, the two directions, w and dinv, 24 bytes per
 * local node, exceed the L2 cache), 0 never, 1 wherever those kernels run.
 * Costs one more L-vector of workspace.  Errors: NB_ERR_ARG (mode). */
nb_status nb_set_x_deferral(nb_mesh *mesh, int mode);

/* Kernel name of operator variant `variant` for (mesh order, prec), or of
 * the variant in use with variant = -1 (a static string owned by the
 * library; NULL for an index out of range, a NULL mesh or a bad prec). */
const char *nb_ax_variant_name(const nb_mesh *mesh, nb_prec prec, int variant);

/* Index of the operator variant that operator applications and solves in
 * precision prec use now (the built-in default until one is chosen), or -1
 * for a NULL mesh or a bad prec. */
int nb_ax_variant_in_use(const nb_mesh *mesh, nb_prec prec);

/* Autotuner: time every operator variant for this mesh's order and
 * precision with nb_time_ax (cg_step = 1, `reps` launches each) and keep the
 * fastest for later calls.  *best_variant and *best_ms (may be NULL) receive
 * the choice.  Variants differ only in launch shape and in how sums inside
 * one element are associated, so their results agree to rounding. */
nb_status nb_autotune(nb_mesh *mesh, nb_prec prec, int reps, void *flush_dev,
                      size_t flush_bytes, int *best_variant, double *best_ms);

/* ------------------------------------------------------------------------
 * Batched solves: many independent Poisson problems of different size and
 * order solved together, every CG iteration of all problems captured in one
 * CUDA graph (the extension of Table 1's loop to a batch; the paper solves one
 * problem per process).
 * ------------------------------------------------------------------------ */
typedef struct nb_batch nb_batch;

/* Build nprob box meshes (arrays of length nprob: element counts, orders
 * 1 <= N <= 15, deformations as in nb_setup_mesh) with their gather-scatter,
 * and lay them out as one batch.  The batch L-vector stores the problems one
 * after another, grouped by order (problems of equal order keep their
 * relative order); nb_batch_layout reports where each problem sits.
 * Errors: NB_ERR_ARG, NB_ERR_MESH, NB_ERR_OOM, NB_ERR_CUDA. */
nb_status nb_batch_create(nb_ctx *ctx, int nprob, const int *nx, const int *ny, const int *nz,
                          const int *N, const double *deform, nb_batch **out);

nb_status nb_batch_destroy(nb_batch *batch);

/* Per problem p (caller's numbering): l_off[p] = offset of its L-vector in
 * the batch L-vector, g_off[p] = offset of its G-vector in the batch G-vector
 * (G-vectors concatenated in the caller's order), and if not NULL
 * totals[0] = batch L length, totals[1] = batch G length. */
nb_status nb_batch_layout(const nb_batch *batch, int64_t *l_off, int64_t *g_off,
                          int64_t totals[2]);

/* The mesh of problem p (owned by the batch), e.g. for nb_to_local on it. */
nb_mesh *nb_batch_mesh(nb_batch *batch, int p);

/* Batch L-vector from the concatenated G-vectors (FP64), masked. */
nb_status nb_batch_to_local(nb_batch *batch, const double *ug_dev, double *uL_dev);

/* Solve every problem of the batch: b_dev, x_dev are FP64 batch L-vectors
 * (x: solution out; opts.use_x0 as in nb_solve).  opts.prec: NB_FP64 (plain
 * PCG for all problems) or NB_FP32 (FP64 refinement around batched FP32 PCG,
 * per-problem scaling and inner tolerances).  Each problem stops on its own
 * criterion; the batch stops when all have.  stats[p] (array of nprob, may
 * be NULL) receives each problem's outcome; *total (may be NULL) the batch's
 * (iters = batched iterations, seconds = wall time, launches).
 * Returns the worst outcome over the problems, or a negative error. */
nb_status nb_batch_solve(nb_batch *batch, const nb_opts *opts, const double *b_dev,
                         double *x_dev, nb_stats *stats, nb_stats *total);

/* Autotuner for the batch: for every order present, time each operator
 * variant on that order's elements (reps launches) and keep the fastest. */
nb_status nb_batch_autotune(nb_batch *batch, int reps, void *flush_dev, size_t flush_bytes);

/* ------------------------------------------------------------------------
 * Learned preconditioner: a per-element network mapping an element's
 * residual x = r_e / |r_e| to a correction on the element's interior nodes,
 * y(x) = W (a * gelu(W^T x)) -- one hidden layer of h units whose output
 * layer reuses the input weights W (d x h) with per-unit gains a, so that
 * its Jacobian is symmetric -- used as z = Dinv r + M_int(|r_e| y(x)) inside
 * flexible CG (orders N <= 11).  BF16 tensor-core products with FP32
 * accumulation, FP32 master weights.  Not in the paper; it takes the slot of
 * the paper's multigrid solveM with a learned element-interior correction.
 * ------------------------------------------------------------------------ */
typedef struct nb_model nb_model;

/* A network for order N: d = (N+1)^3 inputs and outputs, `hidden` units,
 * W uniform(-1,1)/sqrt(d) drawn from SplitMix64(seed), gains a = 1. */
nb_status nb_model_create(nb_ctx *ctx, int N, int hidden, uint64_t seed, nb_model **out);
nb_status nb_model_destroy(nb_model *model);

/* Parameters as one FP32 host array [W (d x h, row-major), a (h)]: copied
 * out to get_host and/or in from set_host (either may be NULL); *nparam (may
 * be NULL) receives the count d h + h. */
nb_status nb_model_params(nb_model *model, float *get_host, const float *set_host,
                          int64_t *nparam);

/* Loss sum((Y - T)^2) / (B d) and its gradient (same layout as the
 * parameters) on B pairs X, T (device, B x d FP32, row-major). */
nb_status nb_model_grad(nb_model *model, const float *X_dev, const float *T_dev, int B,
                        double *loss_host, float *grad_host);

/* Adam (lr, 0.9, 0.999, 1e-8) over `epochs` passes of consecutive minibatches
 * of `batch` pairs; *final_loss (may be NULL) = mean loss of the last epoch. */
nb_status nb_model_train(nb_model *model, const float *X_dev, const float *T_dev, int npairs,
                         int epochs, int batch, float lr, double *final_loss);

/* Training pairs from the solver itself, for b (FP64 L-vector, continuous,
 * masked): for each of nsnap iteration counts k, the solver's iterate x_k
 * after k steps from zero -- Jacobi-PCG in FP64, or with use_learned != 0 the
 * refinement's flexible CG with the attached network -- and its residual
 * r_k = b - A x_k; then for per_snap elements drawn with SplitMix64(seed) the
 * pair of nb_learned_targets.  X_dev, T_dev: device FP32, capacity
 * nsnap * per_snap * d.  *count = pairs written.  Errors: NB_ERR_ARG (also
 * N > 11), NB_ERR_STATE, NB_ERR_OOM, NB_ERR_CUDA. */
nb_status nb_learned_collect(nb_mesh *mesh, const double *b_dev, int nsnap,
                             const int *snap_iters, int per_snap, uint64_t seed,
                             int use_learned, float *X_dev, float *T_dev, int *count);

/* Pairs for given elements (device int32) of a residual L-vector r (FP64,
 * device): X = r_e/|r_e|, T = (A_ii^-1 r_i - Dinv r_i)/|r_e| on the
 * element's interior nodes and 0 on its boundary nodes, A_ii the operator's
 * block on the element interior (solved by conjugate gradients per element
 * to 1e-9 relative, in FP64). */
nb_status nb_learned_targets(nb_mesh *mesh, const double *r_dev, const int32_t *elems_dev,
                             int count, float *X_dev, float *T_dev);

/* Use `model` (NULL detaches) as the mesh's NB_PC_LEARNED preconditioner.
 * The model must outlive its use. */
nb_status nb_learned_attach(nb_mesh *mesh, nb_model *model);

/* Apply the attached preconditioner once: z = B(r), FP32 L-vectors. */
nb_status nb_learned_apply(nb_mesh *mesh, const float *r_dev, float *z_dev);

/* One application of the fused preconditioner step of the learned flexible CG
 * (Sections 4.1 and 6: solveM and the two glsc3 that follow it, with the
 * network of the learned preconditioner as solveM), the kernel the inner FP32
 * solve runs every iteration: z = B(r) as nb_learned_apply, and in the same
 * pass *zw = sum over every local copy of z * w_prev (w_prev the unassembled
 * A p of the previous step) and *rz = (r, c, z) over owner copies.  r_dev,
 * wprev_dev, z_dev: device FP32 L-vectors (r continuous and masked);
 * zw / rz: host doubles.  Available for FP32 meshes with N in {1, 3, 5, 7}
 * and hidden width <= 128 (else NB_ERR_ARG).  Errors: NB_ERR_ARG,
 * NB_ERR_STATE (no model attached), NB_ERR_CUDA (also a timed-out wait inside
 * the kernel). */
nb_status nb_learned_step(nb_mesh *mesh, const float *r_dev, const float *wprev_dev,
                          float *z_dev, double *zw, double *rz);

/* ------------------------------------------------------------------------
 * Emulated reduced precision (Section 2: Verificarlo's VPREC backend
 * computes every floating-point operation in the original type and rounds
 * its result to a pseudo-mantissa of t bits; Section 4.2 sweeps t from 3 to
 * 52 over the CG loop).  Here: binary64 with every +, -, *, / of the loop
 * rounded to t bits (1 <= t <= 52), round to nearest, ties to even, the
 * binary64 exponent range kept.  The operator and the direct-stiffness
 * summation take their operations in the order of the plain definitions
 * (per node the l-loops in turn; per global node the copies in ascending
 * local index); dot products are summed per thread, per block in a fixed
 * tree and over blocks in index order.  A study tool, not a fast path.
 * ------------------------------------------------------------------------ */

/* w = M Q Q^T A_L u with every operation rounded to t bits (FP64 L-vectors,
 * device).  Errors: NB_ERR_ARG (t outside 1..52, NULL), NB_ERR_STATE. */
nb_status nb_apply_vprec(nb_mesh *mesh, int t, const double *u_dev, double *w_dev);

/* `iters` CG iterations from x = 0 (Nekbone's fixed iteration count) with
 * every operation of the loop rounded to t bits; pc: NB_PC_NONE (the
 * paper's no-preconditioner case) or NB_PC_JACOBI.  b_dev: FP64 L-vector
 * (continuous, masked); x_dev receives the iterate.  hist_host (may be NULL,
 * iters doubles) receives the loop's relative residual sqrt(rtr)/|b| after
 * each iteration; *relres (may be NULL) the last.  |b| and the set-up stay
 * in binary64.  Allocates and frees its own scratch. */
nb_status nb_cg_vprec(nb_mesh *mesh, int t, int iters, nb_pc pc, const double *b_dev,
                      double *x_dev, double *hist_host, double *relres);

/* The same loop with Monte Carlo Arithmetic instead of rounding (Section 2,
 * the MCA backend; Section 4.2 runs it at t = 23, 20 samples): every
 * operation is computed in binary64 and its result (mode 1, random
 * rounding) or its operands and result (mode 2, full MCA) are perturbed,
 * inexact(x) = x + 2^(e_x - t) xi, xi uniform on (-1/2, 1/2),
 * 2^(e_x - 1) <= |x| < 2^e_x.  Random numbers: SplitMix64 streams keyed by
 * seed, launch and thread, so a run is reproducible for a given seed and
 * launch shape.  Arguments as nb_cg_vprec; NB_ERR_ARG for another mode. */
nb_status nb_cg_mca(nb_mesh *mesh, int mode, int t, uint64_t seed, int iters, nb_pc pc,
                    const double *b_dev, double *x_dev, double *hist_host, double *relres);

/* ------------------------------------------------------------------------
 * Overlapping Schwarz preconditioner (Section 4.1 names Nekbone's multigrid
 * solveM routines h1mg_schwarz, h1mg_fdm, h1mg_extrude, h1mg_do_fast,
 * h1mg_tnsr3d_el; the paper gives no algorithm, this is the textbook
 * one-level method with minimal overlap): z = sum_e R_e^T A_e^-1 R_e r, R_e
 * the restriction to element e extended by one GLL layer into each
 * neighbour, A_e the separable operator on the undeformed box inverted by
 * fast diagonalisation.  Symmetric positive definite; used by NB_PC_SCHWARZ.
 * ------------------------------------------------------------------------ */

/* z = M r once, FP32 L-vectors (continuous, masked), device.  Builds the 1D
 * eigenvectors and the scratch on first use (allocates).  Orders N <= 11. */
nb_status nb_schwarz_apply(nb_mesh *mesh, const float *r_dev, float *z_dev);

/* Two-level form: z = sum_e R_e^T A_e^-1 R_e r + R_0^T A_0^-1 R_0 r, with R_0^T the
 * trilinear interpolation from the interior element vertices to the GLL nodes and
 * A_0 = R_0 A R_0^T the Galerkin coarse operator of the undeformed box (separable:
 * Q1 stiffness and mass per direction for N >= 2), inverted by fast
 * diagonalisation in one thread block (the coarse-grid level of the multigrid
 * solveM of Section 4.1; textbook two-level additive Schwarz).  Arguments, layout,
 * ownership and errors as nb_schwarz_apply; NB_ERR_ARG beyond 65 elements per
 * direction or 24576 interior vertices.  Used by NB_PC_SCHWARZ2. */
nb_status nb_schwarz2_apply(nb_mesh *mesh, const float *r_dev, float *z_dev);

/* ------------------------------------------------------------------------
 * Slab partition along z and the CG iteration in split phases.  Nekbone runs
 * its CG on MPI ranks that each own a set of elements (Section 4.1: dssum
 * exchanges the shared nodes, glsc3 ends in a global sum; Section 7.2 /
 * Table 5 scale it over ranks).  Here a box of nx x ny x nz elements is cut
 * into z-slabs, one mesh per slab (on one or several GPUs, in one or several
 * processes); the slabs share the node planes between them.  A driver runs
 * Table 1's loop by calling, on every slab, nb_cg_step (then summing the
 * slabs' p.w), the summation of w (nb_slab_face before nb_dssum, the
 * neighbours' planes added with nb_slab_face_add after it), and nb_cg_update
 * (then summing the slabs' dots); paper_2405_11065_gb300/slab.py is such a
 * driver, in-process or over torch.distributed.
 * ------------------------------------------------------------------------ */

/* The slab z0 <= ez < z1 of the nx x ny x nz box of nb_setup_mesh (same
 * arguments otherwise, the box's geometry and deformation): a mesh of
 * nx x ny x (z1 - z0) elements.  After nb_setup_gs its Dirichlet boundary is
 * the box's; the plane at z0 (if z0 > 0) and at z1 (if z1 < nz) are free
 * interface planes, the lower one owned by the slab below (its copies are
 * not owners in the dots), and the dot-product weights c count the copies
 * on both sides.  Its Jacobi diagonal lacks the neighbours' part on the
 * interface planes until nb_slab_finish_diag.
 * Errors: NB_ERR_ARG (bounds, sizes), NB_ERR_MESH, NB_ERR_OOM. */
nb_status nb_setup_slab(nb_ctx *ctx, int nx, int ny, int nz, int z0, int z1, int N,
                        double deform, nb_mesh **out);

/* Interface plane side (0: lower, 1: upper) of a slab: face_dev[gx + Gx gy]
 * (Gx = nx N + 1, Gy = ny N + 1 values, device, precision's type) = the sum
 * over the slab's copies of each plane node of the L-vector u_dev, taken
 * before nb_dssum.  Errors: NB_ERR_ARG (no interface on that side). */
nb_status nb_slab_face(nb_mesh *mesh, nb_prec prec, int side, const void *u_dev,
                       void *face_dev);

/* After nb_dssum: add the neighbouring slab's plane vector face_dev (its
 * nb_slab_face on the shared plane) to every copy of the plane's free nodes
 * of u_dev.  u then holds the box's direct-stiffness sum on this slab.
 * Errors: NB_ERR_ARG. */
nb_status nb_slab_face_add(nb_mesh *mesh, nb_prec prec, int side, void *u_dev,
                           const void *face_dev);

/* The slab's part of the assembled diagonal on interface plane `side`
 * (FP64 plane vector, device). */
nb_status nb_slab_diag_face(nb_mesh *mesh, int side, double *face_dev);

/* Complete the Jacobi inverse diagonal with the neighbours' parts (their
 * nb_slab_diag_face on the shared planes; NULL exactly where the slab has
 * no interface).  Errors: NB_ERR_ARG, NB_ERR_STATE. */
nb_status nb_slab_finish_diag(nb_mesh *mesh, const double *face_lo_dev,
                              const double *face_hi_dev);

/* One step of Table 1 on this mesh (lines 2-5 without the summation of w):
 * p = Dinv r + beta p (solveM, add2s1), w = A_L p element by element, and
 * *pap_host = sum of p.w over the mesh's local nodes in FP64 (for a
 * continuous masked p the partial of glsc3(w, c, p) after summation).
 * L-vectors on the device in the precision's type; p must hold the previous
 * direction (zeros before the first step, with beta = 0).  Synchronises. */
nb_status nb_cg_step(nb_mesh *mesh, nb_prec prec, double beta, const void *r_dev,
                     void *p_dev, void *w_dev, double *pap_host);

/* Lines 7-9: x += alpha p, r -= alpha w with w summed and masked, then
 * dots_host[0] = (r, c, Dinv r) and dots_host[1] = (r, c, r) over this mesh
 * (FP64 accumulation; on a slab the partials of the box's dots). */
nb_status nb_cg_update(nb_mesh *mesh, nb_prec prec, double alpha, void *x_dev, void *r_dev,
                       const void *p_dev, const void *w_dev, double *dots_host);

/* dots_host[0] = (r, c, Dinv r), dots_host[1] = (r, c, r) of r on this mesh
 * (the dots of the first iteration). */
nb_status nb_cg_dots(nb_mesh *mesh, nb_prec prec, const void *r_dev, double *dots_host);

/* nb_glsc3 for callers that cannot let a library allocate memory: a
 * framework whose caching allocator owns the device memory, a process under
 * a hard memory budget, or a latency-critical loop that must not pay for
 * cudaMalloc's device synchronisation.  (The paper has no counterpart: this is
 * an interface variant of glsc3, not part of the method.)
 * Same arguments and result as nb_glsc3; the only difference is where the
 * scratch lives: the per-block partial sums and the final scalar use a fixed
 * array of 2048 + 1 doubles (16 KB) in the library's device memory, which
 * every GPU that loads the library holds until the process exits.  No call
 * to cudaMalloc, cudaFree, cudaMallocHost or any allocating routine is made.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream
 * capture.  Every call shares the array: calls whose kernels overlap on the
 * GPU (several streams, several host threads) race and may return wrong
 * sums; issue them in order on one stream.  The array keeps the last call's
 * contents; each call writes every slot it reads, so nothing is cleared.
 * Errors: NB_ERR_ARG (NULL pointer, bad precision, or a launch that would
 * need more than 2048 partial sums), NB_ERR_STATE, NB_ERR_CUDA. */
nb_status nb_glsc3_noalloc(nb_mesh *mesh, nb_prec prec, const void *a_dev,
                           const void *b_dev, double *out_host);

#ifdef __cplusplus
}
#endif

#endif /* NEKBONE_GB300_H */
