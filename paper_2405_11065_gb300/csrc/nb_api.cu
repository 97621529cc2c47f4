// The C ABI (include/nekbone_gb300.h): argument validation, object lifetime,
// and dispatch to the device code.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "nb_internal.h"

namespace nb {

static thread_local char g_err[512] = "";
thread_local bool g_pdl = false;

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static nb_status arg_error(const char *what)
{
    set_error("invalid argument: %s", what);
    return NB_ERR_ARG;
}

static bool prec_ok(nb_prec p) { return p >= NB_FP64 && p <= NB_TC_BF16; }

static void free_ws(Workspace &ws)
{
    if (ws.exec) cudaGraphExecDestroy(ws.exec);
    if (ws.graph) cudaGraphDestroy(ws.graph);
    if (ws.exec2) cudaGraphExecDestroy(ws.exec2);
    if (ws.graph2) cudaGraphDestroy(ws.graph2);
    cudaFree(ws.x);
    cudaFree(ws.r);
    cudaFree(ws.p);
    cudaFree(ws.w);
    cudaFree(ws.z);
    cudaFree(ws.aux);
    cudaFree(ws.p2);
    cudaFree(ws.part);
    cudaFree(ws.scal);
    cudaFree(ws.hist);
    if (ws.scal_host) cudaFreeHost(ws.scal_host);
    ws = Workspace();
}

void learned_free(nb_mesh *m);  // nb_learned.cu
void schwarz_free(nb_mesh *m);  // nb_schwarz.cu

}  // namespace nb

using namespace nb;

namespace nb {

void ctx_retain(nb_ctx *c) { c->refs.fetch_add(1); }

void ctx_release(nb_ctx *c)
{
    if (c->refs.fetch_sub(1) != 1) return;
    if (c->own_stream) {
        DeviceGuard g(c->device);
        cudaStreamDestroy(c->own_stream);
    }
    delete c;
}

}  // namespace nb

extern "C" {

const char *nb_version(void) { return "nekbone-gb300 0.1 (sm_103a)"; }

const char *nb_last_error(void) { return g_err; }

nb_status nb_create(nb_ctx **ctx, int device, void *cuda_stream)
{
    if (!ctx) return arg_error("ctx is NULL");
    *ctx = nullptr;
    int count = 0;
    NB_CUDA(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return arg_error("device index out of range");
    NB_DEVICE_SCOPE(device);
    nb_ctx *c = new nb_ctx();
    c->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->l2_bytes, cudaDevAttrL2CacheSize, device);
    if (e != cudaSuccess) {
        delete c;
        NB_CUDA(e);
    }
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        // a blocking stream: ordered with work on the legacy default stream
        e = cudaStreamCreate(&c->own_stream);
        if (e != cudaSuccess) {
            delete c;
            NB_CUDA(e);
        }
        c->stream = c->own_stream;
    }
    *ctx = c;
    return NB_OK;
}

nb_status nb_set_stream(nb_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return arg_error("ctx is NULL");
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (!ctx->own_stream) NB_CUDA(cudaStreamCreate(&ctx->own_stream));
        ctx->stream = ctx->own_stream;
    }
    return NB_OK;
}

nb_status nb_destroy(nb_ctx *ctx)
{
    if (!ctx) return NB_OK;
    ::nb::ctx_release(ctx);
    return NB_OK;
}

nb_status nb_mesh_destroy(nb_mesh *m)
{
    if (!m) return NB_OK;
    ::nb::DeviceGuard nb_device_guard_(m->ctx->device);
    cudaStreamSynchronize(m->ctx->stream);
    learned_free(m);
    schwarz_free(m);
    free_ws(m->ws64);
    free_ws(m->ws32);
    void *bufs[] = {m->D64, m->D32, m->G64, m->G32, m->gid, m->gs_off, m->gs_loc, m->gs_gid,
                    m->gs_mask, m->g_first, m->mask_g, m->c32, m->dinv64, m->dinv32,
                    m->ones64, m->ones32, m->r64, m->w64, m->x64, m->b64, m->g64, m->part64,
                    m->red_out, m->kerr, m->gs_zero, m->gs_pair, m->gs_quad, m->gs_oct,
                    m->diag_asm, m->scal_split};
    for (void *b : bufs) cudaFree(b);
    if (m->red_host) cudaFreeHost(m->red_host);
    nb_ctx *ctx = m->ctx;
    delete m;
    ::nb::ctx_release(ctx);
    return NB_OK;
}

// A box of nx x ny x nz elements, or (nz_glob > nz) the slab of elements
// z_off .. z_off + nz - 1 along z of a box of nz_glob elements.
static nb_status setup_mesh_impl(nb_ctx *ctx, int nx, int ny, int nz, int z_off, int nz_glob,
                                 int N, double deform, nb_mesh **out)
{
    if (!ctx || !out) return arg_error("NULL ctx or out");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return arg_error("element counts must be >= 1");
    if (z_off < 0 || z_off + nz > nz_glob) return arg_error("slab outside the box");
    if (N < 1 || N > kMaxN) {
        set_error("order N=%d outside [1, %d]", N, kMaxN);
        return NB_ERR_MESH;
    }
    if (!(deform >= 0.0) || !isfinite(deform)) return arg_error("deform must be finite, >= 0");
    const int64_t n = N + 1;
    const int64_t E = (int64_t)nx * ny * nz;
    const int64_t nL = E * n * n * n;
    const int64_t nG = ((int64_t)nx * N + 1) * ((int64_t)ny * N + 1) * ((int64_t)nz * N + 1);
    if (nL >= (int64_t)1 << 31 || nG >= (int64_t)1 << 31)
        return arg_error("mesh too large for 32-bit local/global indices");
    NB_DEVICE_SCOPE(ctx->device);
    nb_mesh *m = new nb_mesh();
    m->ctx = ctx;
    ::nb::ctx_retain(ctx);
    m->nx = nx;
    m->ny = ny;
    m->nz = nz;
    m->N = N;
    m->n = N + 1;
    m->n3 = m->n * m->n * m->n;
    m->deform = deform;
    m->z_off = z_off;
    m->nz_glob = nz_glob;
    m->iface_lo = z_off > 0;
    m->iface_hi = z_off + nz < nz_glob;
    m->E = E;
    m->nL = nL;
    m->nG = nG;
    nb_status st = build_geometry(m);
    if (st != NB_OK) {
        nb_mesh_destroy(m);
        return st;
    }
    *out = m;
    return NB_OK;
}

nb_status nb_setup_mesh(nb_ctx *ctx, int nx, int ny, int nz, int N, double deform,
                        nb_mesh **out)
{
    return setup_mesh_impl(ctx, nx, ny, nz, 0, nz, N, deform, out);
}

nb_status nb_setup_slab(nb_ctx *ctx, int nx, int ny, int nz, int z0, int z1, int N,
                        double deform, nb_mesh **out)
{
    if (!(z0 >= 0 && z0 < z1 && z1 <= nz)) {
        if (out) *out = nullptr;
        return arg_error("slab bounds need 0 <= z0 < z1 <= nz");
    }
    return setup_mesh_impl(ctx, nx, ny, z1 - z0, z0, nz, N, deform, out);
}

nb_status nb_setup_gs(nb_mesh *m)
{
    if (!m) return arg_error("mesh is NULL");
    if (m->gs_ready) return NB_OK;
    if (!m->G64) {
        set_error("nb_setup_gs before nb_setup_mesh");
        return NB_ERR_STATE;
    }
    NB_DEVICE_SCOPE(m->ctx->device);
    return build_gs(m);
}

nb_status nb_mesh_sizes(const nb_mesh *m, int64_t out[9])
{
    if (!m || !out) return arg_error("NULL mesh or out");
    out[0] = m->E;
    out[1] = m->N;
    out[2] = m->nL;
    out[3] = m->nG;
    out[4] = m->gs_rows;
    out[5] = m->gs_copies;
    out[6] = m->nx;
    out[7] = m->ny;
    out[8] = m->nz;
    return NB_OK;
}

// A pipelined kernel whose bounded wait gave up sets m->kerr (it then exits
// without finishing its elements): report it as a CUDA error.
static nb_status check_kernel_flag(nb_mesh *m)
{
    int flag = 0;
    NB_CUDA(cudaMemcpy(&flag, m->kerr, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        cudaMemset(m->kerr, 0, sizeof(int));
        set_error("a bulk-copy wait in the operator timed out; results are incomplete");
        return NB_ERR_CUDA;
    }
    return NB_OK;
}

static nb_status need_gs(const nb_mesh *m)
{
    if (!m) return arg_error("mesh is NULL");
    if (!m->gs_ready) {
        set_error("call nb_setup_gs first");
        return NB_ERR_STATE;
    }
    return NB_OK;
}

nb_status nb_get_maps(const nb_mesh *m, int32_t *gid, int32_t *mult, uint8_t *mask,
                      int32_t *gs_row_gid, int32_t *gs_off, int32_t *gs_loc, uint8_t *gs_mask)
{
    NB_TRY(need_gs(m));
    NB_DEVICE_SCOPE(m->ctx->device);
    if (gid) NB_CUDA(cudaMemcpy(gid, m->gid, sizeof(int32_t) * m->nL, cudaMemcpyDeviceToHost));
    if (mult) memcpy(mult, m->mult_host.data(), sizeof(int32_t) * m->nG);
    if (mask) memcpy(mask, m->mask_host.data(), m->nG);
    if (gs_row_gid && m->gs_rows)
        NB_CUDA(cudaMemcpy(gs_row_gid, m->gs_gid, sizeof(int32_t) * m->gs_rows,
                           cudaMemcpyDeviceToHost));
    if (gs_off)
        NB_CUDA(cudaMemcpy(gs_off, m->gs_off, sizeof(int32_t) * (m->gs_rows + 1),
                           cudaMemcpyDeviceToHost));
    if (gs_loc && m->gs_copies)
        NB_CUDA(cudaMemcpy(gs_loc, m->gs_loc, sizeof(int32_t) * m->gs_copies,
                           cudaMemcpyDeviceToHost));
    if (gs_mask && m->gs_rows)
        NB_CUDA(cudaMemcpy(gs_mask, m->gs_mask, m->gs_rows, cudaMemcpyDeviceToHost));
    return NB_OK;
}

nb_status nb_get_geom(const nb_mesh *m, double *G, double *dinv, double *c)
{
    if (!m) return arg_error("mesh is NULL");
    NB_DEVICE_SCOPE(m->ctx->device);
    if (G) NB_CUDA(cudaMemcpy(G, m->G64, sizeof(double) * 6 * m->nL, cudaMemcpyDeviceToHost));
    if (dinv || c) NB_TRY(need_gs(m));
    if (dinv) {
        NB_CUDA(cudaMemcpy(dinv, m->dinv64, sizeof(double) * m->nL, cudaMemcpyDeviceToHost));
        for (int64_t l = 0; l < m->nL; ++l) dinv[l] = fabs(dinv[l]);  // drop the owner sign
    }
    if (c) {
        float *tmp = (float *)malloc(sizeof(float) * m->nL);
        if (!tmp) return NB_ERR_OOM;
        cudaError_t e = cudaMemcpy(tmp, m->c32, sizeof(float) * m->nL, cudaMemcpyDeviceToHost);
        for (int64_t l = 0; e == cudaSuccess && l < m->nL; ++l) c[l] = tmp[l];
        free(tmp);
        NB_CUDA(e);
    }
    return NB_OK;
}

nb_status nb_to_local(nb_mesh *m, nb_prec prec, const void *ug, void *uL, int masked)
{
    NB_TRY(need_gs(m));
    if (!prec_ok(prec) || !ug || !uL) return arg_error("precision or NULL vector");
    NB_DEVICE_SCOPE(m->ctx->device);
    NB_TRY(to_local(m, prec, ug, uL, masked, m->ctx->stream));
    NB_CUDA(cudaStreamSynchronize(m->ctx->stream));
    return NB_OK;
}

nb_status nb_to_global(nb_mesh *m, nb_prec prec, const void *uL, void *ug)
{
    NB_TRY(need_gs(m));
    if (!prec_ok(prec) || !ug || !uL) return arg_error("precision or NULL vector");
    NB_DEVICE_SCOPE(m->ctx->device);
    NB_TRY(to_global(m, prec, uL, ug, m->ctx->stream));
    NB_CUDA(cudaStreamSynchronize(m->ctx->stream));
    return NB_OK;
}

nb_status nb_ax(nb_mesh *m, nb_prec prec, int assemble, const void *u, void *w)
{
    if (!m) return arg_error("mesh is NULL");
    if (!prec_ok(prec) || !u || !w) return arg_error("precision or NULL vector");
    if (u == w) return arg_error("u and w must not overlap");
    if (assemble) NB_TRY(need_gs(m));
    NB_DEVICE_SCOPE(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    NB_TRY(ax_local(m, prec, u, w, nullptr, nullptr, s));
    if (assemble) NB_TRY(dssum(m, prec, w, 1, s));
    NB_CUDA(cudaStreamSynchronize(s));
    return check_kernel_flag(m);
}

nb_status nb_dssum(nb_mesh *m, nb_prec prec, void *u, int masked)
{
    NB_TRY(need_gs(m));
    if (!prec_ok(prec) || !u) return arg_error("precision or NULL vector");
    NB_DEVICE_SCOPE(m->ctx->device);
    NB_TRY(dssum(m, prec, u, masked, m->ctx->stream));
    NB_CUDA(cudaStreamSynchronize(m->ctx->stream));
    return NB_OK;
}

nb_status nb_glsc3(nb_mesh *m, nb_prec prec, const void *a, const void *b, double *out)
{
    NB_TRY(need_gs(m));
    if (!prec_ok(prec) || !a || !b || !out) return arg_error("precision or NULL pointer");
    NB_DEVICE_SCOPE(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    if (!m->red_out) {
        NB_CUDA(cudaMalloc(&m->red_out, sizeof(double) * 8));
        NB_CUDA(cudaMallocHost(&m->red_host, sizeof(double) * 8));
    }
    if (!m->part64) NB_CUDA(cudaMalloc(&m->part64, sizeof(double) * kMaxPartials * 2));
    NB_TRY(glsc3_dev(m, prec, a, b, m->part64, m->red_out + 2, s));
    NB_CUDA(cudaMemcpyAsync(m->red_host + 2, m->red_out + 2, sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    *out = m->red_host[2];
    return NB_OK;
}

void nb_default_opts(nb_opts *o)
{
    if (!o) return;
    o->prec = NB_FP32;
    o->pc = NB_PC_JACOBI;
    o->rtol = 1e-10;
    o->maxiter = 10000;
    o->inner_rtol = 1e-4;
    o->max_outer = 30;
    o->use_graph = 1;
    o->record_history = 0;
    o->use_x0 = 0;
    o->restart = 0;
}

static nb_status check_opts(const nb_opts *o)
{
    if (!o) return arg_error("opts is NULL");
    if (!prec_ok(o->prec)) return arg_error("opts.prec");
    if (o->pc < NB_PC_NONE || o->pc > NB_PC_SCHWARZ2) return arg_error("opts.pc");
    if (!(o->rtol > 0.0) || !(o->rtol < 1.0)) return arg_error("opts.rtol must be in (0,1)");
    if (o->maxiter < 0) return arg_error("opts.maxiter");
    if (o->prec != NB_FP64 && (!(o->inner_rtol > 0.0) || !(o->inner_rtol < 1.0)))
        return arg_error("opts.inner_rtol must be in (0,1)");
    if (o->max_outer < 0) return arg_error("opts.max_outer");
    if (o->restart != 0 && o->restart != 1) return arg_error("opts.restart must be 0 or 1");
    if (o->pc == NB_PC_LEARNED && o->prec == NB_FP64)
        return arg_error("the learned preconditioner runs inside refinement (prec != NB_FP64)");
    if ((o->pc == NB_PC_SCHWARZ || o->pc == NB_PC_SCHWARZ2) && o->prec != NB_FP32)
        return arg_error("the Schwarz preconditioner runs inside FP32 refinement (prec = NB_FP32)");
    return NB_OK;
}

nb_status nb_solve(nb_mesh *m, const nb_opts *o, const double *b, double *x, nb_stats *st)
{
    NB_TRY(need_gs(m));
    NB_TRY(check_opts(o));
    if (!b || !x) return arg_error("NULL b or x");
    if (o->pc == NB_PC_LEARNED && !m->learned) {
        set_error("no learned preconditioner attached to this mesh");
        return NB_ERR_STATE;
    }
    NB_DEVICE_SCOPE(m->ctx->device);
    if (st) st->history_len = 0;
    nb_status r = solve(m, o, b, x, st);
    if (r < 0) return r;
    NB_TRY(check_kernel_flag(m));
    return r;
}

nb_status nb_solve_host(nb_mesh *m, const nb_opts *o, const double *bg, double *xg, nb_stats *st)
{
    NB_TRY(need_gs(m));
    NB_TRY(check_opts(o));
    if (!bg || !xg) return arg_error("NULL host vector");
    NB_DEVICE_SCOPE(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    if (!m->b64) {
        NB_CUDA(cudaMalloc(&m->b64, sizeof(double) * m->nL));
        NB_CUDA(cudaMalloc(&m->x64, sizeof(double) * m->nL));
    }
    if (!m->g64) NB_CUDA(cudaMalloc(&m->g64, sizeof(double) * m->nG));
    double *gbuf = m->g64;
    NB_CUDA(cudaMemcpyAsync(gbuf, bg, sizeof(double) * m->nG, cudaMemcpyHostToDevice, s));
    nb_status r = to_local(m, NB_FP64, gbuf, m->b64, 1, s);
    nb_opts o2 = *o;
    o2.use_x0 = 0;
    if (r >= 0) r = solve(m, &o2, m->b64, m->x64, st);
    if (r >= 0) {
        nb_status r2 = to_global(m, NB_FP64, m->x64, gbuf, s);
        if (r2 < 0) r = r2;
    }
    cudaError_t e = cudaSuccess;
    if (r >= 0) e = cudaMemcpyAsync(xg, gbuf, sizeof(double) * m->nG, cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        set_error("nb_solve_host: %s", cudaGetErrorString(e));
        return NB_ERR_CUDA;
    }
    return r;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// operator timing and autotuning
// ---------------------------------------------------------------------------

extern "C" int nb_ax_variants(const nb_mesh *m, nb_prec prec)
{
    if (!m || !prec_ok(prec)) return 0;
    return ax_variant_count(m, prec);
}

extern "C" nb_status nb_time_ax(nb_mesh *m, nb_prec prec, int cg_step, int variant, int reps,
                                void *flush_dev, size_t flush_bytes, double *ms_out)
{
    if (!m || !ms_out || reps < 1 || !prec_ok(prec)) return arg_error("mesh, prec, reps or out");
    if (variant >= ax_variant_count(m, prec)) return arg_error("variant index");
    if (cg_step) NB_TRY(need_gs(m));
    NB_DEVICE_SCOPE(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    Workspace &ws = prec == NB_FP64 ? m->ws64 : m->ws32;
    NB_TRY(ensure_ws(m, ws, prec == NB_FP64 ? 8 : 4, 0));
    const int saved = m->ax_cfg[prec].variant;
    if (variant >= 0) m->ax_cfg[prec].variant = variant;
    const void *dinv = prec == NB_FP64 ? (const void *)m->dinv64 : (const void *)m->dinv32;
    std::vector<cudaEvent_t> ev(2 * reps);
    nb_status st = NB_OK;
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) st = NB_ERR_CUDA;
    for (int r = 0; st == NB_OK && r < reps; ++r) {
        if (flush_dev && flush_bytes) {
            st = l2_flush(m->ctx, flush_dev, flush_bytes, r, s);
            if (st != NB_OK) break;
        }
        // beta = 0 and not done before every launch: the fused step's last
        // block may stop the scalars (pap <= 0 on arbitrary data), and a
        // stopped state would let the next launch return at once
        cudaMemsetAsync(ws.scal, 0, sizeof(CgScalars), s);
        cudaEventRecord(ev[2 * r], s);
        if (cg_step)
            st = ax_cg_step(m, prec, ws.r, dinv, ws.p, ws.w, ws.scal, ws.part, nullptr, s);
        else
            st = ax_local(m, prec, ws.p, ws.w, nullptr, nullptr, s);
        cudaEventRecord(ev[2 * r + 1], s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    double tot = 0.0;
    for (int r = 0; st == NB_OK && e == cudaSuccess && r < reps; ++r) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]);
        tot += ms;
    }
    for (auto &x : ev) cudaEventDestroy(x);
    m->ax_cfg[prec].variant = saved;
    if (st != NB_OK) return st;
    NB_CUDA(e);
    *ms_out = tot / reps;
    return NB_OK;
}

extern "C" const char *nb_ax_variant_name(const nb_mesh *m, nb_prec prec, int variant)
{
    if (!m || !prec_ok(prec)) return nullptr;
    if (variant == -1) variant = ax_variant_in_use(m, prec);
    return ax_variant_name(m, prec, variant);
}

extern "C" int nb_ax_variant_in_use(const nb_mesh *m, nb_prec prec)
{
    if (!m || !prec_ok(prec)) return -1;
    return ax_variant_in_use(m, prec);
}

extern "C" nb_status nb_slab_face(nb_mesh *m, nb_prec prec, int side, const void *u_dev,
                                  void *face_dev)
{
    NB_TRY(need_gs(m));
    if (!prec_ok(prec) || !u_dev || !face_dev) return arg_error("precision or NULL vector");
    NB_DEVICE_SCOPE(m->ctx->device);
    NB_TRY(slab_face(m, prec == NB_FP64 ? NB_FP64 : NB_FP32, side, u_dev, face_dev,
                     m->ctx->stream));
    NB_CUDA(cudaStreamSynchronize(m->ctx->stream));
    return NB_OK;
}

extern "C" nb_status nb_slab_face_add(nb_mesh *m, nb_prec prec, int side, void *u_dev,
                                      const void *face_dev)
{
    NB_TRY(need_gs(m));
    if (!prec_ok(prec) || !u_dev || !face_dev) return arg_error("precision or NULL vector");
    NB_DEVICE_SCOPE(m->ctx->device);
    NB_TRY(slab_face_add(m, prec == NB_FP64 ? NB_FP64 : NB_FP32, side, u_dev, face_dev,
                         m->ctx->stream));
    NB_CUDA(cudaStreamSynchronize(m->ctx->stream));
    return NB_OK;
}

extern "C" nb_status nb_slab_diag_face(nb_mesh *m, int side, double *face_dev)
{
    NB_TRY(need_gs(m));
    if (!face_dev) return arg_error("NULL face vector");
    NB_DEVICE_SCOPE(m->ctx->device);
    NB_TRY(slab_diag_face(m, side, face_dev, m->ctx->stream));
    NB_CUDA(cudaStreamSynchronize(m->ctx->stream));
    return NB_OK;
}

extern "C" nb_status nb_slab_finish_diag(nb_mesh *m, const double *face_lo_dev,
                                         const double *face_hi_dev)
{
    NB_TRY(need_gs(m));
    NB_DEVICE_SCOPE(m->ctx->device);
    return slab_finish_diag(m, face_lo_dev, face_hi_dev, m->ctx->stream);
}

extern "C" nb_status nb_cg_step(nb_mesh *m, nb_prec prec, double beta, const void *r_dev,
                                void *p_dev, void *w_dev, double *pap_host)
{
    NB_TRY(need_gs(m));
    if (!prec_ok(prec) || !r_dev || !p_dev || !w_dev || !pap_host)
        return arg_error("precision or NULL pointer");
    if (!isfinite(beta)) return arg_error("beta is not finite");
    NB_DEVICE_SCOPE(m->ctx->device);
    return split_step(m, prec, beta, r_dev, p_dev, w_dev, pap_host, m->ctx->stream);
}

extern "C" nb_status nb_cg_update(nb_mesh *m, nb_prec prec, double alpha, void *x_dev,
                                  void *r_dev, const void *p_dev, const void *w_dev,
                                  double *dots_host)
{
    NB_TRY(need_gs(m));
    if (!prec_ok(prec) || !x_dev || !r_dev || !p_dev || !w_dev || !dots_host)
        return arg_error("precision or NULL pointer");
    if (!isfinite(alpha)) return arg_error("alpha is not finite");
    NB_DEVICE_SCOPE(m->ctx->device);
    return split_update(m, prec == NB_FP64 ? NB_FP64 : NB_FP32, alpha, x_dev, r_dev, p_dev, w_dev,
                        dots_host, m->ctx->stream);
}

extern "C" nb_status nb_cg_dots(nb_mesh *m, nb_prec prec, const void *r_dev, double *dots_host)
{
    NB_TRY(need_gs(m));
    if (!prec_ok(prec) || !r_dev || !dots_host) return arg_error("precision or NULL pointer");
    NB_DEVICE_SCOPE(m->ctx->device);
    return split_dots(m, prec == NB_FP64 ? NB_FP64 : NB_FP32, r_dev, dots_host, m->ctx->stream);
}

extern "C" nb_status nb_set_update_variant(nb_mesh *m, int variant)
{
    if (!m || variant < 0 || variant > 3) return arg_error("mesh or update variant");
    if (m->update_kind != variant) {
        m->update_kind = variant;
        ++m->ax_epoch;  // captured iteration graphs hold the old kernel
    }
    return NB_OK;
}

extern "C" nb_status nb_set_x_deferral(nb_mesh *m, int mode)
{
    if (!m || mode < -1 || mode > 1) return arg_error("mesh or x deferral mode");
    if (m->x_defer != mode) {
        m->x_defer = mode;
        ++m->ax_epoch;  // captured iteration graphs hold the old form
    }
    return NB_OK;
}

extern "C" nb_status nb_set_ax_variant(nb_mesh *m, nb_prec prec, int variant)
{
    if (!m || !prec_ok(prec)) return arg_error("mesh or prec");
    if (variant < -1 || variant >= ax_variant_count(m, prec)) return arg_error("variant index");
    if (m->ax_cfg[prec].variant != variant) {
        m->ax_cfg[prec].variant = variant;
        ++m->ax_epoch;
    }
    return NB_OK;
}

extern "C" nb_status nb_autotune(nb_mesh *m, nb_prec prec, int reps, void *flush_dev,
                                 size_t flush_bytes, int *best_variant, double *best_ms)
{
    if (!m || !prec_ok(prec) || reps < 1) return arg_error("mesh, prec or reps");
    NB_TRY(need_gs(m));
    const int nv = ax_variant_count(m, prec);
    int best = 0;
    double bms = 1e300;
    for (int v = 0; v < nv; ++v) {
        double ms = 0.0;
        NB_TRY(nb_time_ax(m, prec, 1, v, 1, flush_dev, flush_bytes, &ms));  // warm-up
        NB_TRY(nb_time_ax(m, prec, 1, v, reps, flush_dev, flush_bytes, &ms));
        if (ms < bms) {
            bms = ms;
            best = v;
        }
    }
    if (m->ax_cfg[prec].variant != best) {
        m->ax_cfg[prec].variant = best;
        ++m->ax_epoch;
    }
    if (best_variant) *best_variant = best;
    if (best_ms) *best_ms = bms;
    return NB_OK;
}
