// Slab partition of the box along z: the interface planes between slabs.
//
// A slab mesh (nb_setup_slab) holds the elements z0 <= ez < z1 of the box
// with the box's geometry; the node planes it shares with the slab below and
// the slab above are free (not Dirichlet).  The direct-stiffness summation of
// the whole box is then, per slab, the summation over the slab's own copies
// (nb_dssum) plus, on each interface plane, the neighbouring slab's sum over
// its copies: slab_face packs a slab's sums on one of its interface planes
// into a plane vector [gy][gx] of (nx N + 1)(ny N + 1) values, slab_face_add
// adds a received plane vector to every copy of its free nodes.  This is the
// face exchange of Nekbone's gather-scatter between MPI ranks (Section 4.1:
// dssum is the "accumulations before and after" of ax), laid out for one
// message per interface.
#include <math.h>

#include <algorithm>

#include "nb_reduce.cuh"

namespace nb {

// The (up to two) element / point pairs along one direction that hold global
// line index g: element (g - 1) / N at point N and element g / N at point 0
// when g is an interior element boundary, else the one element holding g.
__device__ __forceinline__ int line_copies(int g, int N, int ne, int el[2], int pt[2])
{
    if (g % N == 0) {
        int c = 0;
        if (g > 0) {
            el[c] = g / N - 1;
            pt[c] = N;
            ++c;
        }
        if (g < ne * N) {
            el[c] = g / N;
            pt[c] = 0;
            ++c;
        }
        return c;
    }
    el[0] = g / N;
    pt[0] = g % N;
    return 1;
}

// face[gx + Gx gy] = sum of u over the slab's copies of plane node (gx, gy)
// of the element layer ez (k = N for the upper plane, 0 for the lower), in
// ascending local index.
template <typename T>
__global__ void k_slab_face(int nx, int ny, int N, int ez, int k, const T *__restrict__ u,
                            T *__restrict__ face)
{
    const int n = N + 1, n3 = n * n * n, Gx = nx * N + 1, Gy = ny * N + 1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Gx * Gy; t += gridDim.x * blockDim.x) {
        const int gx = t % Gx, gy = t / Gx;
        int ex[2], ix[2], ey[2], jy[2];
        const int cx = line_copies(gx, N, nx, ex, ix), cy = line_copies(gy, N, ny, ey, jy);
        T s = T(0);
        for (int b = 0; b < cy; ++b)
            for (int a = 0; a < cx; ++a) {
                const int64_t e = (int64_t)ex[a] + (int64_t)nx * (ey[b] + (int64_t)ny * ez);
                s += u[e * n3 + ((int64_t)k * n + jy[b]) * n + ix[a]];
            }
        face[t] = s;
    }
}

// u += face on every copy of the free nodes of the plane (nodes on the box's
// x / y boundary are Dirichlet and stay as they are).
template <typename T>
__global__ void k_slab_face_add(int nx, int ny, int N, int ez, int k, T *__restrict__ u,
                                const T *__restrict__ face)
{
    const int n = N + 1, n3 = n * n * n, Gx = nx * N + 1, Gy = ny * N + 1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Gx * Gy; t += gridDim.x * blockDim.x) {
        const int gx = t % Gx, gy = t / Gx;
        if (gx == 0 || gx == Gx - 1 || gy == 0 || gy == Gy - 1) continue;
        int ex[2], ix[2], ey[2], jy[2];
        const int cx = line_copies(gx, N, nx, ex, ix), cy = line_copies(gy, N, ny, ey, jy);
        const T v = face[t];
        for (int b = 0; b < cy; ++b)
            for (int a = 0; a < cx; ++a) {
                const int64_t e = (int64_t)ex[a] + (int64_t)nx * (ey[b] + (int64_t)ny * ez);
                u[e * n3 + ((int64_t)k * n + jy[b]) * n + ix[a]] += v;
            }
    }
}

static bool side_ok(const nb_mesh *m, int side)
{
    return (side == 0 && m->iface_lo) || (side == 1 && m->iface_hi);
}

nb_status slab_face(nb_mesh *m, nb_prec prec, int side, const void *u, void *face, cudaStream_t s)
{
    if (!side_ok(m, side)) {
        set_error("the mesh has no interface plane on side %d", side);
        return NB_ERR_ARG;
    }
    const int ez = side == 0 ? 0 : m->nz - 1, k = side == 0 ? 0 : m->N;
    const int64_t np = ((int64_t)m->nx * m->N + 1) * ((int64_t)m->ny * m->N + 1);
    const int grid = (int)std::min<int64_t>((np + 255) / 256, (int64_t)m->ctx->sm_count * 8);
    if (prec == NB_FP64)
        k_slab_face<double><<<grid, 256, 0, s>>>(m->nx, m->ny, m->N, ez, k, (const double *)u,
                                                 (double *)face);
    else
        k_slab_face<float><<<grid, 256, 0, s>>>(m->nx, m->ny, m->N, ez, k, (const float *)u,
                                                (float *)face);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

nb_status slab_face_add(nb_mesh *m, nb_prec prec, int side, void *u, const void *face,
                        cudaStream_t s)
{
    if (!side_ok(m, side)) {
        set_error("the mesh has no interface plane on side %d", side);
        return NB_ERR_ARG;
    }
    const int ez = side == 0 ? 0 : m->nz - 1, k = side == 0 ? 0 : m->N;
    const int64_t np = ((int64_t)m->nx * m->N + 1) * ((int64_t)m->ny * m->N + 1);
    const int grid = (int)std::min<int64_t>((np + 255) / 256, (int64_t)m->ctx->sm_count * 8);
    if (prec == NB_FP64)
        k_slab_face_add<double><<<grid, 256, 0, s>>>(m->nx, m->ny, m->N, ez, k, (double *)u,
                                                     (const double *)face);
    else
        k_slab_face_add<float><<<grid, 256, 0, s>>>(m->nx, m->ny, m->N, ez, k, (float *)u,
                                                    (const float *)face);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// The slab's own (assembled, unmasked over its copies) diagonal on an
// interface plane: the diagonal of the slab-local assembly is the same value
// on every copy, so the plane vector takes one copy per node.
template <typename T>
__global__ void k_slab_diag_face(int nx, int ny, int N, int ez, int k, const T *__restrict__ d,
                                 T *__restrict__ face)
{
    const int n = N + 1, n3 = n * n * n, Gx = nx * N + 1, Gy = ny * N + 1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Gx * Gy; t += gridDim.x * blockDim.x) {
        const int gx = t % Gx, gy = t / Gx;
        int ex[2], ix[2], ey[2], jy[2];
        line_copies(gx, N, nx, ex, ix);
        line_copies(gy, N, ny, ey, jy);
        const int64_t e = (int64_t)ex[0] + (int64_t)nx * (ey[0] + (int64_t)ny * ez);
        face[t] = d[e * n3 + ((int64_t)k * n + jy[0]) * n + ix[0]];
    }
}

nb_status slab_diag_face(nb_mesh *m, int side, double *face, cudaStream_t s)
{
    if (!side_ok(m, side) || !m->diag_asm) {
        set_error("the mesh has no interface plane on side %d (or no gather-scatter)", side);
        return NB_ERR_ARG;
    }
    const int ez = side == 0 ? 0 : m->nz - 1, k = side == 0 ? 0 : m->N;
    const int64_t np = ((int64_t)m->nx * m->N + 1) * ((int64_t)m->ny * m->N + 1);
    const int grid = (int)std::min<int64_t>((np + 255) / 256, (int64_t)m->ctx->sm_count * 8);
    k_slab_diag_face<double><<<grid, 256, 0, s>>>(m->nx, m->ny, m->N, ez, k, m->diag_asm, face);
    NB_CUDA(cudaGetLastError());
    return NB_OK;
}

// The diagonal of the whole box on the slab: its own part plus the
// neighbours' parts on the interface planes (face_lo / face_hi, NULL where
// there is no neighbour), then the Jacobi inverse with the mask and owners.
nb_status finish_jacobi(nb_mesh *m, double *diag, cudaStream_t s);

nb_status slab_finish_diag(nb_mesh *m, const double *face_lo, const double *face_hi,
                           cudaStream_t s)
{
    if (!m->diag_asm) {
        set_error("not a slab with interfaces, or nb_setup_gs not done");
        return NB_ERR_STATE;
    }
    if ((face_lo != nullptr) != m->iface_lo || (face_hi != nullptr) != m->iface_hi) {
        set_error("a neighbour's diagonal is needed exactly on the interface sides");
        return NB_ERR_ARG;
    }
    double *d = nullptr;
    NB_CUDA(cudaMalloc(&d, sizeof(double) * m->nL));
    nb_status st = NB_OK;
    if (cudaMemcpyAsync(d, m->diag_asm, sizeof(double) * m->nL, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        st = NB_ERR_CUDA;
    if (st == NB_OK && face_lo) st = slab_face_add(m, NB_FP64, 0, d, face_lo, s);
    if (st == NB_OK && face_hi) st = slab_face_add(m, NB_FP64, 1, d, face_hi, s);
    if (st == NB_OK) st = finish_jacobi(m, d, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (st == NB_OK && e != cudaSuccess) {
        set_error("slab diagonal: %s", cudaGetErrorString(e));
        st = NB_ERR_CUDA;
    }
    return st;
}

}  // namespace nb
