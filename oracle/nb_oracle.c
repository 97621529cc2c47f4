/*
 * Plain FP64 CPU oracle for the Nekbone-style spectral-element Poisson solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed CPU
 * baseline of the benchmark may load this library.  The CUDA library does not
 * link, include or call anything in this directory, and this file uses nothing
 * from it.
 *
 * The paper (Nekbone case study, Section 4.1 and Table 1) names the kernels of
 * the conjugate-gradient loop -- solveM, glsc3, add2s1, ax, add2s2 -- and
 * their order, but prints no formula of the discretisation.  Every step below
 * is therefore the textbook spectral-element definition that Nekbone
 * implements (Deville, Fischer and Mund, "High-Order Methods for
 * Incompressible Fluid Flow", 2002): Gauss-Lobatto-Legendre (GLL) points,
 * tensor-product Lagrange bases, the stiffness operator applied element by
 * element, and direct-stiffness summation.  All arithmetic is double
 * precision, loops run in the plain order written, and the file is compiled
 * with -ffp-contract=off so that no fused multiply-add changes the rounding.
 *
 * Layouts: an element-local ("L") vector holds E*n^3 values, n = N+1, indexed
 * [e][k][j][i] with i fastest.  Geometric factors are [e][6][n^3] in the order
 * (rr, rs, rt, ss, st, tt).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long long i64;

/* ------------------------------------------------------------------------ */
/* Legendre polynomials and GLL quadrature                                   */
/* ------------------------------------------------------------------------ */

/* P_N(x) and P_{N-1}(x) from Bonnet's recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},  P_0 = 1, P_1 = x. */
static void legendre_pair(int N, double x, double *pN, double *pNm1)
{
    double pm1 = 1.0, p = x;
    if (N == 0) { *pN = 1.0; *pNm1 = 0.0; return; }
    for (int k = 1; k < N; ++k) {
        double pp = ((2.0 * k + 1.0) * x * p - k * pm1) / (k + 1.0);
        pm1 = p;
        p = pp;
    }
    *pN = p;
    *pNm1 = pm1;
}

double nbo_legendre(int N, double x)
{
    double a, b;
    legendre_pair(N, x, &a, &b);
    return a;
}

/* GLL nodes xi[0..N] (ascending) and weights w[0..N].
 * The interior nodes are the zeros of P'_N.  Since
 * (1 - x^2) P'_N(x) = N (P_{N-1}(x) - x P_N(x)), they are the interior zeros of
 * q(x) = P_{N-1}(x) - x P_N(x), whose derivative is q'(x) = -(N+1) P_N(x).
 * Newton's method on q starts from the Chebyshev-Gauss-Lobatto points.
 * Weights: w_j = 2 / (N (N+1) P_N(xi_j)^2).  Returns 0, or -1 if N < 1. */
int nbo_gll(int N, double *xi, double *w)
{
    if (N < 1) return -1;
    const double pi = 3.14159265358979323846;
    xi[0] = -1.0;
    xi[N] = 1.0;
    for (int j = 1; j < N; ++j) {
        double x = -cos(pi * j / N);
        for (int it = 0; it < 100; ++it) {
            double pN, pNm1;
            legendre_pair(N, x, &pN, &pNm1);
            double q = pNm1 - x * pN;
            double dq = -(N + 1.0) * pN;
            double dx = q / dq;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        xi[j] = x;
    }
    /* symmetry of the point set: xi_{N-j} = -xi_j */
    for (int j = 0; j < (N + 1) / 2; ++j) {
        double s = 0.5 * (xi[N - j] - xi[j]);
        xi[j] = -s;
        xi[N - j] = s;
    }
    if (N % 2 == 0) xi[N / 2] = 0.0;
    for (int j = 0; j <= N; ++j) {
        double pN = nbo_legendre(N, xi[j]);
        w[j] = 2.0 / (N * (N + 1.0) * pN * pN);
    }
    return 0;
}

/* Derivative matrix of the GLL Lagrange basis: D[i*n + j] = l_j'(xi_i).
 *   i != j : P_N(xi_i) / (P_N(xi_j) (xi_i - xi_j))
 *   i = j = 0 : -N(N+1)/4,   i = j = N : N(N+1)/4,   otherwise 0. */
void nbo_deriv(int N, const double *xi, double *D)
{
    int n = N + 1;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            double v;
            if (i != j) {
                v = nbo_legendre(N, xi[i]) / (nbo_legendre(N, xi[j]) * (xi[i] - xi[j]));
            } else if (i == 0) {
                v = -0.25 * N * (N + 1.0);
            } else if (i == N) {
                v = 0.25 * N * (N + 1.0);
            } else {
                v = 0.0;
            }
            D[i * n + j] = v;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Box mesh: coordinates and geometric factors                               */
/* ------------------------------------------------------------------------ */

/* Coordinates of the n^3 nodes of element e of an nx*ny*nz box on the unit
 * cube.  Reference node (i,j,k) sits at
 *   X = (ex + (1+xi_i)/2)/nx,  Y = (ey + (1+xi_j)/2)/ny,  Z = (ez + (1+xi_k)/2)/nz
 * and is displaced by a*sin(pi X) sin(pi Y) sin(pi Z) in each of x, y, z, with
 * a = deform / max(nx,ny,nz).  The displacement vanishes on the boundary of
 * the cube, so the domain stays the unit cube.  Output X[3][n^3]. */
void nbo_element_coords(int nx, int ny, int nz, int N, double deform,
                        const double *xi, i64 e, double *X)
{
    const double pi = 3.14159265358979323846;
    int n = N + 1, n3 = n * n * n;
    i64 ex = e % nx, ey = (e / nx) % ny, ez = e / ((i64)nx * ny);
    int m = nx;
    if (ny > m) m = ny;
    if (nz > m) m = nz;
    double a = deform / m;
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double x0 = (ex + 0.5 * (1.0 + xi[i])) / nx;
                double y0 = (ey + 0.5 * (1.0 + xi[j])) / ny;
                double z0 = (ez + 0.5 * (1.0 + xi[k])) / nz;
                double d = a * sin(pi * x0) * sin(pi * y0) * sin(pi * z0);
                int q = (k * n + j) * n + i;
                X[0 * n3 + q] = x0 + d;
                X[1 * n3 + q] = y0 + d;
                X[2 * n3 + q] = z0 + d;
            }
}

/* Geometric factors of one element from its nodal coordinates X[3][n^3].
 * x_r = sum_l D[i][l] x(l,j,k), x_s = sum_l D[j][l] x(i,l,k),
 * x_t = sum_l D[k][l] x(i,j,l) (likewise y, z); J = det(dx/dr);
 * dr_a/dx_d is the inverse of the Jacobian matrix (cofactors over J);
 * G_ab = w_i w_j w_k J sum_d (dr_a/dx_d)(dr_b/dx_d).
 * Writes G[6][n^3] and, if jac is not NULL, J[n^3] and mass[n^3] = w w w J.
 * Returns the number of nodes where J <= 0. */
int nbo_element_geom(int N, const double *w, const double *D, const double *X,
                     double *G, double *jac, double *mass)
{
    int n = N + 1, n3 = n * n * n, bad = 0;
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                int q = (k * n + j) * n + i;
                double dr[3], ds[3], dt[3]; /* d(x,y,z)/dr, /ds, /dt */
                for (int c = 0; c < 3; ++c) {
                    const double *Xc = X + c * n3;
                    double sr = 0.0, ss = 0.0, st = 0.0;
                    for (int l = 0; l < n; ++l) {
                        sr += D[i * n + l] * Xc[(k * n + j) * n + l];
                        ss += D[j * n + l] * Xc[(k * n + l) * n + i];
                        st += D[k * n + l] * Xc[(l * n + j) * n + i];
                    }
                    dr[c] = sr;
                    ds[c] = ss;
                    dt[c] = st;
                }
                /* Jacobian matrix M[c][a] = dx_c / dr_a, columns (r,s,t) */
                double M[3][3] = {{dr[0], ds[0], dt[0]},
                                  {dr[1], ds[1], dt[1]},
                                  {dr[2], ds[2], dt[2]}};
                double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
                           - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
                           + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
                if (!(det > 0.0)) bad++;
                /* inverse: Minv[a][c] = dr_a / dx_c = cof(M)[c][a] / det */
                double Minv[3][3];
                Minv[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / det;
                Minv[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
                Minv[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
                Minv[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / det;
                Minv[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
                Minv[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
                Minv[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / det;
                Minv[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
                Minv[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
                double wq = w[i] * w[j] * w[k] * det;
                static const int A[6] = {0, 0, 0, 1, 1, 2};
                static const int B[6] = {0, 1, 2, 1, 2, 2};
                for (int c = 0; c < 6; ++c) {
                    double s = 0.0;
                    for (int d = 0; d < 3; ++d) s += Minv[A[c]][d] * Minv[B[c]][d];
                    G[c * n3 + q] = wq * s;
                }
                if (jac) jac[q] = det;
                if (mass) mass[q] = w[i] * w[j] * w[k] * det;
            }
    return bad;
}

/* Geometric factors for a list of elements: G[cnt][6][n^3].  Returns the
 * number of nodes with a non-positive Jacobian. */
i64 nbo_geom(int nx, int ny, int nz, int N, double deform, const i64 *elems,
             i64 cnt, double *G, double *mass)
{
    int n = N + 1, n3 = n * n * n;
    double xi[32], w[32], D[32 * 32];
    if (N < 1 || N > 31) return -1;
    nbo_gll(N, xi, w);
    nbo_deriv(N, xi, D);
    double *X = (double *)malloc(sizeof(double) * 3 * n3);
    i64 bad = 0;
    for (i64 t = 0; t < cnt; ++t) {
        nbo_element_coords(nx, ny, nz, N, deform, xi, elems[t], X);
        bad += nbo_element_geom(N, w, D, X, G + t * 6 * (i64)n3, NULL,
                                mass ? mass + t * (i64)n3 : NULL);
    }
    free(X);
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Global numbering, multiplicity, Dirichlet mask, CSR of local copies       */
/* ------------------------------------------------------------------------ */

/* Local node (e; i,j,k) is global node gx + (nx N + 1)(gy + (ny N + 1) gz)
 * with gx = ex N + i, gy = ey N + j, gz = ez N + k.  mult[g] counts the local
 * copies of g; mask[g] = 0 on the boundary of the box (homogeneous Dirichlet),
 * 1 elsewhere. */
void nbo_numbering(int nx, int ny, int nz, int N, i64 *gid, int *mult,
                   unsigned char *mask)
{
    int n = N + 1;
    i64 Gx = (i64)nx * N + 1, Gy = (i64)ny * N + 1, Gz = (i64)nz * N + 1;
    i64 E = (i64)nx * ny * nz, nG = Gx * Gy * Gz;
    for (i64 g = 0; g < nG; ++g) mult[g] = 0;
    for (i64 e = 0; e < E; ++e) {
        i64 ex = e % nx, ey = (e / nx) % ny, ez = e / ((i64)nx * ny);
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    i64 gx = ex * N + i, gy = ey * N + j, gz = ez * N + k;
                    i64 g = gx + Gx * (gy + Gy * gz);
                    gid[(e * n * n + (i64)k * n + j) * n + i] = g;
                    mult[g] += 1;
                }
    }
    for (i64 gz = 0; gz < Gz; ++gz)
        for (i64 gy = 0; gy < Gy; ++gy)
            for (i64 gx = 0; gx < Gx; ++gx) {
                int onb = gx == 0 || gx == Gx - 1 || gy == 0 || gy == Gy - 1 ||
                          gz == 0 || gz == Gz - 1;
                mask[gx + Gx * (gy + Gy * gz)] = onb ? 0 : 1;
            }
}

/* CSR of the local copies of every global node, copies in ascending local
 * index: locals[offsets[g] .. offsets[g+1]) are the l with gid[l] == g. */
void nbo_csr(i64 nL, i64 nG, const i64 *gid, i64 *offsets, i64 *locals)
{
    for (i64 g = 0; g <= nG; ++g) offsets[g] = 0;
    for (i64 l = 0; l < nL; ++l) offsets[gid[l] + 1] += 1;
    for (i64 g = 0; g < nG; ++g) offsets[g + 1] += offsets[g];
    i64 *fill = (i64 *)malloc(sizeof(i64) * (nG > 0 ? nG : 1));
    for (i64 g = 0; g < nG; ++g) fill[g] = offsets[g];
    for (i64 l = 0; l < nL; ++l) locals[fill[gid[l]]++] = l;
    free(fill);
}

/* ------------------------------------------------------------------------ */
/* The operator                                                              */
/* ------------------------------------------------------------------------ */

/* Local stiffness operator w = A_L u on cnt elements (ax_e of Nekbone,
 * Table 1 line 5; local_grad3, the geometric factors, local_grad3_t):
 *   ur = sum_l D[i][l] u(l,j,k),  us = sum_l D[j][l] u(i,l,k),
 *   ut = sum_l D[k][l] u(i,j,l);
 *   wr = Grr ur + Grs us + Grt ut,  ws = Grs ur + Gss us + Gst ut,
 *   wt = Grt ur + Gst us + Gtt ut;
 *   w(i,j,k) = sum_l D[l][i] wr(l,j,k) + D[l][j] ws(i,l,k) + D[l][k] wt(i,j,l). */
void nbo_ax_local(i64 cnt, int N, const double *D, const double *G,
                  const double *u, double *w)
{
    int n = N + 1, n3 = n * n * n;
    /* Elements are independent: with OpenMP each thread takes a fixed
     * contiguous range of them with its own scratch, so the result is the
     * same bit for bit whatever the number of threads. */
#pragma omp parallel
    {
    double *wr = (double *)malloc(sizeof(double) * 3 * n3);
    double *ws = wr + n3, *wt = wr + 2 * n3;
#pragma omp for schedule(static)
    for (i64 e = 0; e < cnt; ++e) {
        const double *ue = u + e * n3;
        const double *Ge = G + e * 6 * (i64)n3;
        double *we = w + e * n3;
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    double ur = 0.0, us = 0.0, ut = 0.0;
                    for (int l = 0; l < n; ++l) {
                        ur += D[i * n + l] * ue[(k * n + j) * n + l];
                        us += D[j * n + l] * ue[(k * n + l) * n + i];
                        ut += D[k * n + l] * ue[(l * n + j) * n + i];
                    }
                    int q = (k * n + j) * n + i;
                    double grr = Ge[0 * n3 + q], grs = Ge[1 * n3 + q], grt = Ge[2 * n3 + q];
                    double gss = Ge[3 * n3 + q], gst = Ge[4 * n3 + q], gtt = Ge[5 * n3 + q];
                    wr[q] = grr * ur + grs * us + grt * ut;
                    ws[q] = grs * ur + gss * us + gst * ut;
                    wt[q] = grt * ur + gst * us + gtt * ut;
                }
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    double s = 0.0;
                    for (int l = 0; l < n; ++l) s += D[l * n + i] * wr[(k * n + j) * n + l];
                    for (int l = 0; l < n; ++l) s += D[l * n + j] * ws[(k * n + l) * n + i];
                    for (int l = 0; l < n; ++l) s += D[l * n + k] * wt[(l * n + j) * n + i];
                    we[(k * n + j) * n + i] = s;
                }
    }
    free(wr);
    }
}

/* Diagonal of the local operator, per element and node (i,j,k):
 *   sum_l D[l][i]^2 Grr(l,j,k) + sum_l D[l][j]^2 Gss(i,l,k)
 *   + sum_l D[l][k]^2 Gtt(i,j,l) + 2 D[i][i] D[j][j] Grs(i,j,k)
 *   + 2 D[i][i] D[k][k] Grt(i,j,k) + 2 D[j][j] D[k][k] Gst(i,j,k). */
void nbo_diag_local(i64 cnt, int N, const double *D, const double *G, double *d)
{
    int n = N + 1, n3 = n * n * n;
    for (i64 e = 0; e < cnt; ++e) {
        const double *Ge = G + e * 6 * (i64)n3;
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    int q = (k * n + j) * n + i;
                    double s = 0.0;
                    for (int l = 0; l < n; ++l) s += D[l * n + i] * D[l * n + i] * Ge[0 * n3 + (k * n + j) * n + l];
                    for (int l = 0; l < n; ++l) s += D[l * n + j] * D[l * n + j] * Ge[3 * n3 + (k * n + l) * n + i];
                    for (int l = 0; l < n; ++l) s += D[l * n + k] * D[l * n + k] * Ge[5 * n3 + (l * n + j) * n + i];
                    s += 2.0 * D[i * n + i] * D[j * n + j] * Ge[1 * n3 + q];
                    s += 2.0 * D[i * n + i] * D[k * n + k] * Ge[2 * n3 + q];
                    s += 2.0 * D[j * n + j] * D[k * n + k] * Ge[4 * n3 + q];
                    d[e * n3 + q] = s;
                }
    }
}

/* Direct-stiffness summation followed by the Dirichlet mask: every local copy
 * of global node g receives mask[g] * (sum of the copies of g), the sum taken
 * in ascending local index.  work must hold nG doubles.  mask may be NULL. */
void nbo_dssum(i64 nL, i64 nG, const i64 *gid, const unsigned char *mask,
               double *u, double *work)
{
    for (i64 g = 0; g < nG; ++g) work[g] = 0.0;
    for (i64 l = 0; l < nL; ++l) work[gid[l]] += u[l];
    for (i64 l = 0; l < nL; ++l) {
        i64 g = gid[l];
        u[l] = (mask && !mask[g]) ? 0.0 : work[g];
    }
}

/* glsc3 (Table 1 lines 3, 6, 9): sum_l a_l b_l c_l in ascending l. */
double nbo_glsc3(const double *a, const double *b, const double *c, i64 n)
{
    double s = 0.0;
    for (i64 l = 0; l < n; ++l) s += a[l] * b[l] * c[l];
    return s;
}

/* ------------------------------------------------------------------------ */
/* Assembled operator and preconditioned CG                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    i64 E;              /* elements */
    int N;              /* order */
    i64 nL, nG;         /* local and global lengths */
    const double *D;    /* n*n */
    const double *G;    /* E*6*n^3 */
    const i64 *gid;     /* nL */
    const unsigned char *mask; /* nG */
    const double *c;    /* nL: 1/multiplicity */
    const double *dinv; /* nL: inverse assembled diagonal (0 where masked) or NULL */
    double *work;       /* nG scratch */
} nbo_op;

/* w = M Q Q^T A_L u: local operator, then dssum and mask. */
void nbo_apply(const nbo_op *op, const double *u, double *w)
{
    nbo_ax_local(op->E, op->N, op->D, op->G, u, w);
    nbo_dssum(op->nL, op->nG, op->gid, op->mask, w, op->work);
}

/* Preconditioned CG in the order of Table 1 (solveM, glsc3, add2s1, ax,
 * glsc3, add2s2 x2, glsc3).  x enters as the initial guess (L-vector,
 * continuous, masked); r = b - A x.  precond: 0 = identity (solveM as a copy,
 * the paper's no-multigrid case), 1 = Jacobi (z = dinv * r).
 * Stops when sqrt(rtr)/sqrt(glsc3(b,c,b)) < tol or after maxit iterations.
 * hist (may be NULL) receives the relative residual after each iteration.
 * Returns the number of iterations; *relres gets the last relative residual. */
int nbo_pcg(const nbo_op *op, const double *b, double *x, int maxit, double tol,
            int precond, double *hist, double *relres)
{
    i64 n = op->nL;
    double *r = (double *)malloc(sizeof(double) * 4 * n);
    double *z = r + n, *p = r + 2 * n, *w = r + 3 * n;
    nbo_apply(op, x, w);
    for (i64 l = 0; l < n; ++l) { r[l] = b[l] - w[l]; p[l] = 0.0; }
    double bnorm = sqrt(nbo_glsc3(b, op->c, b, n));
    if (bnorm == 0.0) bnorm = 1.0;
    double rtz1 = 1.0, rtz2, rel = sqrt(nbo_glsc3(r, op->c, r, n)) / bnorm;
    int iter = 0;
    for (iter = 1; iter <= maxit; ++iter) {
        if (precond == 1) {
            for (i64 l = 0; l < n; ++l) z[l] = op->dinv[l] * r[l];
        } else {
            for (i64 l = 0; l < n; ++l) z[l] = r[l];
        }
        rtz2 = rtz1;
        rtz1 = nbo_glsc3(r, op->c, z, n);
        double beta = (iter == 1) ? 0.0 : rtz1 / rtz2;
        for (i64 l = 0; l < n; ++l) p[l] = beta * p[l] + z[l];
        nbo_apply(op, p, w);
        double pap = nbo_glsc3(w, op->c, p, n);
        double alpha = rtz1 / pap;
        for (i64 l = 0; l < n; ++l) x[l] = x[l] + alpha * p[l];
        for (i64 l = 0; l < n; ++l) r[l] = r[l] - alpha * w[l];
        double rtr = nbo_glsc3(r, op->c, r, n);
        rel = sqrt(rtr) / bnorm;
        if (hist) hist[iter - 1] = rel;
        if (rel < tol) break;
    }
    if (iter > maxit) iter = maxit;
    free(r);
    if (relres) *relres = rel;
    return iter;
}

/* ------------------------------------------------------------------------ */
/* The same PCG on all host cores                                            */
/* ------------------------------------------------------------------------ */

/* Threads used by the OpenMP loops (nt > 0 sets it); returns the count in
 * force (1 when built without OpenMP). */
int nbo_threads(int nt)
{
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
    return omp_get_max_threads();
#else
    (void)nt;
    return 1;
#endif
}

/* Terms per fixed chunk of the parallel dot product. */
#define NBO_CHUNK 65536

/* glsc3 in fixed chunks of NBO_CHUNK consecutive terms: each chunk summed in
 * ascending index, the chunk sums then added in ascending chunk order.  The
 * chunking does not depend on the thread count, so neither does the result;
 * it differs from nbo_glsc3's single running sum by rounding order only. */
static double glsc3_chunked(const double *a, const double *b, const double *c, i64 n,
                            double *csum)
{
    const i64 nc = (n + NBO_CHUNK - 1) / NBO_CHUNK;
#pragma omp parallel for schedule(static)
    for (i64 q = 0; q < nc; ++q) {
        const i64 lo = q * NBO_CHUNK, hi = lo + NBO_CHUNK < n ? lo + NBO_CHUNK : n;
        double s = 0.0;
        for (i64 l = lo; l < hi; ++l) s += a[l] * b[l] * c[l];
        csum[q] = s;
    }
    double s = 0.0;
    for (i64 q = 0; q < nc; ++q) s += csum[q];
    return s;
}

/* dssum + mask over the CSR of copies (nbo_csr): each global node's copies
 * summed in ascending local index -- the order of nbo_dssum's scatter, so the
 * result is bit-identical to it -- and written back; nodes in parallel. */
static void dssum_csr(i64 nG, const i64 *off, const i64 *loc, const unsigned char *mask,
                      double *u)
{
#pragma omp parallel for schedule(static)
    for (i64 g = 0; g < nG; ++g) {
        double s = 0.0;
        for (i64 q = off[g]; q < off[g + 1]; ++q) s += u[loc[q]];
        if (mask && !mask[g]) s = 0.0;
        for (i64 q = off[g]; q < off[g + 1]; ++q) u[loc[q]] = s;
    }
}

/* nbo_pcg with its loops spread over the host cores: the element operator,
 * the per-node sums and the vector updates give the same bits as nbo_pcg's;
 * the three dot products use glsc3_chunked.  off/loc: the CSR of nbo_csr. */
int nbo_pcg_par(const nbo_op *op, const i64 *off, const i64 *loc, const double *b, double *x,
                int maxit, double tol, int precond, double *hist, double *relres)
{
    const i64 n = op->nL;
    double *r = (double *)malloc(sizeof(double) * 4 * n);
    double *z = r + n, *p = r + 2 * n, *w = r + 3 * n;
    double *csum = (double *)malloc(sizeof(double) * ((n + NBO_CHUNK - 1) / NBO_CHUNK + 1));
    nbo_ax_local(op->E, op->N, op->D, op->G, x, w);
    dssum_csr(op->nG, off, loc, op->mask, w);
#pragma omp parallel for schedule(static)
    for (i64 l = 0; l < n; ++l) {
        r[l] = b[l] - w[l];
        p[l] = 0.0;
    }
    double bnorm = sqrt(glsc3_chunked(b, op->c, b, n, csum));
    if (bnorm == 0.0) bnorm = 1.0;
    double rtz1 = 1.0, rtz2, rel = sqrt(glsc3_chunked(r, op->c, r, n, csum)) / bnorm;
    int iter = 0;
    for (iter = 1; iter <= maxit; ++iter) {
#pragma omp parallel for schedule(static)
        for (i64 l = 0; l < n; ++l) z[l] = precond == 1 ? op->dinv[l] * r[l] : r[l];
        rtz2 = rtz1;
        rtz1 = glsc3_chunked(r, op->c, z, n, csum);
        const double beta = iter == 1 ? 0.0 : rtz1 / rtz2;
#pragma omp parallel for schedule(static)
        for (i64 l = 0; l < n; ++l) p[l] = beta * p[l] + z[l];
        nbo_ax_local(op->E, op->N, op->D, op->G, p, w);
        dssum_csr(op->nG, off, loc, op->mask, w);
        const double pap = glsc3_chunked(w, op->c, p, n, csum);
        const double alpha = rtz1 / pap;
#pragma omp parallel for schedule(static)
        for (i64 l = 0; l < n; ++l) {
            x[l] = x[l] + alpha * p[l];
            r[l] = r[l] - alpha * w[l];
        }
        const double rtr = glsc3_chunked(r, op->c, r, n, csum);
        rel = sqrt(rtr) / bnorm;
        if (hist) hist[iter - 1] = rel;
        if (rel < tol) break;
    }
    if (iter > maxit) iter = maxit;
    free(csum);
    free(r);
    if (relres) *relres = rel;
    return iter;
}

/* ------------------------------------------------------------------------ */
/* Emulated reduced precision (Section 2, the VPREC backend; Section 4.2)    */
/* ------------------------------------------------------------------------ */

/* x rounded to a pseudo-mantissa of t bits (1 <= t <= 52): round to nearest,
 * ties to even, applied to the binary64 representation.  The exponent range
 * of binary64 is kept (no emulated range); a carry out of the mantissa raises
 * the exponent as the rounding of the real value requires, up to infinity.
 * NaN and infinities pass unchanged; t >= 52 is the identity. */
double nbo_vround(double x, int t)
{
    if (t >= 52) return x;
    if (t < 1) t = 1;
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    if (((b >> 52) & 0x7ff) == 0x7ff) return x;
    const int drop = 52 - t;
    const uint64_t mask = ((uint64_t)1 << drop) - 1, half = (uint64_t)1 << (drop - 1);
    const uint64_t rem = b & mask;
    b &= ~mask;
    if (rem > half || (rem == half && ((b >> drop) & 1))) b += (uint64_t)1 << drop;
    memcpy(&x, &b, sizeof x);
    return x;
}

/* Monte Carlo Arithmetic (Section 2, the MCA backend; Parker, 1997):
 * inexact(x) = x + 2^(e_x - t) xi with xi uniform on (-1/2, 1/2) and e_x the
 * exponent of x (2^(e_x - 1) <= |x| < 2^e_x); zero and non-finite values are
 * left alone.  Random rounding ("rr") perturbs the result of every operation,
 * full MCA ("mca") its operands and its result.  Random numbers: SplitMix64
 * (Steele, Lea and Flood, 2014), 53-bit uniforms, one stream per run. */
typedef struct {
    int mode;   /* 0: round to t bits (VPREC), 1: rr, 2: mca */
    int t;
    uint64_t s; /* SplitMix64 state */
} nbo_emu;

static double emu_u01(nbo_emu *m)
{
    uint64_t z = (m->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

double nbo_inexact(double x, int t, uint64_t *state)
{
    if (x == 0.0 || !isfinite(x)) return x;
    nbo_emu m = {1, t, *state};
    int e;
    frexp(x, &e);
    const double r = x + ldexp(emu_u01(&m) - 0.5, e - t);
    *state = m.s;
    return r;
}

static double emu_in(nbo_emu *m, double x)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(x, &e);
    return x + ldexp(emu_u01(m) - 0.5, e - m->t);
}

static double emu_out(nbo_emu *m, double r)
{
    return m->mode == 0 ? nbo_vround(r, m->t) : emu_in(m, r);
}

static double eadd(nbo_emu *m, double a, double b)
{
    if (m->mode == 2) { a = emu_in(m, a); b = emu_in(m, b); }
    return emu_out(m, a + b);
}
static double esub(nbo_emu *m, double a, double b)
{
    if (m->mode == 2) { a = emu_in(m, a); b = emu_in(m, b); }
    return emu_out(m, a - b);
}
static double emul(nbo_emu *m, double a, double b)
{
    if (m->mode == 2) { a = emu_in(m, a); b = emu_in(m, b); }
    return emu_out(m, a * b);
}
static double ediv(nbo_emu *m, double a, double b)
{
    if (m->mode == 2) { a = emu_in(m, a); b = emu_in(m, b); }
    return emu_out(m, a / b);
}

/* w = M Q Q^T A_L u with every +, -, *, / emulated, in the order of
 * nbo_ax_local and nbo_dssum (products and sums of each loop in turn). */
static void apply_emu(const nbo_op *op, nbo_emu *m, const double *u, double *w)
{
    const int N = op->N, n = N + 1, n3 = n * n * n;
    const double *D = op->D;
    double *wr = (double *)malloc(sizeof(double) * 3 * n3);
    double *ws = wr + n3, *wt = wr + 2 * n3;
    for (i64 e = 0; e < op->E; ++e) {
        const double *ue = u + e * n3;
        const double *Ge = op->G + e * 6 * (i64)n3;
        double *we = w + e * n3;
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    double ur = 0.0, us = 0.0, ut = 0.0;
                    for (int l = 0; l < n; ++l) {
                        ur = eadd(m, ur, emul(m, D[i * n + l], ue[(k * n + j) * n + l]));
                        us = eadd(m, us, emul(m, D[j * n + l], ue[(k * n + l) * n + i]));
                        ut = eadd(m, ut, emul(m, D[k * n + l], ue[(l * n + j) * n + i]));
                    }
                    const int q = (k * n + j) * n + i;
                    const double grr = Ge[0 * n3 + q], grs = Ge[1 * n3 + q], grt = Ge[2 * n3 + q];
                    const double gss = Ge[3 * n3 + q], gst = Ge[4 * n3 + q], gtt = Ge[5 * n3 + q];
                    wr[q] = eadd(m, eadd(m, emul(m, grr, ur), emul(m, grs, us)), emul(m, grt, ut));
                    ws[q] = eadd(m, eadd(m, emul(m, grs, ur), emul(m, gss, us)), emul(m, gst, ut));
                    wt[q] = eadd(m, eadd(m, emul(m, grt, ur), emul(m, gst, us)), emul(m, gtt, ut));
                }
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    double s = 0.0;
                    for (int l = 0; l < n; ++l) s = eadd(m, s, emul(m, D[l * n + i], wr[(k * n + j) * n + l]));
                    for (int l = 0; l < n; ++l) s = eadd(m, s, emul(m, D[l * n + j], ws[(k * n + l) * n + i]));
                    for (int l = 0; l < n; ++l) s = eadd(m, s, emul(m, D[l * n + k], wt[(l * n + j) * n + i]));
                    we[(k * n + j) * n + i] = s;
                }
    }
    free(wr);
    double *work = op->work;
    for (i64 g = 0; g < op->nG; ++g) work[g] = 0.0;
    for (i64 l = 0; l < op->nL; ++l) work[op->gid[l]] = eadd(m, work[op->gid[l]], w[l]);
    for (i64 l = 0; l < op->nL; ++l) {
        const i64 g = op->gid[l];
        w[l] = (op->mask && !op->mask[g]) ? 0.0 : work[g];
    }
}

static double glsc3_emu(nbo_emu *m, const double *a, const double *b, const double *c, i64 n)
{
    double s = 0.0;
    for (i64 l = 0; l < n; ++l) s = eadd(m, s, emul(m, emul(m, a[l], b[l]), c[l]));
    return s;
}

void nbo_apply_vprec(const nbo_op *op, int t, const double *u, double *w)
{
    nbo_emu m = {0, t, 0};
    apply_emu(op, &m, u, w);
}

/* glsc3 with every operation rounded: s = R(s + R(R(a b) c)), ascending l. */
double nbo_glsc3_vprec(const double *a, const double *b, const double *c, i64 n, int t)
{
    nbo_emu m = {0, t, 0};
    return glsc3_emu(&m, a, b, c, n);
}

/* The CG loop of nbo_pcg with every +, -, *, / of the loop emulated
 * (mode 0: rounded to t bits; 1: random rounding; 2: full MCA, virtual
 * precision t; seed: the run's SplitMix64 seed) -- the paper's "only CG"
 * instrumentation: set-up (geometry, the Jacobi diagonal, the initial
 * residual and |b|) stays in binary64; sqrt is not an arithmetic operation.
 * Runs exactly `iters` iterations (Nekbone's fixed iteration count); hist
 * (may be NULL) receives the loop's relative residual sqrt(rtr)/|b| after
 * each.  Returns the last one. */
double nbo_cg_emu(const nbo_op *op, const double *b, double *x, int iters, int mode, int t,
                  uint64_t seed, int precond, double *hist)
{
    nbo_emu m = {mode, t, seed};
    const i64 n = op->nL;
    double *r = (double *)malloc(sizeof(double) * 4 * n);
    double *z = r + n, *p = r + 2 * n, *w = r + 3 * n;
    nbo_apply(op, x, w);
    for (i64 l = 0; l < n; ++l) {
        r[l] = b[l] - w[l];
        p[l] = 0.0;
    }
    double bnorm = sqrt(nbo_glsc3(b, op->c, b, n));
    if (bnorm == 0.0) bnorm = 1.0;
    double rtz1 = 1.0, rtz2, rel = sqrt(nbo_glsc3(r, op->c, r, n)) / bnorm;
    for (int it = 1; it <= iters; ++it) {
        if (precond == 1) {
            for (i64 l = 0; l < n; ++l) z[l] = emul(&m, op->dinv[l], r[l]);
        } else {
            for (i64 l = 0; l < n; ++l) z[l] = r[l];
        }
        rtz2 = rtz1;
        rtz1 = glsc3_emu(&m, r, op->c, z, n);
        const double beta = (it == 1) ? 0.0 : ediv(&m, rtz1, rtz2);
        for (i64 l = 0; l < n; ++l) p[l] = eadd(&m, emul(&m, beta, p[l]), z[l]);
        apply_emu(op, &m, p, w);
        const double pap = glsc3_emu(&m, w, op->c, p, n);
        const double alpha = ediv(&m, rtz1, pap);
        for (i64 l = 0; l < n; ++l) x[l] = eadd(&m, x[l], emul(&m, alpha, p[l]));
        for (i64 l = 0; l < n; ++l) r[l] = esub(&m, r[l], emul(&m, alpha, w[l]));
        const double rtr = glsc3_emu(&m, r, op->c, r, n);
        rel = ediv(&m, sqrt(rtr), bnorm);
        if (hist) hist[it - 1] = rel;
    }
    free(r);
    return rel;
}

double nbo_cg_vprec(const nbo_op *op, const double *b, double *x, int iters, int t,
                    int precond, double *hist)
{
    return nbo_cg_emu(op, b, x, iters, 0, t, 0, precond, hist);
}


