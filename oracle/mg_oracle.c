/*
 * FP64 CPU oracle for the variable-coefficient pressure Poisson solve
 *        -div( (1/rho) grad p ) = b
 * on a uniform cell-centred grid with homogeneous Neumann walls, solved by a
 * geometric multigrid V-cycle (red-black Gauss-Seidel, residual, 8:1
 * restriction, prolongation, face-coefficient coarsening, dense coarse solve).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * restatement that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product never does.  It shares no code with the CUDA library.
 *
 * Where the method comes from.  The paper (FS3D, §2) solves the incompressible
 * Navier-Stokes equations, Eq. (1) div u = 0 and Eq. (2) with the pressure
 * force -grad p / rho per unit mass; a projection step then needs the Poisson
 * equation above, and §4.3.2 names multigrid as the pressure solver.  Density
 * is volume weighted per Eq. (5).  The paper writes down neither the
 * discretisation nor the multigrid cycle, so this file states each of them as
 * a plain definition:
 *
 *  - grid: cell (i,j,k), i fastest, index (k*ny + j)*nx + i, spacing h.
 *  - faces: bx has shape (nz, ny, nx+1), face i between cells i-1 and i;
 *    by (nz, ny+1, nx); bz (nz+1, ny, nx).  Faces 0 and n of each axis are
 *    walls: their values are never read (zero flux, homogeneous Neumann).
 *  - face coefficient: beta_f = 1 / harmonic_mean(rho_L, rho_R).
 *  - operator: (A p)_c = (1/h^2) sum_{interior faces f of c} beta_f (p_c - p_nb(f)),
 *    i.e. A = -D diag(beta) G with G_f p = (p_R - p_L)/h, (D u)_c = sum +-u_f/h.
 *    A is symmetric positive semidefinite with null space = constants.
 *  - gauge: the solution is the zero-mean p solving A p = b - mean(b).
 *  - red-black Gauss-Seidel: red = (i+j+k) even.  A half sweep replaces every
 *    cell of one colour by the exact solution of its own row,
 *        p_c = (h^2 b_c + sum_f beta_f p_nb) / sum_f beta_f,
 *    summed in the order x-, x+, y-, y+, z-, z+.  Pre-smoothing sweeps go red
 *    then black, post-smoothing sweeps black then red.
 *  - restriction: coarse value = mean of the 8 children.
 *  - prolongation: cell-centred trilinear (1D weights 3/4 parent, 1/4 the
 *    parent's neighbour on the fine cell's side; a missing neighbour at a wall
 *    is replaced by the parent), or piecewise constant.
 *  - face coarsening: a coarse face takes the mean of the 4 fine faces that
 *    tile it; the coarse operator uses the same formula with spacing 2h.
 *  - levels: halve every dimension while all are even and the largest
 *    exceeds `coarsest`; the last level is solved densely.
 *  - coarse solve: e = A_c^+ (r - mean r), computed as the solution of
 *    (A_c + c 1 1^T) e = r - mean(r), c = mean(diag A_c)/n_c > 0, by Cholesky.
 *  - adjoint: for L = sum w p, lambda = A^+ (w - mean w) = dL/db and
 *    dL/dbeta_f = -(lambda_L - lambda_R)(p_L - p_R)/h^2, plus, when the RHS
 *    carries sigma * D(beta * csf), the terms sigma csf_f (lambda_L -
 *    lambda_R)/h, and dL/dsigma = sum_f beta_f csf_f (lambda_L - lambda_R)/h.
 *
 * Reductions are summed per z-plane and then over planes in order, so every
 * result is the same at any OpenMP thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_NOT_CONVERGED (-3)
#define OR_ERR_DIVERGED (-4)
#define OR_ERR_OOM (-6)

#define OR_MAX_LEVELS 24
#define OR_MAX_COARSE 4096

typedef long long idx_t;

/* ---- indexing ---------------------------------------------------------- */
#define CELL(i, j, k) (((idx_t)(k) * ny + (j)) * nx + (i))
#define FXI(i, j, k) (((idx_t)(k) * ny + (j)) * (nx + 1) + (i))
#define FYI(i, j, k) (((idx_t)(k) * (ny + 1) + (j)) * nx + (i))
#define FZI(i, j, k) (((idx_t)(k) * ny + (j)) * nx + (i))

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---- deterministic sums ------------------------------------------------ */
/* sum over all cells of x (and of x^2): per-plane partials, then planes in order */
static void plane_sums(int nx, int ny, int nz, const double *x, double *sum, double *sumsq) {
    double *ps = (double *)calloc((size_t)nz, sizeof(double));
    double *pq = (double *)calloc((size_t)nz, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        double s = 0.0, q = 0.0;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double v = x[CELL(i, j, k)];
                s += v;
                q += v * v;
            }
        ps[k] = s;
        pq[k] = q;
    }
    double s = 0.0, q = 0.0;
    for (int k = 0; k < nz; ++k) {
        s += ps[k];
        q += pq[k];
    }
    if (sum) *sum = s;
    if (sumsq) *sumsq = q;
    free(ps);
    free(pq);
}

double or_mean(int nx, int ny, int nz, const double *x) {
    double s;
    plane_sums(nx, ny, nz, x, &s, NULL);
    return s / ((double)nx * ny * nz);
}

double or_norm2(int nx, int ny, int nz, const double *x) {
    double q;
    plane_sums(nx, ny, nz, x, NULL, &q);
    return sqrt(q);
}

static void add_const(int nx, int ny, int nz, double *x, double c) {
    idx_t n = (idx_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (idx_t m = 0; m < n; ++m) x[m] += c;
}

/* ---- Eq. (5): volume-weighted density ---------------------------------- */
/* rho = sum_{i<nfrac} rho_i f_i + rho_last (1 - sum_{i<nfrac} f_i):
 * the last phase fills what the listed fractions leave. */
void or_density(idx_t ncell, int nfrac, const double *const *frac, const double *rho_phase,
                double *rho) {
#pragma omp parallel for schedule(static)
    for (idx_t m = 0; m < ncell; ++m) {
        double rest = 1.0, r = 0.0;
        for (int q = 0; q < nfrac; ++q) {
            r += rho_phase[q] * frac[q][m];
            rest -= frac[q][m];
        }
        rho[m] = r + rho_phase[nfrac] * rest;
    }
}

/* ---- face coefficients: 1 / harmonic mean of the two cell densities ---- */
static double inv_harmonic(double a, double b) {
    double hm = 2.0 * a * b / (a + b);
    return 1.0 / hm;
}

void or_faces_from_density(int nx, int ny, int nz, const double *rho, double *bx, double *by,
                           double *bz) {
    memset(bx, 0, sizeof(double) * (size_t)nz * ny * (nx + 1));
    memset(by, 0, sizeof(double) * (size_t)nz * (ny + 1) * nx);
    memset(bz, 0, sizeof(double) * (size_t)(nz + 1) * ny * nx);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double rc = rho[CELL(i, j, k)];
                if (i > 0) bx[FXI(i, j, k)] = inv_harmonic(rho[CELL(i - 1, j, k)], rc);
                if (j > 0) by[FYI(i, j, k)] = inv_harmonic(rho[CELL(i, j - 1, k)], rc);
                if (k > 0) bz[FZI(i, j, k)] = inv_harmonic(rho[CELL(i, j, k - 1)], rc);
            }
}

/* ---- the operator -------------------------------------------------------- */
/* out = A p, (A p)_c = (1/h^2) sum_f beta_f (p_c - p_nb), interior faces only */
void or_apply(int nx, int ny, int nz, double h, const double *bx, const double *by,
              const double *bz, const double *p, double *out) {
    double ih2 = 1.0 / (h * h);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double pc = p[CELL(i, j, k)];
                double s = 0.0;
                if (i > 0) s += bx[FXI(i, j, k)] * (pc - p[CELL(i - 1, j, k)]);
                if (i < nx - 1) s += bx[FXI(i + 1, j, k)] * (pc - p[CELL(i + 1, j, k)]);
                if (j > 0) s += by[FYI(i, j, k)] * (pc - p[CELL(i, j - 1, k)]);
                if (j < ny - 1) s += by[FYI(i, j + 1, k)] * (pc - p[CELL(i, j + 1, k)]);
                if (k > 0) s += bz[FZI(i, j, k)] * (pc - p[CELL(i, j, k - 1)]);
                if (k < nz - 1) s += bz[FZI(i, j, k + 1)] * (pc - p[CELL(i, j, k + 1)]);
                out[CELL(i, j, k)] = s * ih2;
            }
}

/* r = b - A p */
void or_residual(int nx, int ny, int nz, double h, const double *bx, const double *by,
                 const double *bz, const double *b, const double *p, double *r) {
    or_apply(nx, ny, nz, h, bx, by, bz, p, r);
    idx_t n = (idx_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (idx_t m = 0; m < n; ++m) r[m] = b[m] - r[m];
}

/* ---- divergence and RHS assembly ----------------------------------------- */
/* (D u)_c = sum over the interior faces of c of (+u on the high face, -u on the
 * low face) / h; wall faces carry no flux. */
void or_divergence(int nx, int ny, int nz, double h, const double *ux, const double *uy,
                   const double *uz, double *out) {
    double ih = 1.0 / h;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double s = 0.0;
                if (i > 0) s -= ux[FXI(i, j, k)];
                if (i < nx - 1) s += ux[FXI(i + 1, j, k)];
                if (j > 0) s -= uy[FYI(i, j, k)];
                if (j < ny - 1) s += uy[FYI(i, j + 1, k)];
                if (k > 0) s -= uz[FZI(i, j, k)];
                if (k < nz - 1) s += uz[FZI(i, j, k + 1)];
                out[CELL(i, j, k)] = s * ih;
            }
}

/* CSF face quantity csf_f = kappa_f (f_R - f_L) / h, kappa_f = (kappa_L + kappa_R)/2,
 * on interior faces; walls 0. */
void or_csf_faces(int nx, int ny, int nz, double h, const double *f, const double *kappa,
                  double *cx, double *cy, double *cz) {
    memset(cx, 0, sizeof(double) * (size_t)nz * ny * (nx + 1));
    memset(cy, 0, sizeof(double) * (size_t)nz * (ny + 1) * nx);
    memset(cz, 0, sizeof(double) * (size_t)(nz + 1) * ny * nx);
    double ih = 1.0 / h;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                idx_t c = CELL(i, j, k);
                if (i > 0) {
                    idx_t l = CELL(i - 1, j, k);
                    cx[FXI(i, j, k)] = 0.5 * (kappa[l] + kappa[c]) * (f[c] - f[l]) * ih;
                }
                if (j > 0) {
                    idx_t l = CELL(i, j - 1, k);
                    cy[FYI(i, j, k)] = 0.5 * (kappa[l] + kappa[c]) * (f[c] - f[l]) * ih;
                }
                if (k > 0) {
                    idx_t l = CELL(i, j, k - 1);
                    cz[FZI(i, j, k)] = 0.5 * (kappa[l] + kappa[c]) * (f[c] - f[l]) * ih;
                }
            }
}

/* b = D u + sigma D(beta * csf)   (csf pointers may be NULL: no surface term) */
void or_rhs(int nx, int ny, int nz, double h, const double *ux, const double *uy,
            const double *uz, const double *bx, const double *by, const double *bz,
            const double *csfx, const double *csfy, const double *csfz, double sigma,
            double *b) {
    or_divergence(nx, ny, nz, h, ux, uy, uz, b);
    if (!csfx) return;
    size_t nfx = (size_t)nz * ny * (nx + 1), nfy = (size_t)nz * (ny + 1) * nx,
           nfz = (size_t)(nz + 1) * ny * nx;
    double *tx = (double *)malloc(sizeof(double) * nfx);
    double *ty = (double *)malloc(sizeof(double) * nfy);
    double *tz = (double *)malloc(sizeof(double) * nfz);
    double *bs = (double *)malloc(sizeof(double) * (size_t)nx * ny * nz);
    for (size_t m = 0; m < nfx; ++m) tx[m] = bx[m] * csfx[m];
    for (size_t m = 0; m < nfy; ++m) ty[m] = by[m] * csfy[m];
    for (size_t m = 0; m < nfz; ++m) tz[m] = bz[m] * csfz[m];
    or_divergence(nx, ny, nz, h, tx, ty, tz, bs);
    idx_t n = (idx_t)nx * ny * nz;
    for (idx_t m = 0; m < n; ++m) b[m] += sigma * bs[m];
    free(tx);
    free(ty);
    free(tz);
    free(bs);
}

/* ---- red-black Gauss-Seidel ---------------------------------------------- */
/* One half sweep over the cells of one colour ((i+j+k) % 2 == colour). */
void or_rbgs_half(int nx, int ny, int nz, double h, const double *bx, const double *by,
                  const double *bz, const double *b, double *p, int colour) {
    double h2 = h * h;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = (colour + j + k) & 1; i < nx; i += 2) {
                double num = 0.0, den = 0.0, bf;
                if (i > 0) {
                    bf = bx[FXI(i, j, k)];
                    num += bf * p[CELL(i - 1, j, k)];
                    den += bf;
                }
                if (i < nx - 1) {
                    bf = bx[FXI(i + 1, j, k)];
                    num += bf * p[CELL(i + 1, j, k)];
                    den += bf;
                }
                if (j > 0) {
                    bf = by[FYI(i, j, k)];
                    num += bf * p[CELL(i, j - 1, k)];
                    den += bf;
                }
                if (j < ny - 1) {
                    bf = by[FYI(i, j + 1, k)];
                    num += bf * p[CELL(i, j + 1, k)];
                    den += bf;
                }
                if (k > 0) {
                    bf = bz[FZI(i, j, k)];
                    num += bf * p[CELL(i, j, k - 1)];
                    den += bf;
                }
                if (k < nz - 1) {
                    bf = bz[FZI(i, j, k + 1)];
                    num += bf * p[CELL(i, j, k + 1)];
                    den += bf;
                }
                p[CELL(i, j, k)] = (h2 * b[CELL(i, j, k)] + num) / den;
            }
}

/* `sweeps` full sweeps; order 0 = red then black (pre), 1 = black then red (post) */
void or_rbgs(int nx, int ny, int nz, double h, const double *bx, const double *by,
             const double *bz, const double *b, double *p, int sweeps, int order) {
    for (int s = 0; s < sweeps; ++s) {
        or_rbgs_half(nx, ny, nz, h, bx, by, bz, b, p, order ? 1 : 0);
        or_rbgs_half(nx, ny, nz, h, bx, by, bz, b, p, order ? 0 : 1);
    }
}

/* ---- grid transfers ------------------------------------------------------ */
/* coarse (nx/2, ny/2, nz/2) value = mean of its 8 children */
void or_restrict(int nx, int ny, int nz, const double *r, double *rc) {
    int cnx = nx / 2, cny = ny / 2, cnz = nz / 2;
#pragma omp parallel for schedule(static)
    for (int K = 0; K < cnz; ++K)
        for (int J = 0; J < cny; ++J)
            for (int I = 0; I < cnx; ++I) {
                double s = 0.0;
                for (int c = 0; c < 2; ++c)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a) s += r[CELL(2 * I + a, 2 * J + b, 2 * K + c)];
                rc[((idx_t)K * cny + J) * cnx + I] = s / 8.0;
            }
}

/* e (fine, 2*cnx x 2*cny x 2*cnz) += P ec; kind 0 = trilinear, 1 = constant */
void or_prolong_correct(int cnx, int cny, int cnz, const double *ec, double *e, int kind) {
    int nx = 2 * cnx, ny = 2 * cny, nz = 2 * cnz;
#define CC(I, J, K) ec[((idx_t)(K) * cny + (J)) * cnx + (I)]
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int I = i / 2, J = j / 2, K = k / 2;
                double v;
                if (kind == 1) {
                    v = CC(I, J, K);
                } else {
                    /* neighbour parent on the fine cell's side; mirror at walls */
                    int I2 = (i & 1) ? I + 1 : I - 1;
                    int J2 = (j & 1) ? J + 1 : J - 1;
                    int K2 = (k & 1) ? K + 1 : K - 1;
                    if (I2 < 0 || I2 >= cnx) I2 = I;
                    if (J2 < 0 || J2 >= cny) J2 = J;
                    if (K2 < 0 || K2 >= cnz) K2 = K;
                    const double w[2] = {0.75, 0.25};
                    int Ii[2] = {I, I2}, Jj[2] = {J, J2}, Kk[2] = {K, K2};
                    v = 0.0;
                    for (int c = 0; c < 2; ++c)
                        for (int b = 0; b < 2; ++b)
                            for (int a = 0; a < 2; ++a)
                                v += w[a] * w[b] * w[c] * CC(Ii[a], Jj[b], Kk[c]);
                }
                e[CELL(i, j, k)] += v;
            }
#undef CC
}

/* coarse face = mean of the 4 fine faces tiling it; coarse walls 0 */
void or_coarsen_faces(int nx, int ny, int nz, const double *bx, const double *by,
                      const double *bz, double *cbx, double *cby, double *cbz) {
    int cnx = nx / 2, cny = ny / 2, cnz = nz / 2;
    memset(cbx, 0, sizeof(double) * (size_t)cnz * cny * (cnx + 1));
    memset(cby, 0, sizeof(double) * (size_t)cnz * (cny + 1) * cnx);
    memset(cbz, 0, sizeof(double) * (size_t)(cnz + 1) * cny * cnx);
    for (int K = 0; K < cnz; ++K)
        for (int J = 0; J < cny; ++J)
            for (int I = 1; I < cnx; ++I) {
                double s = 0.0;
                for (int c = 0; c < 2; ++c)
                    for (int b = 0; b < 2; ++b) s += bx[FXI(2 * I, 2 * J + b, 2 * K + c)];
                cbx[((idx_t)K * cny + J) * (cnx + 1) + I] = s / 4.0;
            }
    for (int K = 0; K < cnz; ++K)
        for (int J = 1; J < cny; ++J)
            for (int I = 0; I < cnx; ++I) {
                double s = 0.0;
                for (int c = 0; c < 2; ++c)
                    for (int a = 0; a < 2; ++a) s += by[FYI(2 * I + a, 2 * J, 2 * K + c)];
                cby[((idx_t)K * (cny + 1) + J) * cnx + I] = s / 4.0;
            }
    for (int K = 1; K < cnz; ++K)
        for (int J = 0; J < cny; ++J)
            for (int I = 0; I < cnx; ++I) {
                double s = 0.0;
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a) s += bz[FZI(2 * I + a, 2 * J + b, 2 * K)];
                cbz[((idx_t)K * cny + J) * cnx + I] = s / 4.0;
            }
}

/* ---- dense coarse solve ---------------------------------------------------- */
/* dense n x n matrix of A (row-major), n = nx*ny*nz */
void or_assemble_dense(int nx, int ny, int nz, double h, const double *bx, const double *by,
                       const double *bz, double *A) {
    idx_t n = (idx_t)nx * ny * nz;
    double ih2 = 1.0 / (h * h);
    memset(A, 0, sizeof(double) * (size_t)(n * n));
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                idx_t c = CELL(i, j, k);
                /* each interior face couples c and its neighbour */
                idx_t nb[6];
                double bf[6];
                int cnt = 0;
                if (i > 0) { nb[cnt] = CELL(i - 1, j, k); bf[cnt++] = bx[FXI(i, j, k)]; }
                if (i < nx - 1) { nb[cnt] = CELL(i + 1, j, k); bf[cnt++] = bx[FXI(i + 1, j, k)]; }
                if (j > 0) { nb[cnt] = CELL(i, j - 1, k); bf[cnt++] = by[FYI(i, j, k)]; }
                if (j < ny - 1) { nb[cnt] = CELL(i, j + 1, k); bf[cnt++] = by[FYI(i, j + 1, k)]; }
                if (k > 0) { nb[cnt] = CELL(i, j, k - 1); bf[cnt++] = bz[FZI(i, j, k)]; }
                if (k < nz - 1) { nb[cnt] = CELL(i, j, k + 1); bf[cnt++] = bz[FZI(i, j, k + 1)]; }
                for (int q = 0; q < cnt; ++q) {
                    A[c * n + c] += bf[q] * ih2;
                    A[c * n + nb[q]] -= bf[q] * ih2;
                }
            }
}

/* In-place Cholesky M = L L^T (lower triangle of row-major M); returns 0 on success */
static int cholesky(idx_t n, double *M) {
    for (idx_t j = 0; j < n; ++j) {
        double d = M[j * n + j];
        for (idx_t q = 0; q < j; ++q) d -= M[j * n + q] * M[j * n + q];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        M[j * n + j] = d;
        for (idx_t i = j + 1; i < n; ++i) {
            double s = M[i * n + j];
            for (idx_t q = 0; q < j; ++q) s -= M[i * n + q] * M[j * n + q];
            M[i * n + j] = s / d;
        }
    }
    return 0;
}

static void chol_solve(idx_t n, const double *L, double *x) {
    for (idx_t i = 0; i < n; ++i) {
        double s = x[i];
        for (idx_t q = 0; q < i; ++q) s -= L[i * n + q] * x[q];
        x[i] = s / L[i * n + i];
    }
    for (idx_t i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (idx_t q = i + 1; q < n; ++q) s -= L[q * n + i] * x[q];
        x[i] = s / L[i * n + i];
    }
}

/* Factor M = A_c + c 1 1^T, c = mean(diag A_c)/n.  L receives the factor. */
static int coarse_factor(int nx, int ny, int nz, double h, const double *bx, const double *by,
                         const double *bz, double *L) {
    idx_t n = (idx_t)nx * ny * nz;
    or_assemble_dense(nx, ny, nz, h, bx, by, bz, L);
    double dsum = 0.0;
    for (idx_t i = 0; i < n; ++i) dsum += L[i * n + i];
    double c = (dsum / (double)n) / (double)n;
    for (idx_t m = 0; m < n * n; ++m) L[m] += c;
    return cholesky(n, L);
}

/* e = A^+ (r - mean r) given the factor of A + c 1 1^T */
static void coarse_apply(int nx, int ny, int nz, const double *L, const double *r, double *e) {
    idx_t n = (idx_t)nx * ny * nz;
    double mr = or_mean(nx, ny, nz, r);
    for (idx_t i = 0; i < n; ++i) e[i] = r[i] - mr;
    chol_solve(n, L, e);
    double me = or_mean(nx, ny, nz, e);
    for (idx_t i = 0; i < n; ++i) e[i] -= me; /* exact no-op up to rounding */
}

/* Stand-alone coarse solve on any small grid: e = A^+ (r - mean r). */
int or_coarse_solve(int nx, int ny, int nz, double h, const double *bx, const double *by,
                    const double *bz, const double *r, double *e) {
    idx_t n = (idx_t)nx * ny * nz;
    if (n < 1 || n > OR_MAX_COARSE) return OR_ERR_ARG;
    double *L = (double *)malloc(sizeof(double) * (size_t)(n * n));
    if (!L) return OR_ERR_OOM;
    int st = coarse_factor(nx, ny, nz, h, bx, by, bz, L);
    if (st == 0) coarse_apply(nx, ny, nz, L, r, e);
    free(L);
    return st == 0 ? OR_OK : OR_ERR_ARG;
}

/* ---- the multigrid hierarchy and V-cycle --------------------------------- */
typedef struct {
    int nx, ny, nz;
    double h;
    double *bx, *by, *bz;   /* faces (API layout) */
    double *b, *x, *r;      /* per-level RHS, iterate, residual */
} or_level;

typedef struct {
    int nlev, pre, post, prolong;
    or_level lv[OR_MAX_LEVELS];
    double *L; /* Cholesky factor of the coarsest operator (+ c 1 1^T) */
} or_mg;

void or_mg_free(or_mg *M) {
    if (!M) return;
    for (int l = 0; l < M->nlev; ++l) {
        free(M->lv[l].bx);
        free(M->lv[l].by);
        free(M->lv[l].bz);
        free(M->lv[l].b);
        free(M->lv[l].x);
        free(M->lv[l].r);
    }
    free(M->L);
    free(M);
}

/* number of levels the halving rule produces (0 on bad input) */
int or_num_levels(int nx, int ny, int nz, int coarsest) {
    if (nx < 1 || ny < 1 || nz < 1 || coarsest < 2) return 0;
    int nl = 1;
    while (nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0) {
        int mx = nx > ny ? nx : ny;
        mx = mx > nz ? mx : nz;
        if (mx <= coarsest) break;
        nx /= 2;
        ny /= 2;
        nz /= 2;
        ++nl;
    }
    return nl;
}

or_mg *or_mg_create(int nx, int ny, int nz, double h, const double *bx, const double *by,
                    const double *bz, int coarsest, int pre, int post, int prolong, int *status) {
    int nl = or_num_levels(nx, ny, nz, coarsest);
    *status = OR_ERR_ARG;
    if (nl < 1 || nl > OR_MAX_LEVELS || (idx_t)nx * ny * nz < 2) return NULL;
    or_mg *M = (or_mg *)calloc(1, sizeof(or_mg));
    M->nlev = nl;
    M->pre = pre;
    M->post = post;
    M->prolong = prolong;
    for (int l = 0; l < nl; ++l) {
        or_level *L = &M->lv[l];
        L->nx = nx >> l;
        L->ny = ny >> l;
        L->nz = nz >> l;
        L->h = ldexp(h, l);
        size_t n = (size_t)L->nx * L->ny * L->nz;
        L->bx = (double *)malloc(sizeof(double) * (size_t)L->nz * L->ny * (L->nx + 1));
        L->by = (double *)malloc(sizeof(double) * (size_t)L->nz * (L->ny + 1) * L->nx);
        L->bz = (double *)malloc(sizeof(double) * (size_t)(L->nz + 1) * L->ny * L->nx);
        L->b = (double *)calloc(n, sizeof(double));
        L->x = (double *)calloc(n, sizeof(double));
        L->r = (double *)calloc(n, sizeof(double));
        if (!L->bx || !L->by || !L->bz || !L->b || !L->x || !L->r) {
            M->nlev = l + 1;
            or_mg_free(M);
            *status = OR_ERR_OOM;
            return NULL;
        }
    }
    memcpy(M->lv[0].bx, bx, sizeof(double) * (size_t)nz * ny * (nx + 1));
    memcpy(M->lv[0].by, by, sizeof(double) * (size_t)nz * (ny + 1) * nx);
    memcpy(M->lv[0].bz, bz, sizeof(double) * (size_t)(nz + 1) * ny * nx);
    for (int l = 0; l + 1 < nl; ++l) {
        or_level *F = &M->lv[l], *C = &M->lv[l + 1];
        or_coarsen_faces(F->nx, F->ny, F->nz, F->bx, F->by, F->bz, C->bx, C->by, C->bz);
    }
    or_level *C = &M->lv[nl - 1];
    idx_t nc = (idx_t)C->nx * C->ny * C->nz;
    if (nc > OR_MAX_COARSE) {
        or_mg_free(M);
        return NULL;
    }
    M->L = (double *)malloc(sizeof(double) * (size_t)(nc * nc));
    if (coarse_factor(C->nx, C->ny, C->nz, C->h, C->bx, C->by, C->bz, M->L) != 0) {
        or_mg_free(M);
        return NULL;
    }
    *status = OR_OK;
    return M;
}

int or_mg_nlevels(const or_mg *M) { return M->nlev; }

void or_mg_level_dims(const or_mg *M, int l, int *dims) {
    dims[0] = M->lv[l].nx;
    dims[1] = M->lv[l].ny;
    dims[2] = M->lv[l].nz;
}

void or_mg_level_faces(const or_mg *M, int l, double *bx, double *by, double *bz) {
    const or_level *L = &M->lv[l];
    memcpy(bx, L->bx, sizeof(double) * (size_t)L->nz * L->ny * (L->nx + 1));
    memcpy(by, L->by, sizeof(double) * (size_t)L->nz * (L->ny + 1) * L->nx);
    memcpy(bz, L->bz, sizeof(double) * (size_t)(L->nz + 1) * L->ny * L->nx);
}

/* V-cycle on level l: improves the iterate x for A_l x = b (x is in/out) */
static void vcycle(or_mg *M, int l, const double *b, double *x) {
    or_level *F = &M->lv[l];
    if (l == M->nlev - 1) {
        coarse_apply(F->nx, F->ny, F->nz, M->L, b, x);
        return;
    }
    or_level *C = &M->lv[l + 1];
    or_rbgs(F->nx, F->ny, F->nz, F->h, F->bx, F->by, F->bz, b, x, M->pre, 0);
    or_residual(F->nx, F->ny, F->nz, F->h, F->bx, F->by, F->bz, b, x, F->r);
    or_restrict(F->nx, F->ny, F->nz, F->r, C->b);
    memset(C->x, 0, sizeof(double) * (size_t)C->nx * C->ny * C->nz);
    vcycle(M, l + 1, C->b, C->x);
    or_prolong_correct(C->nx, C->ny, C->nz, C->x, x, M->prolong);
    or_rbgs(F->nx, F->ny, F->nz, F->h, F->bx, F->by, F->bz, b, x, M->post, 1);
}

/* one V-cycle on the finest level, x in/out (no gauge fix) */
void or_mg_vcycle(or_mg *M, const double *b, double *x) { vcycle(M, 0, b, x); }

/* Solve A p = b - mean(b), mean(p) = 0, by V-cycles until
 * |b~ - A p|_2 / |b~|_2 <= rtol (b~ = b - mean b).  hist[c] = relative residual
 * after c cycles (hist[0] for the initial p).  With stop_on_stall, the loop
 * also ends (OR_OK) once the residual has failed to drop below 0.999 of its
 * best value for 2 consecutive cycles: the discrete solution is then reached
 * to rounding.  Returns OR_OK, OR_ERR_NOT_CONVERGED or OR_ERR_DIVERGED;
 * *ncycles = cycles run. */
int or_mg_solve(or_mg *M, const double *b_in, double *p, double rtol, int max_cycles,
                int warm_start, int stop_on_stall, double *hist, int hist_len, int *ncycles,
                double *relres) {
    or_level *F = &M->lv[0];
    int nx = F->nx, ny = F->ny, nz = F->nz;
    idx_t n = (idx_t)nx * ny * nz;
    double *b = F->b;
    double mb = or_mean(nx, ny, nz, b_in);
    for (idx_t m = 0; m < n; ++m) b[m] = b_in[m] - mb;
    double nb = or_norm2(nx, ny, nz, b);
    *ncycles = 0;
    if (!warm_start) memset(p, 0, sizeof(double) * (size_t)n);
    else add_const(nx, ny, nz, p, -or_mean(nx, ny, nz, p));
    if (nb == 0.0) {
        memset(p, 0, sizeof(double) * (size_t)n);
        *relres = 0.0;
        if (hist && hist_len > 0) hist[0] = 0.0;
        return OR_OK;
    }
    or_residual(nx, ny, nz, F->h, F->bx, F->by, F->bz, b, p, F->r);
    double rr = or_norm2(nx, ny, nz, F->r) / nb;
    if (hist && hist_len > 0) hist[0] = rr;
    *relres = rr;
    if (rr <= rtol) return OR_OK;
    double best = rr;
    int stall = 0;
    for (int c = 1; c <= max_cycles; ++c) {
        vcycle(M, 0, b, p);
        add_const(nx, ny, nz, p, -or_mean(nx, ny, nz, p));
        or_residual(nx, ny, nz, F->h, F->bx, F->by, F->bz, b, p, F->r);
        rr = or_norm2(nx, ny, nz, F->r) / nb;
        if (hist && c < hist_len) hist[c] = rr;
        *ncycles = c;
        *relres = rr;
        if (!isfinite(rr)) return OR_ERR_DIVERGED;
        if (rr <= rtol) return OR_OK;
        if (rr < 0.999 * best) {
            best = rr;
            stall = 0;
        } else if (stop_on_stall && ++stall >= 2) {
            return OR_OK;
        }
    }
    return OR_ERR_NOT_CONVERGED;
}

/* ---- projection: the velocity correction ---------------------------------- */
/* With b = D u + sigma D(beta csf) and A p = b (A = -D diag(beta) G), the corrected face
 * velocities u + beta (G p + sigma csf) have zero discrete divergence: on every interior face
 *     u_f += beta_f ((p_R - p_L) / h + sigma csf_f),
 * wall faces unchanged.  csf pointers may be NULL (no surface term). */
void or_project(int nx, int ny, int nz, double h, const double *bx, const double *by, const double *bz,
                const double *p, const double *csfx, const double *csfy, const double *csfz, double sigma,
                double *ux, double *uy, double *uz) {
    const double ih = 1.0 / h;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                if (i > 0 && i < nx) {
                    idx_t f = ((idx_t)k * ny + j) * (nx + 1) + i;
                    idx_t c = ((idx_t)k * ny + j) * nx + i;
                    ux[f] += bx[f] * ((p[c] - p[c - 1]) * ih + (csfx ? sigma * csfx[f] : 0.0));
                }
            }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                idx_t f = ((idx_t)k * (ny + 1) + j) * nx + i;
                idx_t c = ((idx_t)k * ny + j) * nx + i;
                uy[f] += by[f] * ((p[c] - p[c - nx]) * ih + (csfy ? sigma * csfy[f] : 0.0));
            }
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                idx_t f = ((idx_t)k * ny + j) * nx + i;
                idx_t c = f;
                uz[f] += bz[f] * ((p[c] - p[c - (idx_t)nx * ny]) * ih + (csfz ? sigma * csfz[f] : 0.0));
            }
}

/* ---- density adjoint -------------------------------------------------------- */
/* beta_f = (1/rho_L + 1/rho_R) / 2, so d beta_f / d rho_c = -1 / (2 rho_c^2) for the faces of c:
 *     dL/drho_c = -1/(2 rho_c^2) * sum over the interior faces f of c of dL/dbeta_f.
 * With rho = sum_q rho_q f_q + rho_last (1 - sum_q f_q) (Eq. (5) for nfrac fractions),
 *     dL/df_q = dL/drho * (rho_q - rho_last)   (dfrac: nfrac cell arrays, may be NULL). */
void or_density_grads(int nx, int ny, int nz, const double *rho, const double *gx, const double *gy,
                      const double *gz, double *drho, int nfrac, const double *rho_phase, double *dfrac) {
    const idx_t n = (idx_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                idx_t c = ((idx_t)k * ny + j) * nx + i;
                idx_t fx = ((idx_t)k * ny + j) * (nx + 1) + i;
                idx_t fy = ((idx_t)k * (ny + 1) + j) * nx + i;
                double g = 0.0;
                if (i > 0) g += gx[fx];
                if (i < nx - 1) g += gx[fx + 1];
                if (j > 0) g += gy[fy];
                if (j < ny - 1) g += gy[fy + nx];
                if (k > 0) g += gz[c];
                if (k < nz - 1) g += gz[c + (idx_t)nx * ny];
                double d = -g / (2.0 * rho[c] * rho[c]);
                drho[c] = d;
                if (dfrac)
                    for (int q = 0; q < nfrac; ++q) dfrac[q * n + c] = d * (rho_phase[q] - rho_phase[nfrac]);
            }
}

/* ---- flexible preconditioned conjugate gradients ------------------------- */
/* a . b, summed per z-plane then over planes in order (deterministic at any thread count) */
static double dot(int nx, int ny, int nz, const double *a, const double *b) {
    const idx_t nxy = (idx_t)nx * ny;
    double *ps = (double *)calloc((size_t)nz, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        double s = 0.0;
        for (idx_t m = (idx_t)k * nxy; m < (idx_t)(k + 1) * nxy; ++m) s += a[m] * b[m];
        ps[k] = s;
    }
    double s = 0.0;
    for (int k = 0; k < nz; ++k) s += ps[k];
    free(ps);
    return s;
}

/* Solve A p = b~ (b~ = b - mean b) by conjugate gradients preconditioned with one V-cycle
 * from zero, z = V(r), in the flexible form: the Polak-Ribiere choice of beta keeps it a
 * descent method when the preconditioner is not exactly symmetric (trilinear prolongation
 * with averaging restriction, or a preconditioner applied in lower precision); with a
 * symmetric preconditioner it is ordinary preconditioned CG.  Starting from p = 0:
 *     r_0 = b~,  z_0 = V(r_0),  d_0 = z_0
 *     for k = 0, 1, ...
 *         q = A d_k,   alpha = (r_k . z_k) / (d_k . q)
 *         p += alpha d_k,   r_{k+1} = r_k - alpha q        (stop once |r_{k+1}| <= rtol |b~|)
 *         z_{k+1} = V(r_{k+1})
 *         beta = z_{k+1} . (r_{k+1} - r_k) / (r_k . z_k) = -alpha (z_{k+1} . q) / (r_k . z_k)
 *         d_{k+1} = z_{k+1} + beta d_k
 * hist[k] = |r_k| / |b~| (the updated residual); at exit p gets zero mean and *relres is
 * the true relative residual |b~ - A p| / |b~|.  rec_r, rec_z (may be NULL) receive r_k
 * and z_k for k < rec_n, one cell array each. */
int or_mg_fcg(or_mg *M, const double *b_in, double *p, double rtol, int max_it, double *hist,
              int hist_len, int *nit, double *relres, double *rec_r, double *rec_z, int rec_n) {
    or_level *F = &M->lv[0];
    int nx = F->nx, ny = F->ny, nz = F->nz;
    idx_t n = (idx_t)nx * ny * nz;
    double h = F->h;
    double *b = F->b;
    double mb = or_mean(nx, ny, nz, b_in);
    for (idx_t m = 0; m < n; ++m) b[m] = b_in[m] - mb;
    double nb = or_norm2(nx, ny, nz, b);
    memset(p, 0, sizeof(double) * (size_t)n);
    *nit = 0;
    *relres = 0.0;
    if (hist && hist_len > 0) hist[0] = nb == 0.0 ? 0.0 : 1.0;
    if (nb == 0.0) return OR_OK;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)calloc((size_t)n, sizeof(double));
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    memcpy(r, b, sizeof(double) * (size_t)n);
    vcycle(M, 0, r, z);
    memcpy(d, z, sizeof(double) * (size_t)n);
    double rz = dot(nx, ny, nz, r, z);
    int status = OR_ERR_NOT_CONVERGED;
    for (int k = 0; k < max_it; ++k) {
        if (rec_r && k < rec_n) memcpy(rec_r + (idx_t)k * n, r, sizeof(double) * (size_t)n);
        if (rec_z && k < rec_n) memcpy(rec_z + (idx_t)k * n, z, sizeof(double) * (size_t)n);
        or_apply(nx, ny, nz, h, F->bx, F->by, F->bz, d, q);
        double alpha = rz / dot(nx, ny, nz, d, q);
        for (idx_t m = 0; m < n; ++m) {
            p[m] += alpha * d[m];
            r[m] -= alpha * q[m];
        }
        double rr = or_norm2(nx, ny, nz, r) / nb;
        *nit = k + 1;
        if (hist && k + 1 < hist_len) hist[k + 1] = rr;
        if (!isfinite(rr)) {
            status = OR_ERR_DIVERGED;
            break;
        }
        if (rr <= rtol) {
            status = OR_OK;
            break;
        }
        memset(z, 0, sizeof(double) * (size_t)n);
        vcycle(M, 0, r, z);
        double beta = -alpha * dot(nx, ny, nz, z, q) / rz;
        rz = dot(nx, ny, nz, r, z);
        for (idx_t m = 0; m < n; ++m) d[m] = z[m] + beta * d[m];
    }
    add_const(nx, ny, nz, p, -or_mean(nx, ny, nz, p));
    or_residual(nx, ny, nz, h, F->bx, F->by, F->bz, b, p, F->r);
    *relres = or_norm2(nx, ny, nz, F->r) / nb;
    free(r);
    free(z);
    free(d);
    free(q);
    return status;
}

/* ---- adjoint gradients ------------------------------------------------------ */
/* Given lambda = A^+(w - mean w) and the forward p, write
 *   g_f = -(lambda_L - lambda_R)(p_L - p_R)/h^2 + sigma csf_f (lambda_L - lambda_R)/h
 * on interior faces (walls 0) and dL/dsigma = sum_f beta_f csf_f (lambda_L - lambda_R)/h.
 * csf pointers may be NULL (no surface term; *dLdsigma = 0). */
void or_adjoint_grads(int nx, int ny, int nz, double h, const double *bx, const double *by,
                      const double *bz, const double *lam, const double *p, const double *csfx,
                      const double *csfy, const double *csfz, double sigma, double *gx,
                      double *gy, double *gz, double *dLdsigma) {
    double ih = 1.0 / h, ih2 = 1.0 / (h * h);
    memset(gx, 0, sizeof(double) * (size_t)nz * ny * (nx + 1));
    memset(gy, 0, sizeof(double) * (size_t)nz * (ny + 1) * nx);
    memset(gz, 0, sizeof(double) * (size_t)(nz + 1) * ny * nx);
    double *ps = (double *)calloc((size_t)nz, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        double s = 0.0;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                idx_t c = CELL(i, j, k);
                if (i > 0) {
                    idx_t l = CELL(i - 1, j, k), f = FXI(i, j, k);
                    double dl = lam[l] - lam[c];
                    gx[f] = -dl * (p[l] - p[c]) * ih2;
                    if (csfx) {
                        gx[f] += sigma * csfx[f] * dl * ih;
                        s += bx[f] * csfx[f] * dl * ih;
                    }
                }
                if (j > 0) {
                    idx_t l = CELL(i, j - 1, k), f = FYI(i, j, k);
                    double dl = lam[l] - lam[c];
                    gy[f] = -dl * (p[l] - p[c]) * ih2;
                    if (csfy) {
                        gy[f] += sigma * csfy[f] * dl * ih;
                        s += by[f] * csfy[f] * dl * ih;
                    }
                }
                if (k > 0) {
                    idx_t l = CELL(i, j, k - 1), f = FZI(i, j, k);
                    double dl = lam[l] - lam[c];
                    gz[f] = -dl * (p[l] - p[c]) * ih2;
                    if (csfz) {
                        gz[f] += sigma * csfz[f] * dl * ih;
                        s += bz[f] * csfz[f] * dl * ih;
                    }
                }
            }
        ps[k] = s;
    }
    double s = 0.0;
    for (int k = 0; k < nz; ++k) s += ps[k];
    free(ps);
    *dLdsigma = s;
}
