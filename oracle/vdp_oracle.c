/*
 * vdp_oracle.c -- TEST INFRASTRUCTURE ONLY (the CPU oracle).
 *
 * A plain, slow, obviously correct FP64 CPU restatement of the variable-coefficient pressure
 * Poisson problem of Pouransari, Mortazavi & Mani, "Parallel variable-density particle-laden
 * turbulence simulation" (arXiv:1601.05448):
 *
 *      div( (1/rho) grad p ) = f          (Sec. 3.4, the Poisson equation)
 *
 * on a uniform, triply periodic, staggered grid (Sec. 3.1, Sec. 3.2 case 1): rho, p and f live
 * at cell centres, the pressure gradient lives on cell faces. Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load this file; the GPU library shares no code,
 * header, table or constant with it, and neither side calls the other.
 *
 * Layout: every field is n = nx*ny*nz doubles, cell (i,j,k) at index c = i + nx*(j + ny*k)
 * (x fastest); spacing h_d = L / n_d; neighbours wrap periodically.  The `_g` entry points take
 * the box lengths per direction and the boundary condition in x: periodic, or the inflow-outflow
 * duct of Sec. 3.2 (case 2), where the pressure has no flux through the two x ends (see geom).  Face arrays bx, by, bz hold
 * one coefficient per cell: bx[c] belongs to the LOW x-face of cell c, i.e. the face shared by
 * cells (i-1,j,k) and (i,j,k); likewise by, bz.
 *
 * Readings of the paper taken here (the paper states the continuous equation only):
 *  - Face coefficient: 1/rho on a face is 1 / (arithmetic mean of the two adjacent cell-centre
 *    densities), the averaging App. B uses to carry rho to non-centre points; the 1/h_d^2 of the
 *    second difference is folded into the coefficient:  b_d[c] = 2 / (rho[c-e_d] + rho[c]) / h_d^2.
 *  - Discrete operator (conservative face-flux form of Sec. 3.4):
 *        (A p)_c = sum_d  b_d[c+e_d] (p[c+e_d] - p[c])  -  b_d[c] (p[c] - p[c-e_d]).
 *  - Compatibility (App. A, the chi' equation): on the periodic box the left side integrates to
 *    zero, so f is replaced by f - <f> (<.> = arithmetic mean over cells) and <f> is reported.
 *  - Gauge: p is unique up to a constant; the oracle returns the zero-mean p.
 *  - Tolerance: relative L2 residual ||(f-<f>) - A p|| / ||f-<f>||, recomputed from p at the end.
 *
 * Parity pins (see tests/test_oracle_pins.py): discrete Fourier eigen-solution for constant rho,
 * 1-D flux-integration closed form for rho varying along one axis (each axis), operator symmetry /
 * null space / energy identity, a dense direct solve on tiny grids, second-order convergence to a
 * smooth continuous solution, and agreement of the two independent solvers below (conjugate
 * gradients, and the paper's own fixed-point iteration of Eq. (Pois)).  The face-average choice is
 * a reading, not something the paper fixes: it is pinned only through the 1-D closed form, which
 * is written from that same reading.  The projection steps around the solve (App. A: the Poisson
 * right side and the momentum correction of Eq. (mom)) are pinned by a pure-gradient field that
 * the projection removes, a face-density-weighted solenoidal field it leaves alone, the App. A
 * divergence constraint on the corrected velocity, idempotence, and, on tiny grids, the
 * density-weighted least-change projection onto the discrete divergence constraint computed by
 * dense null-space linear algebra.
 *
 * Reductions are deterministic: each z-plane is summed in index order, then the planes are summed
 * in order, so results do not depend on the OpenMP thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define VDPO_OK 0
#define VDPO_EINVAL 1
#define VDPO_ENOMEM 2
#define VDPO_EDENSITY 3
#define VDPO_ENOTCONV 4
#define VDPO_EBREAKDOWN 5

static long wrap(long i, long n) { return (i % n + n) % n; }

static long idx(long i, long j, long k, long nx, long ny, long nz) {
  return wrap(i, nx) + nx * (wrap(j, ny) + ny * wrap(k, nz));
}

/* ---- deterministic reductions ------------------------------------------------------------ */

static double sum_planes(const double *plane_sums, long nz) {
  double s = 0.0;
  for (long k = 0; k < nz; ++k) s += plane_sums[k];
  return s;
}

double vdpo_sum(int nx, int ny, int nz, const double *x) {
  double *ps = (double *)malloc(sizeof(double) * (size_t)nz);
  long plane = (long)nx * ny;
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nz; ++k) {
    double s = 0.0;
    for (long m = 0; m < plane; ++m) s += x[k * plane + m];
    ps[k] = s;
  }
  double s = sum_planes(ps, nz);
  free(ps);
  return s;
}

double vdpo_dot(int nx, int ny, int nz, const double *x, const double *y) {
  double *ps = (double *)malloc(sizeof(double) * (size_t)nz);
  long plane = (long)nx * ny;
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nz; ++k) {
    double s = 0.0;
    for (long m = 0; m < plane; ++m) s += x[k * plane + m] * y[k * plane + m];
    ps[k] = s;
  }
  double s = sum_planes(ps, nz);
  free(ps);
  return s;
}

double vdpo_mean(int nx, int ny, int nz, const double *x) {
  return vdpo_sum(nx, ny, nz, x) / ((double)nx * ny * nz);
}

/* ---- face coefficients (Sec. 3.1 staggered layout, App. B averaging) ------------------------ */

/*
 * Geometry: box lengths per direction and the boundary condition in x.  bc_x = 0: periodic (the
 * triply periodic box, Sec. 3.2 case 1).  bc_x = 1: the inflow-outflow duct (Sec. 3.2 case 2):
 * periodic in y and z, and the pressure has no flux through the inflow and outflow faces
 * (homogeneous Neumann; the paper does not state the pressure condition, this is the reading
 * taken).  The face at x = 0 and the face at x = Lx share the storage slot bx[i = 0], whose
 * coefficient is then 0: no term couples cell 0 with cell nx - 1.
 */
typedef struct {
  double Lx, Ly, Lz;
  int bc_x;
} geom;

static geom cube(double L) {
  geom g = {L, L, L, 0};
  return g;
}

static int geom_ok(geom g) {
  return g.Lx > 0.0 && g.Ly > 0.0 && g.Lz > 0.0 && isfinite(g.Lx) && isfinite(g.Ly) &&
         isfinite(g.Lz) && (g.bc_x == 0 || g.bc_x == 1);
}

static int face_coefficients_g(int nx, int ny, int nz, geom G, const double *rho, double *bx,
                               double *by, double *bz) {
  if (nx < 1 || ny < 1 || nz < 1 || !geom_ok(G)) return VDPO_EINVAL;
  long n = (long)nx * ny * nz;
  for (long c = 0; c < n; ++c)
    if (!(rho[c] > 0.0) || !isfinite(rho[c])) return VDPO_EDENSITY;
  double hx = G.Lx / nx, hy = G.Ly / ny, hz = G.Lz / nz;
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        long c = idx(i, j, k, nx, ny, nz);
        /* face density = mean of the two cell-centre densities it separates */
        double rx = 0.5 * (rho[idx(i - 1, j, k, nx, ny, nz)] + rho[c]);
        double ry = 0.5 * (rho[idx(i, j - 1, k, nx, ny, nz)] + rho[c]);
        double rz = 0.5 * (rho[idx(i, j, k - 1, nx, ny, nz)] + rho[c]);
        bx[c] = (G.bc_x == 1 && i == 0) ? 0.0 : (1.0 / rx) / (hx * hx);  /* duct: no x wrap */
        by[c] = (1.0 / ry) / (hy * hy);
        bz[c] = (1.0 / rz) / (hz * hz);
      }
  return VDPO_OK;
}

int vdpo_face_coefficients(int nx, int ny, int nz, double L, const double *rho, double *bx,
                           double *by, double *bz) {
  return face_coefficients_g(nx, ny, nz, cube(L), rho, bx, by, bz);
}

int vdpo_face_coefficients_g(int nx, int ny, int nz, double Lx, double Ly, double Lz, int bc_x,
                             const double *rho, double *bx, double *by, double *bz) {
  geom G = {Lx, Ly, Lz, bc_x};
  return face_coefficients_g(nx, ny, nz, G, rho, bx, by, bz);
}

/* ---- the discrete operator A ~ div((1/rho) grad .)  (Sec. 3.4) ------------------------------ */

void vdpo_apply(int nx, int ny, int nz, const double *bx, const double *by, const double *bz,
                const double *p, double *out) {
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        long c = idx(i, j, k, nx, ny, nz);
        long xm = idx(i - 1, j, k, nx, ny, nz), xp = idx(i + 1, j, k, nx, ny, nz);
        long ym = idx(i, j - 1, k, nx, ny, nz), yp = idx(i, j + 1, k, nx, ny, nz);
        long zm = idx(i, j, k - 1, nx, ny, nz), zp = idx(i, j, k + 1, nx, ny, nz);
        /* flux through the high face minus flux through the low face, per direction */
        double ax = bx[xp] * (p[xp] - p[c]) - bx[c] * (p[c] - p[xm]);
        double ay = by[yp] * (p[yp] - p[c]) - by[c] * (p[c] - p[ym]);
        double az = bz[zp] * (p[zp] - p[c]) - bz[c] * (p[c] - p[zm]);
        out[c] = ax + ay + az;
      }
}

/* diagonal of -A: the sum of the six face coefficients around each cell */
static void neg_diagonal(int nx, int ny, int nz, const double *bx, const double *by,
                         const double *bz, double *diag) {
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        long c = idx(i, j, k, nx, ny, nz);
        diag[c] = bx[c] + bx[idx(i + 1, j, k, nx, ny, nz)] + by[c] +
                  by[idx(i, j + 1, k, nx, ny, nz)] + bz[c] + bz[idx(i, j, k + 1, nx, ny, nz)];
      }
}

/* relative residual ||f0 - A p|| / ||f0|| with f0 already mean-free; r receives f0 - A p */
static double true_residual(int nx, int ny, int nz, const double *bx, const double *by,
                            const double *bz, const double *f0, const double *p, double *r,
                            double f0norm) {
  long n = (long)nx * ny * nz;
  vdpo_apply(nx, ny, nz, bx, by, bz, p, r);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < n; ++c) r[c] = f0[c] - r[c];
  return sqrt(vdpo_dot(nx, ny, nz, r, r)) / f0norm;
}

static double relative_residual_g(int nx, int ny, int nz, geom G, const double *rho,
                                  const double *f, const double *p) {
  long n = (long)nx * ny * nz;
  double *bx = malloc(sizeof(double) * n), *by = malloc(sizeof(double) * n);
  double *bz = malloc(sizeof(double) * n), *f0 = malloc(sizeof(double) * n);
  double *r = malloc(sizeof(double) * n);
  double res = -1.0;
  if (bx && by && bz && f0 && r &&
      face_coefficients_g(nx, ny, nz, G, rho, bx, by, bz) == VDPO_OK) {
    double mf = vdpo_mean(nx, ny, nz, f);
    for (long c = 0; c < n; ++c) f0[c] = f[c] - mf;
    double fn = sqrt(vdpo_dot(nx, ny, nz, f0, f0));
    res = fn > 0.0 ? true_residual(nx, ny, nz, bx, by, bz, f0, p, r, fn)
                   : sqrt(vdpo_dot(nx, ny, nz, p, p));
  }
  free(bx); free(by); free(bz); free(f0); free(r);
  return res;
}

double vdpo_relative_residual(int nx, int ny, int nz, double L, const double *rho,
                              const double *f, const double *p) {
  return relative_residual_g(nx, ny, nz, cube(L), rho, f, p);
}

double vdpo_relative_residual_g(int nx, int ny, int nz, double Lx, double Ly, double Lz, int bc_x,
                                const double *rho, const double *f, const double *p) {
  geom G = {Lx, Ly, Lz, bc_x};
  return relative_residual_g(nx, ny, nz, G, rho, f, p);
}

/*
 * Solver 1: Jacobi-preconditioned conjugate gradients on the symmetric positive semi-definite
 * system (-A) p = -(f - <f>), started from p = 0 so every iterate stays mean-free in exact
 * arithmetic.  The recursive residual decides when to look; the true residual decides when to
 * stop (on a miss the true residual replaces the recursive one and the search restarts).
 * info[0] = iterations, info[1] = final relative residual, info[2] = <f> removed (chi' of App. A).
 */
static int solve_cg_g(int nx, int ny, int nz, geom G, const double *rho, const double *f,
                      double *p, double tol, int maxit, double *info) {
  long n = (long)nx * ny * nz;
  int status = VDPO_OK;
  double *bx = malloc(sizeof(double) * n), *by = malloc(sizeof(double) * n);
  double *bz = malloc(sizeof(double) * n), *dg = malloc(sizeof(double) * n);
  double *f0 = malloc(sizeof(double) * n), *r = malloc(sizeof(double) * n);
  double *z = malloc(sizeof(double) * n), *d = malloc(sizeof(double) * n);
  double *q = malloc(sizeof(double) * n);
  info[0] = 0; info[1] = 0; info[2] = 0;
  if (!bx || !by || !bz || !dg || !f0 || !r || !z || !d || !q) { status = VDPO_ENOMEM; goto done; }
  status = face_coefficients_g(nx, ny, nz, G, rho, bx, by, bz);
  if (status != VDPO_OK) goto done;
  neg_diagonal(nx, ny, nz, bx, by, bz, dg);

  double mf = vdpo_mean(nx, ny, nz, f);
  info[2] = mf;
  for (long c = 0; c < n; ++c) { f0[c] = f[c] - mf; p[c] = 0.0; }
  double fn = sqrt(vdpo_dot(nx, ny, nz, f0, f0));
  if (fn == 0.0) goto done; /* zero (or constant) right-hand side: p = 0 */

  /* M = -A, b = -f0;  r = b - M p = -f0 at p = 0 */
  for (long c = 0; c < n; ++c) r[c] = -f0[c];
  double rnorm = fn;
  int it = 0, restart = 1;
  double rz = 0.0;
  while (1) {
    if (restart) {
      for (long c = 0; c < n; ++c) { z[c] = r[c] / dg[c]; d[c] = z[c]; }
      rz = vdpo_dot(nx, ny, nz, r, z);
      restart = 0;
    }
    if (it >= maxit) { status = VDPO_ENOTCONV; break; }
    /* q = M d = -A d */
    vdpo_apply(nx, ny, nz, bx, by, bz, d, q);
    for (long c = 0; c < n; ++c) q[c] = -q[c];
    double dq = vdpo_dot(nx, ny, nz, d, q);
    if (!(dq > 0.0)) { status = VDPO_EBREAKDOWN; break; }
    double alpha = rz / dq;
    for (long c = 0; c < n; ++c) { p[c] += alpha * d[c]; r[c] -= alpha * q[c]; }
    ++it;
    rnorm = sqrt(vdpo_dot(nx, ny, nz, r, r));
    if (rnorm <= tol * fn) {
      /* verify with the true residual of the original equation A p = f0 */
      double tr = true_residual(nx, ny, nz, bx, by, bz, f0, p, q, fn);
      if (tr <= tol) break;
      for (long c = 0; c < n; ++c) r[c] = -q[c]; /* r = -(f0 - A p) */
      restart = 1;
      continue;
    }
    for (long c = 0; c < n; ++c) z[c] = r[c] / dg[c];
    double rz_new = vdpo_dot(nx, ny, nz, r, z);
    double beta = rz_new / rz;
    rz = rz_new;
    for (long c = 0; c < n; ++c) d[c] = z[c] + beta * d[c];
  }
  info[0] = it;
  {
    /* gauge: zero-mean p */
    double mp = vdpo_mean(nx, ny, nz, p);
    for (long c = 0; c < n; ++c) p[c] -= mp;
    info[1] = true_residual(nx, ny, nz, bx, by, bz, f0, p, q, fn);
  }
done:
  free(bx); free(by); free(bz); free(dg); free(f0); free(r); free(z); free(d); free(q);
  return status;
}

int vdpo_solve_cg(int nx, int ny, int nz, double L, const double *rho, const double *f, double *p,
                  double tol, int maxit, double *info) {
  return solve_cg_g(nx, ny, nz, cube(L), rho, f, p, tol, maxit, info);
}

int vdpo_solve_cg_g(int nx, int ny, int nz, double Lx, double Ly, double Lz, int bc_x,
                    const double *rho, const double *f, double *p, double tol, int maxit,
                    double *info) {
  geom G = {Lx, Ly, Lz, bc_x};
  return solve_cg_g(nx, ny, nz, G, rho, f, p, tol, maxit, info);
}

/* ---- Solver 2: the paper's iteration, Eq. (Pois) of Sec. 3.4 -------------------------------- */

/*
 * Plain separable complex DFT along one axis of a 3-D array (re, im), sign = -1 forward,
 * +1 backward (unnormalised).  O(n^2) per line: slow and obviously correct.
 */
static void dft_axis(int nx, int ny, int nz, double *re, double *im, int axis, int sign) {
  int nn = axis == 0 ? nx : (axis == 1 ? ny : nz);
  long stride = axis == 0 ? 1 : (axis == 1 ? nx : (long)nx * ny);
  long nlines = (long)nx * ny * nz / nn;
  double *cs = malloc(sizeof(double) * nn), *sn = malloc(sizeof(double) * nn);
  for (int m = 0; m < nn; ++m) {
    cs[m] = cos(2.0 * M_PI * m / nn);
    sn[m] = sin(2.0 * M_PI * m / nn);
  }
#pragma omp parallel
  {
    double *lr = malloc(sizeof(double) * nn), *li = malloc(sizeof(double) * nn);
#pragma omp for schedule(static)
    for (long line = 0; line < nlines; ++line) {
      /* base index of this line: all indices with the axis coordinate 0 */
      long base;
      if (axis == 0) base = line * nx;
      else if (axis == 1) base = (line % nx) + (line / nx) * (long)nx * ny;
      else base = line;
      for (int a = 0; a < nn; ++a) { lr[a] = re[base + a * stride]; li[a] = im[base + a * stride]; }
      for (int kk = 0; kk < nn; ++kk) {
        double sr = 0.0, si = 0.0;
        for (int a = 0; a < nn; ++a) {
          int m = (int)(((long)kk * a) % nn);
          double c = cs[m], s = sign * sn[m]; /* e^{sign * 2 pi i kk a / nn} = c + i s */
          sr += lr[a] * c - li[a] * s;
          si += lr[a] * s + li[a] * c;
        }
        re[base + kk * stride] = sr;
        im[base + kk * stride] = si;
      }
    }
    free(lr); free(li);
  }
  free(cs); free(sn);
}

/*
 * Plain cosine transforms along x of a real 3-D array (the eigenvectors of the x second
 * difference with zero flux through both ends, cell-centred: cos(pi k (2i + 1) / (2 nx))).
 * Forward: C_k = sum_i v_i cos(pi k (2i + 1) / (2 nx)).  Inverse:
 * v_i = (C_0 + 2 sum_{k >= 1} C_k cos(pi k (2i + 1) / (2 nx))) / nx.  O(nx^2) per line.
 */
static void dct_x(int nx, int ny, int nz, double *v, int inverse) {
  long nlines = (long)ny * nz;
  double *cs = malloc(sizeof(double) * (size_t)nx * nx);
  for (int k = 0; k < nx; ++k)
    for (int i = 0; i < nx; ++i) cs[(long)k * nx + i] = cos(M_PI * k * (2.0 * i + 1.0) / (2.0 * nx));
#pragma omp parallel
  {
    double *line = malloc(sizeof(double) * nx);
#pragma omp for schedule(static)
    for (long l = 0; l < nlines; ++l) {
      double *row = v + l * nx;
      for (int a = 0; a < nx; ++a) line[a] = row[a];
      for (int o = 0; o < nx; ++o) {
        double s = 0.0;
        if (!inverse) {
          for (int i = 0; i < nx; ++i) s += line[i] * cs[(long)o * nx + i];
        } else {
          s = line[0];
          for (int k = 1; k < nx; ++k) s += 2.0 * line[k] * cs[(long)k * nx + o];
          s /= nx;
        }
        row[o] = s;
      }
    }
    free(line);
  }
  free(cs);
}

/*
 * out = L_h^{-1} g for the constant-coefficient 7-point Laplacian L_h (coefficient 1/h_d^2 on
 * every face; in the duct no face at the x ends) with the zero mode set to zero.  Eigenvalues:
 *   periodic x:  lambda(k) = -sum_d 4 sin^2(pi k_d / n_d) / h_d^2 (Fourier modes in x, y, z);
 *   duct:        lambda(k) = -4 sin^2(pi k_x / (2 n_x)) / h_x^2 - (the y, z terms) (cosine modes
 *                in x, Fourier modes in y, z).
 */
static void inverse_laplacian_g(int nx, int ny, int nz, geom G, const double *g, double *out) {
  long n = (long)nx * ny * nz;
  double hx = G.Lx / nx, hy = G.Ly / ny, hz = G.Lz / nz;
  double *re = malloc(sizeof(double) * n), *im = calloc((size_t)n, sizeof(double));
  memcpy(re, g, sizeof(double) * n);
  if (G.bc_x == 1) dct_x(nx, ny, nz, re, 0);
  else dft_axis(nx, ny, nz, re, im, 0, -1);
  for (int a = 1; a < 3; ++a) dft_axis(nx, ny, nz, re, im, a, -1);
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        long c = i + nx * (j + ny * k);
        double sx = G.bc_x == 1 ? sin(M_PI * i / (2.0 * nx)) : sin(M_PI * i / nx);
        double sy = sin(M_PI * j / ny), sz = sin(M_PI * k / nz);
        double lam = -4.0 * (sx * sx / (hx * hx) + sy * sy / (hy * hy) + sz * sz / (hz * hz));
        if (c == 0) { re[c] = 0.0; im[c] = 0.0; }
        else { re[c] /= lam; im[c] /= lam; }
      }
  for (int a = 2; a >= 1; --a) dft_axis(nx, ny, nz, re, im, a, +1);
  if (G.bc_x == 1) {
    dct_x(nx, ny, nz, re, 1);
    for (long c = 0; c < n; ++c) out[c] = re[c] / ((double)ny * nz);
  } else {
    dft_axis(nx, ny, nz, re, im, 0, +1);
    for (long c = 0; c < n; ++c) out[c] = re[c] / (double)n;
  }
  free(re); free(im);
}

void vdpo_inverse_laplacian(int nx, int ny, int nz, double L, const double *g, double *out) {
  inverse_laplacian_g(nx, ny, nz, cube(L), g, out);
}

void vdpo_inverse_laplacian_g(int nx, int ny, int nz, double Lx, double Ly, double Lz, int bc_x,
                              const double *g, double *out) {
  geom G = {Lx, Ly, Lz, bc_x};
  inverse_laplacian_g(nx, ny, nz, G, g, out);
}

/*
 * The paper's fixed-point iteration.  With p = p_g + dp, Eq. (Pois) drops the term
 * rho grad(1/rho) . grad(dp) and solves the constant-coefficient equation
 *     lap(dp) = rho f - rho grad(1/rho) . grad(p_g) - lap(p_g)
 * then updates p_g <- p_g + dp until convergence.  Continuously the right side equals
 * rho (f - div((1/rho) grad p_g)); it is discretised as rho * (f0 - A p_g) with the same A as
 * solver 1, and lap^{-1} is the constant-coefficient inverse above.  An optional damping
 * omega (1 = the paper's update) scales dp.  Its fixed point is the solution of A p = f0.
 * info[0] = iterations, info[1] = final relative residual, info[2] = <f>.
 */
static int solve_fixed_point_g(int nx, int ny, int nz, geom G, const double *rho,
                               const double *f, double *p, double tol, int maxit, double omega,
                               double *info) {
  long n = (long)nx * ny * nz;
  int status = VDPO_OK;
  double *bx = malloc(sizeof(double) * n), *by = malloc(sizeof(double) * n);
  double *bz = malloc(sizeof(double) * n), *f0 = malloc(sizeof(double) * n);
  double *r = malloc(sizeof(double) * n), *dp = malloc(sizeof(double) * n);
  info[0] = 0; info[1] = 0; info[2] = 0;
  if (!bx || !by || !bz || !f0 || !r || !dp) { status = VDPO_ENOMEM; goto done; }
  status = face_coefficients_g(nx, ny, nz, G, rho, bx, by, bz);
  if (status != VDPO_OK) goto done;
  double mf = vdpo_mean(nx, ny, nz, f);
  info[2] = mf;
  for (long c = 0; c < n; ++c) { f0[c] = f[c] - mf; p[c] = 0.0; }
  double fn = sqrt(vdpo_dot(nx, ny, nz, f0, f0));
  if (fn == 0.0) goto done;
  int it = 0;
  double res = true_residual(nx, ny, nz, bx, by, bz, f0, p, r, fn);
  while (res > tol) {
    if (it >= maxit || !isfinite(res)) { status = VDPO_ENOTCONV; break; }
    for (long c = 0; c < n; ++c) r[c] *= rho[c]; /* rho (f0 - A p_g) */
    inverse_laplacian_g(nx, ny, nz, G, r, dp);
    for (long c = 0; c < n; ++c) p[c] += omega * dp[c];
    ++it;
    res = true_residual(nx, ny, nz, bx, by, bz, f0, p, r, fn);
  }
  {
    double mp = vdpo_mean(nx, ny, nz, p);
    for (long c = 0; c < n; ++c) p[c] -= mp;
  }
  info[0] = it;
  info[1] = true_residual(nx, ny, nz, bx, by, bz, f0, p, r, fn);
done:
  free(bx); free(by); free(bz); free(f0); free(r); free(dp);
  return status;
}

int vdpo_solve_fixed_point(int nx, int ny, int nz, double L, const double *rho, const double *f,
                           double *p, double tol, int maxit, double omega, double *info) {
  return solve_fixed_point_g(nx, ny, nz, cube(L), rho, f, p, tol, maxit, omega, info);
}

int vdpo_solve_fixed_point_g(int nx, int ny, int nz, double Lx, double Ly, double Lz, int bc_x,
                             const double *rho, const double *f, double *p, double tol, int maxit,
                             double omega, double *info) {
  geom G = {Lx, Ly, Lz, bc_x};
  return solve_fixed_point_g(nx, ny, nz, G, rho, f, p, tol, maxit, omega, info);
}

/* ---- the steps either side of the solve (App. A) ----------------------------------------------
 *
 * Face momenta (rho u_d) are stored like the face coefficients: mx[c] on the low x-face of cell c
 * (shared with cell c - e_x), likewise my, mz.  The face velocity is the face momentum divided by
 * the face density of App. B (mean of the two adjacent cell-centre densities), the same face
 * density the operator A uses, so that the projection below is exact for the discrete operator.
 */

/* discrete divergence at cell centres of a face field (ux, uy, uz) stored on low faces */
void vdpo_divergence(int nx, int ny, int nz, double L, const double *ux, const double *uy,
                     const double *uz, double *out) {
  double hx = L / nx, hy = L / ny, hz = L / nz;
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        long c = idx(i, j, k, nx, ny, nz);
        double dx = (ux[idx(i + 1, j, k, nx, ny, nz)] - ux[c]) / hx;
        double dy = (uy[idx(i, j + 1, k, nx, ny, nz)] - uy[c]) / hy;
        double dz = (uz[idx(i, j, k + 1, nx, ny, nz)] - uz[c]) / hz;
        out[c] = dx + dy + dz;
      }
}

/* face velocities u_d = m_d / rho_face (App. B face density) */
int vdpo_face_velocity(int nx, int ny, int nz, const double *rho, const double *mx,
                       const double *my, const double *mz, double *ux, double *uy, double *uz) {
  if (nx < 1 || ny < 1 || nz < 1) return VDPO_EINVAL;
  long n = (long)nx * ny * nz;
  for (long c = 0; c < n; ++c)
    if (!(rho[c] > 0.0) || !isfinite(rho[c])) return VDPO_EDENSITY;
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        long c = idx(i, j, k, nx, ny, nz);
        ux[c] = mx[c] / (0.5 * (rho[idx(i - 1, j, k, nx, ny, nz)] + rho[c]));
        uy[c] = my[c] / (0.5 * (rho[idx(i, j - 1, k, nx, ny, nz)] + rho[c]));
        uz[c] = mz[c] / (0.5 * (rho[idx(i, j, k - 1, nx, ny, nz)] + rho[c]));
      }
  return VDPO_OK;
}

/* Right side of the variable-coefficient Poisson equation of App. A, before its mean is removed:
 *     RHS^Pois = ( div( m~ / rho_new ) - RHS^div ) / c,     c = C_pre[k] * dt,
 * m~ the face momenta without the pressure gradient, rho_new the cell densities (through the face
 * density above), RHS^div the cell-centre divergence target (NULL: zero). */
int vdpo_projection_rhs(int nx, int ny, int nz, double L, const double *rho, const double *mx,
                        const double *my, const double *mz, const double *rhs_div, double c,
                        double *f) {
  if (nx < 1 || ny < 1 || nz < 1 || !(L > 0.0) || !(c > 0.0) || !isfinite(c)) return VDPO_EINVAL;
  long n = (long)nx * ny * nz;
  double *ux = (double *)malloc(sizeof(double) * (size_t)n);
  double *uy = (double *)malloc(sizeof(double) * (size_t)n);
  double *uz = (double *)malloc(sizeof(double) * (size_t)n);
  int status = VDPO_ENOMEM;
  if (!ux || !uy || !uz) goto done;
  status = vdpo_face_velocity(nx, ny, nz, rho, mx, my, mz, ux, uy, uz);
  if (status != VDPO_OK) goto done;
  vdpo_divergence(nx, ny, nz, L, ux, uy, uz, f);
  for (long q = 0; q < n; ++q) f[q] = (f[q] - (rhs_div ? rhs_div[q] : 0.0)) / c;
done:
  free(ux); free(uy); free(uz);
  return status;
}

/* Eq. (mom): (rho u_d)_new = (rho u_d)~ - c (dp/dx_d), the pressure difference across each low
 * face divided by the spacing. */
int vdpo_projection_correct(int nx, int ny, int nz, double L, const double *p, double c,
                            const double *mx, const double *my, const double *mz, double *ox,
                            double *oy, double *oz) {
  if (nx < 1 || ny < 1 || nz < 1 || !(L > 0.0) || !(c > 0.0) || !isfinite(c)) return VDPO_EINVAL;
  double hx = L / nx, hy = L / ny, hz = L / nz;
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        long q = idx(i, j, k, nx, ny, nz);
        ox[q] = mx[q] - c * ((p[q] - p[idx(i - 1, j, k, nx, ny, nz)]) / hx);
        oy[q] = my[q] - c * ((p[q] - p[idx(i, j - 1, k, nx, ny, nz)]) / hy);
        oz[q] = mz[q] - c * ((p[q] - p[idx(i, j, k - 1, nx, ny, nz)]) / hz);
      }
  return VDPO_OK;
}

int vdpo_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
