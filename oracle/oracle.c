/*
 * FP64 CPU oracle for the FTLE hot path.  TEST INFRASTRUCTURE ONLY: the tests, the smoke
 * check and the benchmark's CPU-baseline leg call it; the product path never does.
 *
 * It is the plain definition of what the GPU path computes, written for a reader who checks
 * it against the mathematics, not for speed:
 *
 *  1. Flowmap (the input of the paper's FTLE kernel, Section 2.2): each node is advected
 *     independently by the classic fourth-order Runge-Kutta method with a fixed step h
 *     (signed like the horizon T), n = round(|T| / |h|) steps from t0; step k evaluates the
 *     velocity at t_k, t_k + h/2 (twice) and t_k + h, with t_k = t0 + k h.
 *  2. FTLE kernel (the computation the paper's FTLE core pipeline performs, Section 2.1,
 *     Table 1; its definition comes from the UVaFTLE application the paper ports): for node
 *     i with mesh neighbours j, the flowmap gradient F is the least-squares fit of
 *     F dx_j ~ dphi_j, dx_j = x_j - x_i, dphi_j = phi_j - phi_i.  Its normal equations give
 *     F = (sum dphi dx^T)(sum dx dx^T)^-1; here it is solved by Householder QR of the k x d
 *     matrix X whose rows are dx_j^T (Golub & Van Loan, Matrix Computations, Sec. 5.2/5.3),
 *     the same minimiser by a different algorithm.
 *  3. Cauchy-Green tensor C = F^T F; its eigenvalues by the cyclic Jacobi method (Golub &
 *     Van Loan, Sec. 8.5).  mu = lambda_max(C) - 1 is taken as the largest eigenvalue of
 *     C - I (Jacobi again), so it keeps its relative accuracy when C is close to I.
 *     FTLE = ln(sqrt(lambda_max)) / |T| = log1p(mu) / (2 |T|).
 *  4. Parameter derivative d(sum_i w_i FTLE_i)/d(A, eps, omega) of the double gyre by
 *     forward-mode tangent-linear propagation through the same RK4 steps, the same QR
 *     solve, and the eigenvalue derivative d lambda = v^T dC v (v the unit eigenvector).
 *
 * Velocity fields:
 *   double gyre: f(x,t) = a x^2 + b x, a = eps sin(omega t), b = 1 - 2 eps sin(omega t),
 *                u = -pi A sin(pi f) cos(pi y),  v = pi A cos(pi f) sin(pi y) df/dx
 *   ABC:         u = A sin z + C cos y,  v = B sin x + A cos z,  w = C sin y + B cos x
 *   linear:      u = M x (M row-major d x d)
 *   saddle:      u = (x, -y) in 2D, (x, -y, 0) in 3D
 *
 * Degenerate neighbourhoods: fewer than d neighbours, or det(X^T X) <= 1e-12 (tr(X^T X)/d)^d
 * (det from the QR factor, prod R_jj^2), give FTLE = NaN and a set flag bit.
 *
 * Parallelism is over nodes only (OpenMP, static schedule); per-node arithmetic is serial
 * and identical for any thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_DOUBLE_GYRE 0
#define ORC_ABC 1
#define ORC_LINEAR 2
#define ORC_SADDLE 3

#define ORC_MAX_NBR 256
#define ORC_PI 3.14159265358979323846

#define ORC_FLAG_DEGENERATE 1

/* ------------------------------------------------------------------------- velocity */

static void velocity(int kind, const double* p, int dim, double t, const double* x, double* u) {
  if (kind == ORC_DOUBLE_GYRE) {
    double A = p[0], eps = p[1], om = p[2];
    double s = sin(om * t);
    double a = eps * s, b = 1.0 - 2.0 * eps * s;
    double f = a * x[0] * x[0] + b * x[0];
    double fx = 2.0 * a * x[0] + b;
    u[0] = -ORC_PI * A * sin(ORC_PI * f) * cos(ORC_PI * x[1]);
    u[1] = ORC_PI * A * cos(ORC_PI * f) * sin(ORC_PI * x[1]) * fx;
  } else if (kind == ORC_ABC) {
    double A = p[0], B = p[1], C = p[2];
    u[0] = A * sin(x[2]) + C * cos(x[1]);
    u[1] = B * sin(x[0]) + A * cos(x[2]);
    u[2] = C * sin(x[1]) + B * cos(x[0]);
  } else if (kind == ORC_LINEAR) {
    for (int a = 0; a < dim; ++a) {
      double s = 0.0;
      for (int b = 0; b < dim; ++b) s += p[a * dim + b] * x[b];
      u[a] = s;
    }
  } else { /* saddle */
    u[0] = x[0];
    u[1] = -x[1];
    if (dim == 3) u[2] = 0.0;
  }
}

/* Double gyre only: Jacobian J[a][b] = du_a/dx_b and parameter derivatives
 * P[a][q] = du_a/dtheta_q for theta = (A, eps, omega). */
static void dg_derivs(const double* p, double t, const double* x, double J[2][2], double P[2][3]) {
  double A = p[0], eps = p[1], om = p[2];
  double s = sin(om * t), c = cos(om * t);
  double a = eps * s, b = 1.0 - 2.0 * eps * s;
  double f = a * x[0] * x[0] + b * x[0];
  double fx = 2.0 * a * x[0] + b;
  double fxx = 2.0 * a;
  double sf = sin(ORC_PI * f), cf = cos(ORC_PI * f);
  double sy = sin(ORC_PI * x[1]), cy = cos(ORC_PI * x[1]);
  double pi = ORC_PI, pi2 = ORC_PI * ORC_PI;
  J[0][0] = -pi2 * A * cf * fx * cy;
  J[0][1] = pi2 * A * sf * sy;
  J[1][0] = pi * A * sy * (-pi * sf * fx * fx + cf * fxx);
  J[1][1] = pi2 * A * cf * cy * fx;
  /* d/dA */
  P[0][0] = -pi * sf * cy;
  P[1][0] = pi * cf * sy * fx;
  /* d/deps: df/deps = s (x^2 - 2x), d(fx)/deps = s (2x - 2) */
  double fe = s * (x[0] * x[0] - 2.0 * x[0]), fxe = s * (2.0 * x[0] - 2.0);
  P[0][1] = -pi2 * A * cf * cy * fe;
  P[1][1] = pi * A * sy * (-pi * sf * fe * fx + cf * fxe);
  /* d/domega: df/domega = eps t cos(omega t) (x^2 - 2x), d(fx)/domega = eps t cos(omega t)(2x - 2) */
  double fo = eps * t * c * (x[0] * x[0] - 2.0 * x[0]), fxo = eps * t * c * (2.0 * x[0] - 2.0);
  P[0][2] = -pi2 * A * cf * cy * fo;
  P[1][2] = pi * A * sy * (-pi * sf * fo * fx + cf * fxo);
}

int orc_velocity(int kind, const double* p, int dim, double t, const double* x, double* u) {
  if (dim < 2 || dim > 3) return -1;
  if (kind == ORC_DOUBLE_GYRE && dim != 2) return -1;
  if (kind == ORC_ABC && dim != 3) return -1;
  velocity(kind, p, dim, t, x, u);
  return 0;
}

int orc_dg_derivs(const double* p, double t, const double* x, double* J4, double* P6) {
  double J[2][2], P[2][3];
  dg_derivs(p, t, x, J, P);
  memcpy(J4, J, sizeof J);
  memcpy(P6, P, sizeof P);
  return 0;
}

/* ------------------------------------------------------------------------- RK4 */

static long n_steps(double T, double dt) { return lround(fabs(T) / fabs(dt)); }

static void rk4(int kind, const double* p, int dim, double t0, double h, long n, double* x) {
  double k1[3], k2[3], k3[3], k4[3], y[3];
  for (long k = 0; k < n; ++k) {
    double t = t0 + (double)k * h;
    velocity(kind, p, dim, t, x, k1);
    for (int a = 0; a < dim; ++a) y[a] = x[a] + 0.5 * h * k1[a];
    velocity(kind, p, dim, t + 0.5 * h, y, k2);
    for (int a = 0; a < dim; ++a) y[a] = x[a] + 0.5 * h * k2[a];
    velocity(kind, p, dim, t + 0.5 * h, y, k3);
    for (int a = 0; a < dim; ++a) y[a] = x[a] + h * k3[a];
    velocity(kind, p, dim, t + h, y, k4);
    for (int a = 0; a < dim; ++a) x[a] += h / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
  }
}

/* Flowmap of every node: x0, phi are SoA [dim][n].  Returns the step count or -1. */
long orc_advect(int kind, const double* p, int dim, int64_t n, const double* x0, double t0, double T,
                double dt, double* phi) {
  if (dim < 2 || dim > 3 || dt == 0.0 || n < 0) return -1;
  if (kind == ORC_DOUBLE_GYRE && dim != 2) return -1;
  if (kind == ORC_ABC && dim != 3) return -1;
  long ns = n_steps(T, dt);
  double h = (T < 0 ? -1.0 : 1.0) * fabs(dt);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double x[3];
    for (int a = 0; a < dim; ++a) x[a] = x0[(int64_t)a * n + i];
    rk4(kind, p, dim, t0, h, ns, x);
    for (int a = 0; a < dim; ++a) phi[(int64_t)a * n + i] = x[a];
  }
  return ns;
}

/* Double gyre flowmap and its tangents dphi/dtheta (theta = A, eps, omega):
 * dphi is [3][2][n]: dphi[(q * 2 + a) * n + i] = d phi_a(i) / d theta_q. */
long orc_advect_tangent(const double* p, int64_t n, const double* x0, double t0, double T, double dt,
                        double* phi, double* dphi) {
  if (dt == 0.0 || n < 0) return -1;
  long ns = n_steps(T, dt);
  double h = (T < 0 ? -1.0 : 1.0) * fabs(dt);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double x[2] = {x0[i], x0[n + i]};
    double X[2][3] = {{0, 0, 0}, {0, 0, 0}}; /* dx/dtheta */
    for (long k = 0; k < ns; ++k) {
      double t = t0 + (double)k * h;
      double ks[4][2], Ks[4][2][3];
      double ts[4] = {t, t + 0.5 * h, t + 0.5 * h, t + h};
      double cs[4] = {0.0, 0.5 * h, 0.5 * h, h}; /* stage offset times the previous slope */
      for (int st = 0; st < 4; ++st) {
        double y[2], Y[2][3];
        for (int a = 0; a < 2; ++a) {
          y[a] = x[a] + (st ? cs[st] * ks[st - 1][a] : 0.0);
          for (int q = 0; q < 3; ++q) Y[a][q] = X[a][q] + (st ? cs[st] * Ks[st - 1][a][q] : 0.0);
        }
        double J[2][2], P[2][3];
        velocity(ORC_DOUBLE_GYRE, p, 2, ts[st], y, ks[st]);
        dg_derivs(p, ts[st], y, J, P);
        for (int a = 0; a < 2; ++a)
          for (int q = 0; q < 3; ++q) Ks[st][a][q] = J[a][0] * Y[0][q] + J[a][1] * Y[1][q] + P[a][q];
      }
      for (int a = 0; a < 2; ++a) {
        x[a] += h / 6.0 * (ks[0][a] + 2.0 * ks[1][a] + 2.0 * ks[2][a] + ks[3][a]);
        for (int q = 0; q < 3; ++q)
          X[a][q] += h / 6.0 * (Ks[0][a][q] + 2.0 * Ks[1][a][q] + 2.0 * Ks[2][a][q] + Ks[3][a][q]);
      }
    }
    phi[i] = x[0];
    phi[n + i] = x[1];
    for (int q = 0; q < 3; ++q)
      for (int a = 0; a < 2; ++a) dphi[((int64_t)q * 2 + a) * n + i] = X[a][q];
  }
  return ns;
}

/* ------------------------------------------------------------------------- least squares */

/* Householder QR least squares, min || X Y - B || for X (k x d, row-major, overwritten) and
 * B (k x m, row-major, overwritten).  Writes Y (d x m).  Returns 0, or 1 if X is
 * rank-deficient by the determinant test in the file header. */
static int lsq_qr(int k, int d, int m, double* X, double* B, double* Y, double* detM) {
  double trM = 0.0;
  for (int r = 0; r < k * d; ++r) trM += X[r] * X[r];
  if (k < d) {
    *detM = 0.0;
    return 1;
  }
  double diag[3];
  for (int j = 0; j < d; ++j) {
    double nrm = 0.0;
    for (int r = j; r < k; ++r) nrm += X[r * d + j] * X[r * d + j];
    nrm = sqrt(nrm);
    if (nrm == 0.0) {
      diag[j] = 0.0;
      continue;
    }
    double alpha = X[j * d + j] > 0 ? -nrm : nrm;
    /* Householder vector v = x - alpha e_1, stored in place below the diagonal */
    double v[ORC_MAX_NBR];
    for (int r = j; r < k; ++r) v[r] = X[r * d + j];
    v[j] -= alpha;
    double vv = 0.0;
    for (int r = j; r < k; ++r) vv += v[r] * v[r];
    if (vv > 0.0) {
      for (int c = j; c < d; ++c) {
        double s = 0.0;
        for (int r = j; r < k; ++r) s += v[r] * X[r * d + c];
        s = 2.0 * s / vv;
        for (int r = j; r < k; ++r) X[r * d + c] -= s * v[r];
      }
      for (int c = 0; c < m; ++c) {
        double s = 0.0;
        for (int r = j; r < k; ++r) s += v[r] * B[r * m + c];
        s = 2.0 * s / vv;
        for (int r = j; r < k; ++r) B[r * m + c] -= s * v[r];
      }
    }
    diag[j] = X[j * d + j];
  }
  double det = 1.0;
  for (int j = 0; j < d; ++j) det *= diag[j] * diag[j];
  *detM = det;
  if (!(det > 1e-12 * pow(trM / d, d))) return 1;
  /* back substitution R Y = (Q^T B)[0:d] */
  for (int c = 0; c < m; ++c)
    for (int j = d - 1; j >= 0; --j) {
      double s = B[j * m + c];
      for (int l = j + 1; l < d; ++l) s -= X[j * d + l] * Y[l * m + c];
      Y[j * m + c] = s / X[j * d + j];
    }
  return 0;
}

/* ------------------------------------------------------------------------- eigenvalues */

/* Cyclic Jacobi on a symmetric d x d matrix A (overwritten by its near-diagonal form).
 * w gets the eigenvalues, V (row-major, columns = eigenvectors) the rotations' product. */
static void jacobi(int d, double A[3][3], double w[3], double V[3][3]) {
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) V[a][b] = (a == b) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, fro = 0.0;
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        fro += A[a][b] * A[a][b];
        if (a != b) off += A[a][b] * A[a][b];
      }
    if (off == 0.0 || off <= 1e-34 * fro) break;
    for (int pp = 0; pp < d - 1; ++pp)
      for (int qq = pp + 1; qq < d; ++qq) {
        double apq = A[pp][qq];
        if (apq == 0.0) continue;
        double tau = (A[qq][qq] - A[pp][pp]) / (2.0 * apq);
        double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int r = 0; r < d; ++r) { /* A <- A J */
          double arp = A[r][pp], arq = A[r][qq];
          A[r][pp] = c * arp - s * arq;
          A[r][qq] = s * arp + c * arq;
        }
        for (int r = 0; r < d; ++r) { /* A <- J^T A */
          double apr = A[pp][r], aqr = A[qq][r];
          A[pp][r] = c * apr - s * aqr;
          A[qq][r] = s * apr + c * aqr;
        }
        for (int r = 0; r < d; ++r) { /* V <- V J */
          double vrp = V[r][pp], vrq = V[r][qq];
          V[r][pp] = c * vrp - s * vrq;
          V[r][qq] = s * vrp + c * vrq;
        }
      }
  }
  for (int a = 0; a < d; ++a) w[a] = A[a][a];
}

int orc_jacobi(int d, const double* A_in, double* w, double* V_out) {
  double A[3][3], V[3][3];
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) A[a][b] = A_in[a * d + b];
  jacobi(d, A, w, V);
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) V_out[a * d + b] = V[a][b];
  return 0;
}

/* ------------------------------------------------------------------------- per-node FTLE */

/* Per node: the gradient F (solved together with optional extra right-hand sides),
 * C = F^T F, lambda_max, mu and the unit eigenvector of lambda_max.  Returns 0 or 1
 * (degenerate).  extra: m_extra columns per neighbour row (k x m_extra, row-major), solved
 * into Yextra (d x m_extra). */
static int node_ftle(int d, int k, const double* dx, const double* dphi, int m_extra,
                     const double* dextra, double F[3][3], double* lam, double* mu, double vmax[3],
                     double* Yextra, double* detM) {
  double X[ORC_MAX_NBR * 3];
  int m = d + m_extra; /* at most 3 + 6 */
  double B[ORC_MAX_NBR * 9];
  double Y[3 * 9];
  memcpy(X, dx, sizeof(double) * (size_t)k * (size_t)d);
  for (int r = 0; r < k; ++r) {
    for (int c = 0; c < d; ++c) B[r * m + c] = dphi[r * d + c];
    for (int c = 0; c < m_extra; ++c) B[r * m + d + c] = dextra[r * m_extra + c];
  }
  int deg = lsq_qr(k, d, m, X, B, Y, detM);
  if (deg) return 1;
  /* Y[0:d, 0:d] = F^T */
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) F[a][b] = Y[b * m + a];
  for (int b = 0; b < d; ++b)
    for (int c = 0; c < m_extra; ++c) Yextra[b * m_extra + c] = Y[b * m + d + c];
  double C[3][3], E[3][3], w[3], V[3][3], we[3], Ve[3][3];
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double s = 0.0;
      for (int c = 0; c < d; ++c) s += F[c][a] * F[c][b];
      C[a][b] = s;
      E[a][b] = s - (a == b ? 1.0 : 0.0);
    }
  jacobi(d, C, w, V);
  jacobi(d, E, we, Ve);
  int im = 0, ie = 0;
  for (int a = 1; a < d; ++a) {
    if (w[a] > w[im]) im = a;
    if (we[a] > we[ie]) ie = a;
  }
  *lam = w[im];
  *mu = we[ie];
  for (int a = 0; a < d; ++a) vmax[a] = V[a][im];
  return 0;
}

/* FTLE of every CSR row.  x, phi: SoA [dim][n] (FP64).  Outputs (nullable except ftle):
 * ftle[n], lam[n], mu[n], Fout[n][dim*dim] (row-major F per node), flags[n].
 * Returns the number of degenerate rows, or -1 on bad arguments. */
int64_t orc_ftle(int dim, int64_t n, const double* x, const int32_t* row_ptr, const int32_t* col_idx,
                 const double* phi, double T, double* ftle, double* lam, double* mu, double* Fout,
                 int32_t* flags) {
  if (dim < 2 || dim > 3 || n < 0 || T == 0.0) return -1;
  for (int64_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] - row_ptr[i] < 0 || row_ptr[i + 1] - row_ptr[i] > ORC_MAX_NBR) return -1;
  int64_t ndeg = 0;
#pragma omp parallel for schedule(static) reduction(+ : ndeg)
  for (int64_t i = 0; i < n; ++i) {
    int k = row_ptr[i + 1] - row_ptr[i];
    double F[3][3] = {{0}}, l = NAN, m_ = NAN, v[3], detM = 0.0;
    int deg = 1;
    {
      double dx[ORC_MAX_NBR * 3], dp[ORC_MAX_NBR * 3];
      for (int r = 0; r < k; ++r) {
        int64_t j = col_idx[row_ptr[i] + r];
        for (int a = 0; a < dim; ++a) {
          dx[r * dim + a] = x[(int64_t)a * n + j] - x[(int64_t)a * n + i];
          dp[r * dim + a] = phi[(int64_t)a * n + j] - phi[(int64_t)a * n + i];
        }
      }
      deg = node_ftle(dim, k, dx, dp, 0, NULL, F, &l, &m_, v, NULL, &detM);
    }
    if (deg) {
      ndeg += 1;
      l = NAN;
      m_ = NAN;
    }
    ftle[i] = deg ? NAN : log1p(m_) / (2.0 * fabs(T));
    if (lam) lam[i] = l;
    if (mu) mu[i] = m_;
    if (Fout)
      for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) Fout[i * dim * dim + a * dim + b] = deg ? NAN : F[a][b];
    if (flags) flags[i] = deg ? ORC_FLAG_DEGENERATE : 0;
  }
  return ndeg;
}

/* d(sum_i w_i FTLE_i)/d(A, eps, omega) for the double gyre (2D), forward mode.
 * x0: SoA [2][n] initial nodes (FP64); w[n] weights (rows with w = 0 are skipped);
 * grad[3] out; ftle[n] out (nullable).  Returns 0, 1 if a weighted row is degenerate, -1 on
 * bad arguments. */
int orc_param_grad(int64_t n, const double* x0, const int32_t* row_ptr, const int32_t* col_idx,
                   const double* p, double t0, double T, double dt, const double* w, double* grad,
                   double* ftle) {
  if (n < 0 || T == 0.0 || dt == 0.0) return -1;
  for (int64_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] - row_ptr[i] < 0 || row_ptr[i + 1] - row_ptr[i] > ORC_MAX_NBR) return -1;
  double* phi = (double*)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
  double* dphi = (double*)malloc(sizeof(double) * 6 * (size_t)(n > 0 ? n : 1));
  orc_advect_tangent(p, n, x0, t0, T, dt, phi, dphi);
  double g0 = 0.0, g1 = 0.0, g2 = 0.0;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : g0, g1, g2) reduction(| : bad)
  for (int64_t i = 0; i < n; ++i) {
    int k = row_ptr[i + 1] - row_ptr[i];
    double F[3][3], l = NAN, m_ = NAN, v[3], detM, Yx[2 * 6];
    int deg = 1;
    if (w[i] != 0.0 || ftle) {
      double dx[ORC_MAX_NBR * 2], dp[ORC_MAX_NBR * 2], de[ORC_MAX_NBR * 6];
      for (int r = 0; r < k; ++r) {
        int64_t j = col_idx[row_ptr[i] + r];
        for (int a = 0; a < 2; ++a) {
          dx[r * 2 + a] = x0[(int64_t)a * n + j] - x0[(int64_t)a * n + i];
          dp[r * 2 + a] = phi[(int64_t)a * n + j] - phi[(int64_t)a * n + i];
        }
        /* extra right-hand sides: column (q * 2 + a) holds d(dphi_a)/d theta_q */
        for (int q = 0; q < 3; ++q)
          for (int a = 0; a < 2; ++a)
            de[r * 6 + q * 2 + a] = dphi[((int64_t)q * 2 + a) * n + j] - dphi[((int64_t)q * 2 + a) * n + i];
      }
      deg = node_ftle(2, k, dx, dp, 6, de, F, &l, &m_, v, Yx, &detM);
    }
    if (ftle) ftle[i] = deg ? NAN : log1p(m_) / (2.0 * fabs(T));
    if (w[i] == 0.0) continue;
    if (deg) {
      bad |= 1;
      continue;
    }
    /* dF_q^T = Yx[:, q*2 : q*2+2]  ->  dF_q[a][b] = Yx[b * 6 + q * 2 + a];
     * d lambda = 2 (F v) . (dF v);  d FTLE = d lambda / (2 |T| lambda) */
    double Fv[2] = {F[0][0] * v[0] + F[0][1] * v[1], F[1][0] * v[0] + F[1][1] * v[1]};
    double gq[3];
    for (int q = 0; q < 3; ++q) {
      double dFv[2];
      for (int a = 0; a < 2; ++a)
        dFv[a] = Yx[0 * 6 + q * 2 + a] * v[0] + Yx[1 * 6 + q * 2 + a] * v[1];
      double dlam = 2.0 * (Fv[0] * dFv[0] + Fv[1] * dFv[1]);
      gq[q] = w[i] * dlam / (2.0 * fabs(T) * l);
    }
    g0 += gq[0];
    g1 += gq[1];
    g2 += gq[2];
  }
  grad[0] = g0;
  grad[1] = g1;
  grad[2] = g2;
  free(phi);
  free(dphi);
  return bad ? 1 : 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
