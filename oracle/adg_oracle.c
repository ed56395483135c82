/*
 * adg_oracle.c -- plain FP64 CPU ADER-DG.  TEST INFRASTRUCTURE ONLY: the tests,
 * the smoke check and the benchmark's CPU-baseline leg are its only users; the
 * CUDA library never links, loads or calls it, and it shares no code with it.
 *
 * Everything is written in the order and notation of arXiv 2504.06889, Sec. 3:
 * no blocking, fusion or reordering beyond what the equations state.  Loops are
 * over (cell, time node k, variable v, spatial node i) in the obvious way.
 *
 * Readings where the paper is silent (listed with the design notes):
 *   - reference element [0,1]^d in space and [0,1] in time, GL support points;
 *   - Picard starts from q = Q^n constant in time and runs a fixed number of
 *     sweeps (default N+1);
 *   - the Riemann problem is solved once per face on the time-averaged traces;
 *     the Rusanov speed is one scalar per face: max over face nodes and sides;
 *   - dt^n is computed from Q^n with eq. (CFL_condition), C_CFL given, d kept.
 */
#include "adg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* 1D tables.  Sec. 3, eq. (piecewise_solution): Lagrange polynomials with    */
/* Gauss-Legendre support points.  GL nodes by Newton on P_n (long double).   */
/* ------------------------------------------------------------------------ */

static void legendre_and_deriv(int n, long double x, long double* P, long double* dP) {
  long double p0 = 1.0L, p1 = x;
  if (n == 0) {
    *P = 1.0L;
    *dP = 0.0L;
    return;
  }
  for (int k = 1; k < n; ++k) {
    long double p2 = ((2.0L * k + 1.0L) * x * p1 - (long double)k * p0) / (k + 1.0L);
    p0 = p1;
    p1 = p2;
  }
  *P = p1;                                  /* P_n   */
  *dP = n * (x * p1 - p0) / (x * x - 1.0L); /* P_n'  */
}

double or_lagrange(int n, const double* xi, int j, double x) {
  double r = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != j) r *= (x - xi[m]) / (xi[j] - xi[m]);
  return r;
}

/* psi_j'(x) by the product rule: sum over l != j of 1/(xi_j-xi_l) * prod_{m != j,l} */
static long double lagrange_deriv(int n, const long double* xi, int j, long double x) {
  long double s = 0.0L;
  for (int l = 0; l < n; ++l) {
    if (l == j) continue;
    long double t = 1.0L / (xi[j] - xi[l]);
    for (int m = 0; m < n; ++m)
      if (m != j && m != l) t *= (x - xi[m]) / (xi[j] - xi[m]);
    s += t;
  }
  return s;
}

static long double lagrange_ld(int n, const long double* xi, int j, long double x) {
  long double r = 1.0L;
  for (int m = 0; m < n; ++m)
    if (m != j) r *= (x - xi[m]) / (xi[j] - xi[m]);
  return r;
}

void or_tables(int n, double* xi, double* w, double* D, double* psi0, double* psi1, double* K1,
               double* K1inv) {
  long double X[OR_MAXN], W[OR_MAXN];
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int j = 0; j < n; ++j) {
    /* standard initial guess, then Newton on [-1,1] */
    long double x = cosl(pi * (j + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      long double P, dP;
      legendre_and_deriv(n, x, &P, &dP);
      long double dx = P / dP;
      x -= dx;
      if (fabsl(dx) < 1e-19L) break;
    }
    long double P, dP;
    legendre_and_deriv(n, x, &P, &dP);
    long double wstd = 2.0L / ((1.0L - x * x) * dP * dP);
    /* map [-1,1] -> [0,1]; cos ordering is descending, store ascending */
    X[n - 1 - j] = (x + 1.0L) / 2.0L;
    W[n - 1 - j] = wstd / 2.0L;
  }
  for (int j = 0; j < n; ++j) {
    xi[j] = (double)X[j];
    w[j] = (double)W[j];
    psi0[j] = (double)lagrange_ld(n, X, j, 0.0L);
    psi1[j] = (double)lagrange_ld(n, X, j, 1.0L);
  }
  /* D[a][b] = psi_b'(xi_a) */
  long double Dl[OR_MAXN][OR_MAXN];
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      Dl[a][b] = lagrange_deriv(n, X, b, X[a]);
      D[a * n + b] = (double)Dl[a][b];
    }
  /* Eq. (Picard), time part divided by the spatial mass:
   *   K1[k][l] = psi_k(1) psi_l(1) - int_0^1 psi_k'(tau) psi_l(tau) dtau
   *            = psi_k(1) psi_l(1) - w_l psi_k'(xi_l)        (GL exact for degree 2N-1) */
  long double A[OR_MAXN][2 * OR_MAXN];
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) {
      long double v = lagrange_ld(n, X, k, 1.0L) * lagrange_ld(n, X, l, 1.0L) - W[l] * Dl[l][k];
      K1[k * n + l] = (double)v;
      A[k][l] = v;
      A[k][n + l] = (k == l) ? 1.0L : 0.0L;
    }
  /* Gauss-Jordan with partial pivoting */
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r][c]) > fabsl(A[p][c])) p = r;
    if (p != c)
      for (int j = 0; j < 2 * n; ++j) {
        long double t = A[c][j];
        A[c][j] = A[p][j];
        A[p][j] = t;
      }
    long double piv = A[c][c];
    for (int j = 0; j < 2 * n; ++j) A[c][j] /= piv;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      long double f = A[r][c];
      if (f != 0.0L)
        for (int j = 0; j < 2 * n; ++j) A[r][j] -= f * A[c][j];
    }
  }
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) K1inv[k * n + l] = (double)A[k][n + l];
}

/* ------------------------------------------------------------------------ */
/* Mesh setup                                                                 */
/* ------------------------------------------------------------------------ */

int or_nvar(int pde, int dim) {
  switch (pde) {
    case OR_ACOUSTIC: return 1 + dim;          /* p, v_1..v_d */
    case OR_ELASTIC: return dim == 3 ? 9 : 5;  /* stresses (Voigt), velocities */
    case OR_EULER: return 2 + dim;             /* rho, rho v_1..v_d, E */
    case OR_SWE: return 3;                     /* h, hu, hv (flat bathymetry) */
    case OR_SWE_B: return 4;                   /* h, hu, hv, b (Sec. 5.4) */
  }
  return -1;
}

int or_setup(or_mesh* M, int dim, int N, const int* m, const double* lo, const double* hi, int pde,
             const double* params, int nparams, double cfl, int picard_iters) {
  memset(M, 0, sizeof(*M));
  if (dim < 2 || dim > 3 || N < 0 || N + 1 > OR_MAXN) return -1;
  if ((pde == OR_SWE || pde == OR_SWE_B) && dim != 2) return -1;
  M->dim = dim;
  M->N = N;
  M->n = N + 1;
  M->pde = pde;
  M->nvar = or_nvar(pde, dim);
  for (int d = 0; d < 3; ++d) {
    M->m[d] = d < dim ? m[d] : 1;
    M->lo[d] = d < dim ? lo[d] : 0.0;
    M->h[d] = d < dim ? (hi[d] - lo[d]) / m[d] : 1.0;
  }
  for (int j = 0; j < nparams && j < 8; ++j) M->pp[j] = params[j];
  M->cfl = cfl;
  M->picard_iters = picard_iters > 0 ? picard_iters : N + 1;
  M->picard_tol = 0.0;
  M->use_ck = 0;
  M->storage = OR_ST_FP64;
  M->cell_c = NULL;
  /* or_tables stores n x n matrices with row stride n; the mesh keeps stride OR_MAXN */
  {
    double D[OR_MAXN * OR_MAXN], K1[OR_MAXN * OR_MAXN], K1i[OR_MAXN * OR_MAXN];
    or_tables(M->n, M->xi, M->w, D, M->psi0, M->psi1, K1, K1i);
    int n = M->n;
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        M->D[a][b] = D[a * n + b];
        M->K1[a][b] = K1[a * n + b];
        M->K1inv[a][b] = K1i[a * n + b];
      }
  }
  return 0;
}

void or_set_cell_c(or_mesh* M, const double* cell_c) { M->cell_c = cell_c; }

/* ------------------------------------------------------------------------ */
/* PDE fluxes, Sec. 5.  F_dir(q) and the spectral radius of dF_dir/dq.        */
/* ------------------------------------------------------------------------ */

void or_flux(const or_mesh* M, int cell, const double* q, int dir, double* F) {
  const int V = M->nvar, d = M->dim;
  for (int v = 0; v < V; ++v) F[v] = 0.0;
  if (M->pde == OR_ACOUSTIC) {
    /* eq. (acoustic): p_t + K div v = 0, rho v_t + grad p = 0;  F_dir = A_dir Q */
    double rho = M->pp[0], K = M->pp[1];
    if (M->cell_c) K = rho * M->cell_c[cell] * M->cell_c[cell];
    F[0] = K * q[1 + dir];
    F[1 + dir] = q[0] / rho;
  } else if (M->pde == OR_ELASTIC) {
    /* eq. (lin_elastic) with the matrices of eq. (elastic_matrices); the 3D
     * velocity-stress system is the same construction in three directions. */
    double rho = M->pp[0], cp = M->pp[1], cs = M->pp[2];
    double mu = rho * cs * cs, lam = rho * cp * cp - 2.0 * mu;
    if (d == 2) {
      /* Q = (sxx, syy, sxy, vx, vy) */
      double sxx = q[0], syy = q[1], sxy = q[2], vx = q[3], vy = q[4];
      if (dir == 0) {
        F[0] = -(lam + 2.0 * mu) * vx;
        F[1] = -lam * vx;
        F[2] = -mu * vy;
        F[3] = -sxx / rho;
        F[4] = -sxy / rho;
      } else {
        F[0] = -lam * vy;
        F[1] = -(lam + 2.0 * mu) * vy;
        F[2] = -mu * vx;
        F[3] = -sxy / rho;
        F[4] = -syy / rho;
      }
    } else {
      /* Q = (sxx, syy, szz, sxy, syz, sxz, vx, vy, vz) */
      double s[3][3];
      s[0][0] = q[0];
      s[1][1] = q[1];
      s[2][2] = q[2];
      s[0][1] = s[1][0] = q[3];
      s[1][2] = s[2][1] = q[4];
      s[0][2] = s[2][0] = q[5];
      const double* vel = q + 6;
      /* sigma_t = lam (div v) I + mu (grad v + grad v^T); flux along dir carries
       * -(lam v_dir I + mu (e_dir v^T + v e_dir^T)) */
      double T[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double e_a = (a == dir) ? 1.0 : 0.0, e_b = (b == dir) ? 1.0 : 0.0;
          T[a][b] = -((a == b ? lam * vel[dir] : 0.0) + mu * (e_a * vel[b] + vel[a] * e_b));
        }
      F[0] = T[0][0];
      F[1] = T[1][1];
      F[2] = T[2][2];
      F[3] = T[0][1];
      F[4] = T[1][2];
      F[5] = T[0][2];
      /* rho v_t = div sigma: flux along dir is -sigma[:,dir]/rho */
      for (int a = 0; a < 3; ++a) F[6 + a] = -s[a][dir] / rho;
    }
  } else if (M->pde == OR_EULER) {
    /* eq. (euler_eq): Q = (rho, rho v, E), p = (gamma-1)(E - rho |v|^2 / 2),
     * F_dir = (rho v_dir, rho v v_dir + p e_dir, v_dir (E + p)) */
    double gamma = M->pp[0];
    double rho = q[0], E = q[1 + d];
    double vel[3] = {0, 0, 0}, v2 = 0.0;
    for (int a = 0; a < d; ++a) {
      vel[a] = q[1 + a] / rho;
      v2 += vel[a] * vel[a];
    }
    double p = (gamma - 1.0) * (E - 0.5 * rho * v2);
    F[0] = q[1 + dir];
    for (int a = 0; a < d; ++a) F[1 + a] = q[1 + a] * vel[dir] + (a == dir ? p : 0.0);
    F[1 + d] = vel[dir] * (E + p);
  } else if (M->pde == OR_SWE) {
    /* Sec. 5.4 with flat bathymetry: the hydrostatic non-conservative term
     * g h grad(b + h) reduces to grad(g h^2 / 2), so F_dir = (h v_dir,
     * h v v_dir + g h^2/2 e_dir) */
    double g = M->pp[0];
    double h = q[0];
    double vel[2] = {q[1] / h, q[2] / h};
    F[0] = q[1 + dir];
    for (int a = 0; a < 2; ++a) F[1 + a] = q[1 + a] * vel[dir] + (a == dir ? 0.5 * g * h * h : 0.0);
  } else if (M->pde == OR_SWE_B) {
    /* eq. (swe_cons): G = (h v_x, h v_x^2, h v_x v_y, 0), H likewise; the hydrostatic
     * pressure is in the non-conservative product (or_ncp) */
    double h = q[0];
    double vel[2] = {q[1] / h, q[2] / h};
    F[0] = q[1 + dir];
    for (int a = 0; a < 2; ++a) F[1 + a] = q[1 + a] * vel[dir];
    F[3] = 0.0;
  }
}

/* eq. (swe_noncons): C(Q) (along x) and D(Q) (along y) have the single nonzero row of the
 * momentum along that direction, (g h, 0, 0, g h): B_dir(q) dq = g h (dh + db) e_{1+dir} */
void or_ncp(const or_mesh* M, const double* q, int dir, const double* dq, double* out) {
  for (int v = 0; v < M->nvar; ++v) out[v] = 0.0;
  if (M->pde != OR_SWE_B) return;
  double g = M->pp[0];
  out[1 + dir] = g * q[0] * dq[0] + g * q[0] * dq[3];
}

double or_speed(const or_mesh* M, int cell, const double* q, int dir) {
  const int d = M->dim;
  if (M->pde == OR_ACOUSTIC) {
    double rho = M->pp[0], K = M->pp[1];
    if (M->cell_c) return fabs(M->cell_c[cell]);
    return sqrt(K / rho);
  }
  if (M->pde == OR_ELASTIC) {
    return fabs(M->pp[1]); /* c_p is the largest elastic wave speed */
  }
  if (M->pde == OR_EULER) {
    double gamma = M->pp[0];
    double rho = q[0], E = q[1 + d], v2 = 0.0;
    for (int a = 0; a < d; ++a) v2 += (q[1 + a] / rho) * (q[1 + a] / rho);
    double p = (gamma - 1.0) * (E - 0.5 * rho * v2);
    return fabs(q[1 + dir] / rho) + sqrt(gamma * p / rho);
  }
  if (M->pde == OR_SWE || M->pde == OR_SWE_B) {
    double g = M->pp[0];
    return fabs(q[1 + dir] / q[0]) + sqrt(g * q[0]);
  }
  return 0.0;
}

/* ------------------------------------------------------------------------ */
/* Exact solutions / initial data (Sec. 5 scenarios and the synthetic ones)  */
/* ------------------------------------------------------------------------ */

void or_exact(const or_mesh* M, int scen, const double* sp, int nsp, const double* x, double t,
              double* Q) {
  const int V = M->nvar, d = M->dim;
  (void)nsp;
  for (int v = 0; v < V; ++v) Q[v] = 0.0;
  if (scen == OR_SC_PLANAR) {
    /* sp = [Q0[V], nw, {amp, kx, ky, kz, omega, r[V]} x nw];
     * Q = Q0 + sum amp sin(k.x - omega t) r  (planar wave, Sec. 5.2.1) */
    for (int v = 0; v < V; ++v) Q[v] = sp[v];
    int nw = (int)sp[V];
    const double* p = sp + V + 1;
    for (int j = 0; j < nw; ++j, p += 5 + V) {
      double kx = 0.0;
      for (int a = 0; a < d; ++a) kx += p[1 + a] * x[a];
      double s = p[0] * sin(kx - p[4] * t);
      for (int v = 0; v < V; ++v) Q[v] += s * p[5 + v];
    }
  } else if (scen == OR_SC_EULER_WAVE) {
    /* sp = [rho0, A, k[3], u[3], p0]: rho = rho0 + A sin(k.(x - u t)), constant u, p */
    double gamma = M->pp[0];
    double ph = 0.0, u2 = 0.0;
    for (int a = 0; a < d; ++a) {
      ph += sp[2 + a] * (x[a] - sp[5 + a] * t);
      u2 += sp[5 + a] * sp[5 + a];
    }
    double rho = sp[0] + sp[1] * sin(ph);
    Q[0] = rho;
    for (int a = 0; a < d; ++a) Q[1 + a] = rho * sp[5 + a];
    Q[1 + d] = sp[8] / (gamma - 1.0) + 0.5 * rho * u2;
  } else if (scen == OR_SC_SWE_MODES) {
    /* sp = [h0, a0, kx0, ky0, nm, {a, kx, ky, phi} x nm], at rest (t ignored:
     * this scenario has no closed form for t > 0) */
    double h = sp[0] + sp[1] * sin(sp[2] * x[0]) * sin(sp[3] * x[1]);
    int nm = (int)sp[4];
    const double* p = sp + 5;
    for (int j = 0; j < nm; ++j, p += 4) h += p[0] * sin(p[1] * x[0] + p[2] * x[1] + p[3]);
    Q[0] = h;
  } else if (scen == OR_SC_EULER_BELL) {
    /* Sec. 5.3.1: sp = [rho0, amp, width, x0, y0, ux, uy, p0]; rho = rho0 (1 + amp
     * exp(-width |x - x0 - u t|^2)) (the squared exponent of the figure; nearest periodic
     * image), velocity u, pressure p0: an exact solution of the Euler equations */
    double gamma = M->pp[0], r2 = 0.0, u2 = 0.0;
    for (int a = 0; a < 2; ++a) {
      double L = M->h[a] * M->m[a];
      double dx = x[a] - sp[3 + a] - sp[5 + a] * t;
      dx -= L * floor(dx / L + 0.5);
      r2 += dx * dx;
      u2 += sp[5 + a] * sp[5 + a];
    }
    double rho = sp[0] * (1.0 + sp[1] * exp(-sp[2] * r2));
    Q[0] = rho;
    Q[1] = rho * sp[5];
    Q[2] = rho * sp[6];
    Q[3] = sp[7] / (gamma - 1.0) + 0.5 * rho * u2;
  } else if (scen == OR_SC_EULER_VORTEX) {
    /* Sec. 5.3.2 (Hu and Shu's isentropic vortex): sp = [rho_inf, p_inf, beta, x0, y0, u_inf,
     * v_inf]; with r the distance to the centre x0 + u_inf t (nearest periodic image):
     * dT = (1 - gamma) beta^2 / (8 gamma pi^2) e^(1 - r^2), rho = rho_inf + (1 + dT)^(1/(gamma-1))
     * - 1, p = p_inf + (1 + dT)^(gamma/(gamma-1)) - 1 (the printed dp repeats drho; this is the
     * isentropic form, p / rho^gamma = 1 for rho_inf = p_inf = 1), (du, dv) = beta / (2 pi)
     * e^((1 - r^2)/2) (-y, x) */
    double gamma = M->pp[0], d[2], r2 = 0.0;
    for (int a = 0; a < 2; ++a) {
      double L = M->h[a] * M->m[a];
      d[a] = x[a] - sp[3 + a] - sp[5 + a] * t;
      d[a] -= L * floor(d[a] / L + 0.5);
      r2 += d[a] * d[a];
    }
    const double pi = 3.14159265358979323846;
    double dT = (1.0 - gamma) * sp[2] * sp[2] / (8.0 * gamma * pi * pi) * exp(1.0 - r2);
    double rho = sp[0] + (pow(1.0 + dT, 1.0 / (gamma - 1.0)) - 1.0);
    double p = sp[1] + (pow(1.0 + dT, gamma / (gamma - 1.0)) - 1.0);
    double f = sp[2] / (2.0 * pi) * exp(0.5 * (1.0 - r2));
    double u = sp[5] - d[1] * f, v = sp[6] + d[0] * f;
    Q[0] = rho;
    Q[1] = rho * u;
    Q[2] = rho * v;
    Q[3] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v);
  } else if (scen == OR_SC_LAKE) {
    /* eq. (lake_initial) with an optional disturbed surface: sp = [eta0, b0, ab, kbx, kby,
     * nm, {a, kx, ky, phi} x nm]; b = b0 + ab sin(kbx x + kby y), eta = eta0 + sum a
     * sin(k.x + phi), h = eta - b, v = 0.  With nm = 0 the lake is at rest for all t. */
    double b = sp[1] + sp[2] * sin(sp[3] * x[0] + sp[4] * x[1]);
    double eta = sp[0];
    int nm = (int)sp[5];
    const double* p = sp + 6;
    for (int j = 0; j < nm; ++j, p += 4) eta += p[0] * sin(p[1] * x[0] + p[2] * x[1] + p[3]);
    Q[0] = eta - b;
    Q[3] = b;
  } else if (scen == OR_SC_GAUSS_PULSE) {
    /* sp = [x0[3], sigma, amp]: p = amp exp(-|x - x0|^2 / (2 sigma^2)), periodic
     * distance on the mesh box, v = 0 (t ignored) */
    double r2 = 0.0;
    for (int a = 0; a < d; ++a) {
      double L = M->h[a] * M->m[a];
      double dx = x[a] - sp[a];
      dx -= L * floor(dx / L + 0.5);
      r2 += dx * dx;
    }
    Q[0] = sp[4] * exp(-r2 / (2.0 * sp[3] * sp[3]));
  }
}

static void node_coords(const or_mesh* M, int c, int i, double* x) {
  int cc[3] = {c % M->m[0], (c / M->m[0]) % M->m[1], c / (M->m[0] * M->m[1])};
  int ii[3] = {i % M->n, (i / M->n) % M->n, i / (M->n * M->n)};
  for (int a = 0; a < 3; ++a) x[a] = a < M->dim ? M->lo[a] + (cc[a] + M->xi[ii[a]]) * M->h[a] : 0.0;
}

static int ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

static int ncells(const or_mesh* M) { return M->m[0] * M->m[1] * M->m[2]; }

/* Sec. 5.5: Q_h^* interpolates the exact solution at the GL nodes */
void or_interpolate(const or_mesh* M, int scen, const double* sp, int nsp, double t, double* Q) {
  const int V = M->nvar, NS = ipow(M->n, M->dim), C = ncells(M);
#pragma omp parallel for schedule(static)
  for (int c = 0; c < C; ++c)
    for (int i = 0; i < NS; ++i) {
      double x[3], q[OR_MAXV];
      node_coords(M, c, i, x);
      or_exact(M, scen, sp, nsp, x, t, q);
      for (int v = 0; v < V; ++v) Q[((size_t)c * V + v) * NS + i] = q[v];
    }
}

static double node_weight(const or_mesh* M, int i) {
  double W = 1.0;
  int r = i;
  for (int a = 0; a < M->dim; ++a) {
    W *= M->w[r % M->n];
    r /= M->n;
  }
  return W;
}

/* eq. (L2gauss): sqrt(sum_c sum_i sum_v V_c w_i (Q*_v - Q_h,v)^2), per variable
 * in out[0..V-1] and over all variables in out[V]. */
void or_l2_error(const or_mesh* M, const double* Q, int scen, const double* sp, int nsp, double t,
                 double* out) {
  const int V = M->nvar, NS = ipow(M->n, M->dim), C = ncells(M);
  double Vc = 1.0;
  for (int a = 0; a < M->dim; ++a) Vc *= M->h[a];
  double acc[OR_MAXV] = {0};
  for (int c = 0; c < C; ++c)
    for (int i = 0; i < NS; ++i) {
      double x[3], q[OR_MAXV];
      node_coords(M, c, i, x);
      or_exact(M, scen, sp, nsp, x, t, q);
      double W = node_weight(M, i);
      for (int v = 0; v < V; ++v) {
        double e = q[v] - Q[((size_t)c * V + v) * NS + i];
        acc[v] += Vc * W * e * e;
      }
    }
  double tot = 0.0;
  for (int v = 0; v < V; ++v) {
    out[v] = sqrt(acc[v]);
    tot += acc[v];
  }
  out[V] = sqrt(tot);
}

/* the same norm between two discrete states */
void or_l2_diff(const or_mesh* M, const double* Qa, const double* Qb, double* out) {
  const int V = M->nvar, NS = ipow(M->n, M->dim), C = ncells(M);
  double Vc = 1.0;
  for (int a = 0; a < M->dim; ++a) Vc *= M->h[a];
  double acc[OR_MAXV] = {0};
  for (int c = 0; c < C; ++c)
    for (int i = 0; i < NS; ++i) {
      double W = node_weight(M, i);
      for (int v = 0; v < V; ++v) {
        size_t o = ((size_t)c * V + v) * NS + i;
        double e = Qa[o] - Qb[o];
        acc[v] += Vc * W * e * e;
      }
    }
  double tot = 0.0;
  for (int v = 0; v < V; ++v) {
    out[v] = sqrt(acc[v]);
    tot += acc[v];
  }
  out[V] = sqrt(tot);
}

/* integral of each variable over the domain (GL quadrature, exact for Q_h) */
void or_totals(const or_mesh* M, const double* Q, double* tot) {
  const int V = M->nvar, NS = ipow(M->n, M->dim), C = ncells(M);
  double Vc = 1.0;
  for (int a = 0; a < M->dim; ++a) Vc *= M->h[a];
  for (int v = 0; v < V; ++v) tot[v] = 0.0;
  for (int c = 0; c < C; ++c)
    for (int v = 0; v < V; ++v)
      for (int i = 0; i < NS; ++i) tot[v] += Vc * node_weight(M, i) * Q[((size_t)c * V + v) * NS + i];
}

/* ------------------------------------------------------------------------ */
/* Predictor, Sec. 3.1.  Eq. (Picard) divided by the spatial mass h^d prod w: */
/*   sum_l K1[k][l] q_{l,i} + dt w_k R_{k,i} = psi_k(0) Q_i,                  */
/*   R_{k,i} = sum_dir (1/h_dir) sum_a D[i_dir][a] F_dir(q_{k, i[dir<-a]}).    */
/* Picard: q^(r) = K1^{-1} (psi(0) Q - dt w o R(q^(r-1))), q^(0) = Q.          */
/* ------------------------------------------------------------------------ */

static int node_dir_index(const or_mesh* M, int i, int dir) { return (i / ipow(M->n, dir)) % M->n; }

static int node_with(const or_mesh* M, int i, int dir, int a) {
  int s = ipow(M->n, dir);
  return i - node_dir_index(M, i, dir) * s + a * s;
}

/* derivative along dir of every variable of the state polynomial qs[v*NS+i] at node i,
 * including 1/h_dir */
static void ncp_state_derivative(const or_mesh* M, const double* qs, int i, int dir, double* dq) {
  const int V = M->nvar, NS = ipow(M->n, M->dim);
  int idir = node_dir_index(M, i, dir);
  for (int v = 0; v < V; ++v) {
    double s = 0.0;
    for (int a = 0; a < M->n; ++a) s += M->D[idir][a] * qs[v * NS + node_with(M, i, dir, a)];
    dq[v] = s / M->h[dir];
  }
}

/* R[(k*V+v)*NS+i] for the space-time field q[(k*V+v)*NS+i] */
static void space_derivative_of_flux(const or_mesh* M, int cell, const double* q, int nt,
                                     double* R) {
  const int n = M->n, V = M->nvar, d = M->dim, NS = ipow(n, d);
  double* F = (double*)malloc(sizeof(double) * (size_t)nt * d * V * NS);
  for (int k = 0; k < nt; ++k)
    for (int i = 0; i < NS; ++i) {
      double qv[OR_MAXV], Fv[OR_MAXV];
      for (int v = 0; v < V; ++v) qv[v] = q[(k * V + v) * NS + i];
      for (int dir = 0; dir < d; ++dir) {
        or_flux(M, cell, qv, dir, Fv);
        for (int v = 0; v < V; ++v) F[((k * d + dir) * V + v) * NS + i] = Fv[v];
      }
    }
  (void)n;
  for (int k = 0; k < nt; ++k)
    for (int v = 0; v < V; ++v)
      for (int i = 0; i < NS; ++i) {
        double r = 0.0;
        for (int dir = 0; dir < d; ++dir) {
          double s = 0.0;
          int idir = node_dir_index(M, i, dir);
          for (int a = 0; a < M->n; ++a)
            s += M->D[idir][a] * F[((k * d + dir) * V + v) * NS + node_with(M, i, dir, a)];
          r += s / M->h[dir];
        }
        R[(k * V + v) * NS + i] = r;
      }
  /* non-conservative product, eq. (swe_canonical): R += sum_dir B_dir(q) dq/dx_dir, the
   * derivative of the state polynomial taken at the node */
  if (M->pde == OR_SWE_B)
    for (int k = 0; k < nt; ++k)
      for (int i = 0; i < NS; ++i) {
        double qv[OR_MAXV];
        for (int v = 0; v < V; ++v) qv[v] = q[(k * V + v) * NS + i];
        for (int dir = 0; dir < d; ++dir) {
          double dq[OR_MAXV], b[OR_MAXV];
          ncp_state_derivative(M, q + (size_t)k * V * NS, i, dir, dq);
          or_ncp(M, qv, dir, dq, b);
          for (int v = 0; v < V; ++v) R[(k * V + v) * NS + i] += b[v];
        }
      }
  free(F);
}

int or_predictor_cell(const or_mesh* M, int cell, const double* Qc, double dt, int iters,
                      double* q) {
  const int n = M->n, V = M->nvar, NS = ipow(n, M->dim);
  for (int k = 0; k < n; ++k)
    for (int v = 0; v < V; ++v)
      for (int i = 0; i < NS; ++i) q[(k * V + v) * NS + i] = Qc[v * NS + i];
  double* R = (double*)malloc(sizeof(double) * (size_t)n * V * NS);
  int r = 0;
  while (r < iters) {
    space_derivative_of_flux(M, cell, q, n, R);
    double change = 0.0; /* max |q^(r+1) - q^(r)| over the cell's space-time DOFs */
    for (int v = 0; v < V; ++v)
      for (int i = 0; i < NS; ++i) {
        double rhs[OR_MAXN];
        for (int l = 0; l < n; ++l) rhs[l] = M->psi0[l] * Qc[v * NS + i] - dt * M->w[l] * R[(l * V + v) * NS + i];
        for (int k = 0; k < n; ++k) {
          double s = 0.0;
          for (int l = 0; l < n; ++l) s += M->K1inv[k][l] * rhs[l];
          const double d = fabs(s - q[(k * V + v) * NS + i]);
          if (d > change) change = d;
          q[(k * V + v) * NS + i] = s;
        }
      }
    ++r;
    if (M->picard_tol > 0.0 && change <= M->picard_tol) break;
  }
  free(R);
  return r;
}

/* Cauchy-Kowalevskaya predictor for linear PDEs (Sec. 3.1, last paragraph):
 * q(tau) = sum_{m=0}^{N} (tau dt)^m / m! d_t^m Q, d_t^{m+1} Q = -sum_dir d_dir F_dir(d_t^m Q). */
void or_ck_cell(const or_mesh* M, int cell, const double* Qc, double dt, double* q) {
  const int n = M->n, V = M->nvar, NS = ipow(n, M->dim), N = M->N;
  double* dQ = (double*)malloc(sizeof(double) * (size_t)(N + 1) * V * NS);
  memcpy(dQ, Qc, sizeof(double) * (size_t)V * NS);
  for (int m = 0; m < N; ++m) {
    space_derivative_of_flux(M, cell, dQ + (size_t)m * V * NS, 1, dQ + (size_t)(m + 1) * V * NS);
    for (int j = 0; j < V * NS; ++j) dQ[(size_t)(m + 1) * V * NS + j] *= -1.0;
  }
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < V * NS; ++j) {
      double s = 0.0, fac = 1.0;
      for (int m = 0; m <= N; ++m) {
        if (m > 0) fac *= (M->xi[k] * dt) / m;
        s += fac * dQ[(size_t)m * V * NS + j];
      }
      q[(size_t)k * V * NS + j] = s;
    }
  free(dQ);
}

/* ------------------------------------------------------------------------ */
/* Time step, eq. (CFL_condition): dt = C h / (d (2N+1) lambda_max)           */
/* ------------------------------------------------------------------------ */

double or_dt(const or_mesh* M, const double* Q) {
  const int V = M->nvar, NS = ipow(M->n, M->dim), C = ncells(M);
  double lam = 0.0;
  for (int c = 0; c < C; ++c)
    for (int i = 0; i < NS; ++i) {
      double q[OR_MAXV];
      for (int v = 0; v < V; ++v) q[v] = Q[((size_t)c * V + v) * NS + i];
      for (int dir = 0; dir < M->dim; ++dir) {
        double s = or_speed(M, c, q, dir);
        if (s > lam) lam = s;
      }
    }
  double h = M->h[0];
  for (int a = 1; a < M->dim; ++a)
    if (M->h[a] < h) h = M->h[a];
  return M->cfl * h / ((double)M->dim * (2.0 * M->N + 1.0) * lam);
}

/* ------------------------------------------------------------------------ */
/* Rusanov flux, eq. (rusanov_flux), with one speed per face (max over nodes */
/* and both sides).  qm/Fm: left (lower) cell's trace, qp/Fp: right cell's.  */
/* Arrays are [v][j].                                                        */
/* ------------------------------------------------------------------------ */

void or_rusanov(const or_mesh* M, int cellL, int cellR, int dir, int nface, const double* qm,
                const double* qp, const double* Fm, const double* Fp, double* G) {
  const int V = M->nvar;
  double s = 0.0;
  for (int j = 0; j < nface; ++j) {
    double a[OR_MAXV], b[OR_MAXV];
    for (int v = 0; v < V; ++v) {
      a[v] = qm[v * nface + j];
      b[v] = qp[v * nface + j];
    }
    double sa = or_speed(M, cellL, a, dir), sb = or_speed(M, cellR, b, dir);
    if (sa > s) s = sa;
    if (sb > s) s = sb;
  }
  for (int v = 0; v < V; ++v)
    for (int j = 0; j < nface; ++j) {
      int o = v * nface + j;
      double jump = qm[o] - qp[o];
      if (M->pde == OR_SWE_B) {
        /* eq. (swe_custom_riemann): the dissipation acts on the surface elevation h + b
         * instead of h, and not on b */
        if (v == 0) jump = (qm[j] + qm[3 * nface + j]) - (qp[j] + qp[3 * nface + j]);
        if (v == 3) jump = 0.0;
      }
      G[o] = 0.5 * (Fm[o] + Fp[o]) + 0.5 * s * jump;
    }
}

void or_ncp_fluctuation(const or_mesh* M, int dir, int nface, const double* qm, const double* qp,
                        double* Dh) {
  const int V = M->nvar;
  for (int o = 0; o < V * nface; ++o) Dh[o] = 0.0;
  if (M->pde != OR_SWE_B) return;
  double g = M->pp[0];
  for (int j = 0; j < nface; ++j) {
    /* B_dir is linear in h along the straight path: int_0^1 g h(s) ds = g (h- + h+) / 2 */
    double hbar = 0.5 * (qm[j] + qp[j]);
    double deta = (qp[j] + qp[3 * nface + j]) - (qm[j] + qm[3 * nface + j]);
    Dh[(1 + dir) * nface + j] = 0.5 * g * hbar * deta;
  }
}

static int neighbour(const or_mesh* M, int c, int dir, int side) {
  int cc[3] = {c % M->m[0], (c / M->m[0]) % M->m[1], c / (M->m[0] * M->m[1])};
  cc[dir] = (cc[dir] + (side ? 1 : -1) + M->m[dir]) % M->m[dir]; /* periodic */
  return cc[0] + M->m[0] * (cc[1] + M->m[1] * cc[2]);
}

/* index of the face node j of spatial node i for a face normal to dir:
 * the remaining indices in increasing dimension order */
static int face_index(const or_mesh* M, int i, int dir) {
  int j = 0, s = 1, r = i;
  for (int a = 0; a < M->dim; ++a) {
    int ia = r % M->n;
    r /= M->n;
    if (a == dir) continue;
    j += ia * s;
    s *= M->n;
  }
  return j;
}

/* ------------------------------------------------------------------------ */
/* One ADER-DG step, Sec. 3 and Algorithm 1:                                 */
/*  pass 1 per cell: predictor, time averages, face traces (expansion),      */
/*         Q += dt vol   (eq. weak_form_volume_surface, volume term)          */
/*  pass 2 per cell: Rusanov on each face, Q -= dt surf (surface term)       */
/* ------------------------------------------------------------------------ */

/* Pass 1 for one cell: reads Qc (the cell's Q^n), writes Qout = Q^n + dt vol and the
 * cell's traces tq/tf [dir][side][v][j] of Qbar and Fbar_dir. */
static void predict_cell(const or_mesh* M, int c, const double* Qc, double dt, double* Qout,
                         double* tq_cell, double* tf_cell) {
  const int n = M->n, V = M->nvar, d = M->dim, NS = ipow(n, d), NF = ipow(n, d - 1);
  double* q = (double*)malloc(sizeof(double) * (size_t)n * V * NS);
  double* Fbar = (double*)malloc(sizeof(double) * (size_t)d * V * NS);
  double* Qbar = (double*)malloc(sizeof(double) * (size_t)V * NS);
  if (M->use_ck)
    or_ck_cell(M, c, Qc, dt, q);
  else
    or_predictor_cell(M, c, Qc, dt, M->picard_iters, q);
  /* time averages over [t^n, t^n+dt] divided by dt: sum_k w_k (.)_k */
  for (int j = 0; j < d * V * NS; ++j) Fbar[j] = 0.0;
  for (int j = 0; j < V * NS; ++j) Qbar[j] = 0.0;
  for (int k = 0; k < n; ++k)
    for (int i = 0; i < NS; ++i) {
      double qv[OR_MAXV], Fv[OR_MAXV];
      for (int v = 0; v < V; ++v) qv[v] = q[(k * V + v) * NS + i];
      for (int v = 0; v < V; ++v) Qbar[v * NS + i] += M->w[k] * qv[v];
      for (int dir = 0; dir < d; ++dir) {
        or_flux(M, c, qv, dir, Fv);
        for (int v = 0; v < V; ++v) Fbar[(dir * V + v) * NS + i] += M->w[k] * Fv[v];
      }
    }
  /* face traces (expansion): extrapolate along dir to xi = 0 and xi = 1 */
  for (int dir = 0; dir < d; ++dir)
    for (int side = 0; side < 2; ++side) {
      const double* psi = side ? M->psi1 : M->psi0;
      double* tq = tq_cell + (dir * 2 + side) * V * NF;
      double* tf = tf_cell + (dir * 2 + side) * V * NF;
      for (int j = 0; j < V * NF; ++j) tq[j] = tf[j] = 0.0;
      for (int v = 0; v < V; ++v)
        for (int i = 0; i < NS; ++i) {
          int a = node_dir_index(M, i, dir), j = face_index(M, i, dir);
          tq[v * NF + j] += psi[a] * Qbar[v * NS + i];
          tf[v * NF + j] += psi[a] * Fbar[(dir * V + v) * NS + i];
        }
    }
  /* volume integral, mass-matrix inverted:
   * vol_i = sum_dir (1/h_dir)(1/w_{i_dir}) sum_a w_a D[a][i_dir] Fbar_dir(i[dir<-a]) */
  for (int v = 0; v < V; ++v)
    for (int i = 0; i < NS; ++i) {
      double vol = 0.0;
      for (int dir = 0; dir < d; ++dir) {
        int idir = node_dir_index(M, i, dir);
        double s = 0.0;
        for (int a = 0; a < n; ++a)
          s += M->w[a] * M->D[a][idir] * Fbar[(dir * V + v) * NS + node_with(M, i, dir, a)];
        vol += s / (M->h[dir] * M->w[idir]);
      }
      Qout[v * NS + i] = Qc[v * NS + i] + dt * vol;
    }
  /* non-conservative volume term, eq. (swe_canonical): Q_i -= dt sum_k w_k sum_dir
   * B_dir(q_{k,i}) dq_k/dx_dir (i) (mass-inverted; the nodal quadrature of the cell integral
   * of the test function times B grad q) */
  if (M->pde == OR_SWE_B)
    for (int i = 0; i < NS; ++i) {
      double acc[OR_MAXV] = {0};
      for (int k = 0; k < n; ++k) {
        double qv[OR_MAXV];
        for (int v = 0; v < V; ++v) qv[v] = q[(k * V + v) * NS + i];
        for (int dir = 0; dir < d; ++dir) {
          double dq[OR_MAXV], b[OR_MAXV];
          ncp_state_derivative(M, q + (size_t)k * V * NS, i, dir, dq);
          or_ncp(M, qv, dir, dq, b);
          for (int v = 0; v < V; ++v) acc[v] += M->w[k] * b[v];
        }
      }
      for (int v = 0; v < V; ++v) Qout[v * NS + i] -= dt * acc[v];
    }
  free(q);
  free(Fbar);
  free(Qbar);
}

/* Pass 2 for one cell c: trace(cell, dir, side) returns that cell's [v][j] block.
 * Qcell holds Q^n + dt vol on entry and Q^{n+1} on exit. */
typedef const double* (*trace_fn)(const void* ctx, int cell, int dir, int side, int which);

static void correct_cell(const or_mesh* M, int c, double dt, trace_fn tr, const void* ctx,
                         double* Qcell) {
  const int V = M->nvar, d = M->dim, NS = ipow(M->n, d), NF = ipow(M->n, d - 1);
  double* G0 = (double*)malloc(sizeof(double) * (size_t)V * NF);
  double* G1 = (double*)malloc(sizeof(double) * (size_t)V * NF);
  for (int dir = 0; dir < d; ++dir) {
    int cl = neighbour(M, c, dir, 0), cr = neighbour(M, c, dir, 1);
    /* left face of c: (cl side 1 | c side 0);  right face: (c side 1 | cr side 0) */
    or_rusanov(M, cl, c, dir, NF, tr(ctx, cl, dir, 1, 0), tr(ctx, c, dir, 0, 0),
               tr(ctx, cl, dir, 1, 1), tr(ctx, c, dir, 0, 1), G0);
    or_rusanov(M, c, cr, dir, NF, tr(ctx, c, dir, 1, 0), tr(ctx, cr, dir, 0, 0),
               tr(ctx, c, dir, 1, 1), tr(ctx, cr, dir, 0, 1), G1);
    if (M->pde == OR_SWE_B) {
      /* path-conservative jump term: c is the plus cell of its left face and the minus cell of
       * its right face */
      double* Dh = (double*)malloc(sizeof(double) * (size_t)V * NF);
      or_ncp_fluctuation(M, dir, NF, tr(ctx, cl, dir, 1, 0), tr(ctx, c, dir, 0, 0), Dh);
      for (int o = 0; o < V * NF; ++o) G0[o] -= Dh[o];
      or_ncp_fluctuation(M, dir, NF, tr(ctx, c, dir, 1, 0), tr(ctx, cr, dir, 0, 0), Dh);
      for (int o = 0; o < V * NF; ++o) G1[o] += Dh[o];
      free(Dh);
    }
    /* surface integral: int phi_k G.n dS on the right (n = +e_dir) and
     * left (n = -e_dir) faces, mass-matrix inverted */
    for (int v = 0; v < V; ++v)
      for (int i = 0; i < NS; ++i) {
        int a = node_dir_index(M, i, dir), j = face_index(M, i, dir);
        double surf = (M->psi1[a] * G1[v * NF + j] - M->psi0[a] * G0[v * NF + j]) /
                      (M->h[dir] * M->w[a]);
        Qcell[v * NS + i] -= dt * surf;
      }
  }
  free(G0);
  free(G1);
}

typedef struct {
  const double* TQ;
  const double* TF;
  int d, V, NF;
} all_traces;

static const double* all_trace(const void* ctx, int cell, int dir, int side, int which) {
  const all_traces* A = (const all_traces*)ctx;
  const double* base = which ? A->TF : A->TQ;
  return base + (((size_t)cell * A->d + dir) * 2 + side) * A->V * A->NF;
}

/* ------------------------------------------------------------------------ */
/* Storage precision (Sec. 4.1): rounding to a binary format of Table         */
/* precision_bits from the definition of its values.  A format with p         */
/* significand bits (hidden bit included) and exponents emin..emax holds      */
/* m 2^(e-p+1) with integer |m| < 2^p and e in [emin, emax]; below 2^emin the */
/* spacing stays 2^(emin-p+1) (subnormals).  Round to nearest, ties to even.  */
/* ------------------------------------------------------------------------ */

double or_round_format(double x, int fmt) {
  int p, emin, emax;
  switch (fmt) {
    case OR_ST_FP32: p = 24; emin = -126; emax = 127; break;
    case OR_ST_BF16: p = 8; emin = -126; emax = 127; break;
    case OR_ST_FP16: p = 11; emin = -14; emax = 15; break;
    default: return x;
  }
  if (x == 0.0 || !isfinite(x)) return x;
  int e2;
  frexp(x, &e2);             /* |x| in [2^(e2-1), 2^e2) */
  int lead = e2 - 1;         /* exponent of the leading bit */
  if (lead < emin) lead = emin;
  const int q = lead - (p - 1); /* exponent of the spacing of representable values */
  const double s = ldexp(x, -q);  /* x in units of the spacing; exact (power-of-two scaling) */
  const double r = nearbyint(s);  /* nearest integer, ties to even (default rounding mode) */
  const double y = ldexp(r, q);
  const double maxv = ldexp(2.0 - ldexp(1.0, 1 - p), emax);
  if (fabs(y) > maxv) return x > 0 ? INFINITY : -INFINITY;
  return y;
}

void or_round_array(double* x, long long count, int fmt) {
  if (fmt == OR_ST_FP64) return;
  for (long long i = 0; i < count; ++i) x[i] = or_round_format(x[i], fmt);
}

void or_set_storage(or_mesh* M, int fmt) { M->storage = fmt; }

double or_step(const or_mesh* M, double* Q, double dt) {
  const int n = M->n, V = M->nvar, d = M->dim, NS = ipow(n, d), NF = ipow(n, d - 1),
            C = ncells(M);
  size_t tsz = (size_t)C * d * 2 * V * NF;
  double* TQ = (double*)malloc(sizeof(double) * tsz);
  double* TF = (double*)malloc(sizeof(double) * tsz);
#pragma omp parallel
  {
    double* Qc = (double*)malloc(sizeof(double) * (size_t)V * NS);
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < C; ++c) {
      double* Qcell = Q + (size_t)c * V * NS;
      memcpy(Qc, Qcell, sizeof(double) * (size_t)V * NS);
      predict_cell(M, c, Qc, dt, Qcell, TQ + (size_t)c * d * 2 * V * NF,
                   TF + (size_t)c * d * 2 * V * NF);
    }
    free(Qc);
  }
  /* the solution is stored in the storage format between the two traversals */
  or_round_array(Q, (long long)C * V * NS, M->storage);
  all_traces A = {TQ, TF, d, V, NF};
#pragma omp parallel for schedule(static)
  for (int c = 0; c < C; ++c) correct_cell(M, c, dt, all_trace, &A, Q + (size_t)c * V * NS);
  or_round_array(Q, (long long)C * V * NS, M->storage);
  free(TQ);
  free(TF);
  (void)n;
  return dt;
}

/* The same step evaluated only at the listed cells: out[s] = Q^{n+1} of cells[s].  Each listed
 * cell needs the predictors of itself and its 2d face neighbours. */
typedef struct {
  int d, V, NF, nloc;
  const int* ids;
  const double* TQ;
  const double* TF;
} local_traces;

static const double* local_trace(const void* ctx, int cell, int dir, int side, int which) {
  const local_traces* L = (const local_traces*)ctx;
  int s = 0;
  while (s < L->nloc && L->ids[s] != cell) ++s;
  const double* base = which ? L->TF : L->TQ;
  return base + (((size_t)s * L->d + dir) * 2 + side) * L->V * L->NF;
}

void or_step_cells(const or_mesh* M, const double* Q, double dt, int nsample, const int* cells,
                   double* out) {
  const int V = M->nvar, d = M->dim, NS = ipow(M->n, d), NF = ipow(M->n, d - 1);
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < nsample; ++s) {
    int ids[7];
    int nloc = 0;
    ids[nloc++] = cells[s];
    for (int dir = 0; dir < d; ++dir)
      for (int side = 0; side < 2; ++side) {
        int nb = neighbour(M, cells[s], dir, side), seen = 0;
        for (int t = 0; t < nloc; ++t) seen |= ids[t] == nb;
        if (!seen) ids[nloc++] = nb;
      }
    double* TQ = (double*)malloc(sizeof(double) * (size_t)nloc * d * 2 * V * NF);
    double* TF = (double*)malloc(sizeof(double) * (size_t)nloc * d * 2 * V * NF);
    double* Qv = (double*)malloc(sizeof(double) * (size_t)V * NS);
    for (int t = 0; t < nloc; ++t) {
      predict_cell(M, ids[t], Q + (size_t)ids[t] * V * NS, dt, Qv, TQ + (size_t)t * d * 2 * V * NF,
                   TF + (size_t)t * d * 2 * V * NF);
      if (t == 0) memcpy(out + (size_t)s * V * NS, Qv, sizeof(double) * (size_t)V * NS);
    }
    or_round_array(out + (size_t)s * V * NS, (long long)V * NS, M->storage);
    local_traces L = {d, V, NF, nloc, ids, TQ, TF};
    correct_cell(M, cells[s], dt, local_trace, &L, out + (size_t)s * V * NS);
    or_round_array(out + (size_t)s * V * NS, (long long)V * NS, M->storage);
    free(TQ);
    free(TF);
    free(Qv);
  }
}

int or_run(const or_mesh* M, double* Q, int nsteps, double* t, double* dt_last) {
  double tt = t ? *t : 0.0, dt = 0.0;
  for (int s = 0; s < nsteps; ++s) {
    dt = or_dt(M, Q);
    or_step(M, Q, dt);
    tt += dt;
  }
  if (t) *t = tt;
  if (dt_last) *dt_last = dt;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Heap-allocated mesh handles for the ctypes wrapper                        */
/* ------------------------------------------------------------------------ */

or_mesh* or_create(int dim, int N, const int* m, const double* lo, const double* hi, int pde,
                   const double* params, int nparams, double cfl, int picard_iters) {
  or_mesh* M = (or_mesh*)malloc(sizeof(or_mesh));
  if (!M) return NULL;
  if (or_setup(M, dim, N, m, lo, hi, pde, params, nparams, cfl, picard_iters) != 0) {
    free(M);
    return NULL;
  }
  return M;
}

void or_destroy(or_mesh* M) { free(M); }

void or_set_ck(or_mesh* M, int use_ck) { M->use_ck = use_ck; }

void or_set_picard_iters(or_mesh* M, int iters) { M->picard_iters = iters; }

void or_set_picard_tol(or_mesh* M, double tol) { M->picard_tol = tol; }

/* ------------------------------------------------------------------------ */
/* Receivers and misfit (acoustics).  A receiver samples the pressure of the */
/* DG polynomial (eq. piecewise_solution) of the cell that contains it.      */
/* ------------------------------------------------------------------------ */

void or_receiver_weights(const or_mesh* M, const double* x, int* cell, double* wts) {
  int cc[3] = {0, 0, 0};
  double xi[3] = {0, 0, 0};
  for (int a = 0; a < M->dim; ++a) {
    double s = (x[a] - M->lo[a]) / M->h[a];
    double f = floor(s);
    int ci = (int)f;
    xi[a] = s - f;
    ci %= M->m[a];
    if (ci < 0) ci += M->m[a];
    cc[a] = ci;
  }
  *cell = cc[0] + M->m[0] * (cc[1] + M->m[1] * cc[2]);
  const int NS = ipow(M->n, M->dim);
  for (int i = 0; i < NS; ++i) {
    double w = 1.0;
    int r = i;
    for (int a = 0; a < M->dim; ++a) {
      w *= or_lagrange(M->n, M->xi, r % M->n, xi[a]);
      r /= M->n;
    }
    wts[i] = w;
  }
}

void or_receivers_eval(const or_mesh* M, const double* Q, int nrecv, const double* xyz, double* out) {
  const int V = M->nvar, NS = ipow(M->n, M->dim);
  double* w = (double*)malloc(sizeof(double) * NS);
  for (int r = 0; r < nrecv; ++r) {
    int c;
    or_receiver_weights(M, xyz + (size_t)r * M->dim, &c, w);
    double p = 0.0;
    for (int i = 0; i < NS; ++i) p += w[i] * Q[((size_t)c * V + 0) * NS + i];
    out[r] = p;
  }
  free(w);
}

/* Forward run from Q (overwritten with Q^nsteps): J = 1/2 sum_{n=1..nsteps} sum_r (p_h(x_r, t^n)
 * - d_r^n)^2 with observed[n-1][r]; the sampled pressures go to record[n-1][r] if not NULL. */
double or_misfit(const or_mesh* M, double* Q, int nsteps, int nrecv, const double* xyz,
                 const double* observed, double* record) {
  double J = 0.0;
  double* p = (double*)malloc(sizeof(double) * (nrecv > 0 ? nrecv : 1));
  for (int s = 0; s < nsteps; ++s) {
    or_step(M, Q, or_dt(M, Q));
    or_receivers_eval(M, Q, nrecv, xyz, p);
    for (int r = 0; r < nrecv; ++r) {
      double e = p[r] - (observed ? observed[(size_t)s * nrecv + r] : 0.0);
      J += 0.5 * e * e;
      if (record) record[(size_t)s * nrecv + r] = p[r];
    }
  }
  free(p);
  return J;
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of one step for linear acoustics with per-cell c.  dt is */
/* that of the forward step, held fixed.  The step is linear in Q; each part */
/* of or_step is transposed in reverse order.  On entry lam holds dJ/dQ^{n+1};*/
/* on exit dJ/dQ^n (without the misfit source of step n).  gK[c] accumulates */
/* dJ/dK_c (K = rho c^2, through the fluxes), gS[c] dJ/dc_c through the      */
/* Rusanov face speed s = max(c_minus, c_plus).                              */
/* ------------------------------------------------------------------------ */

void or_adjoint_step(const or_mesh* M, const double* Qn, double dt, double* lam, double* gK,
                     double* gS) {
  const int n = M->n, V = M->nvar, d = M->dim, NS = ipow(n, d), NF = ipow(n, d - 1), C = ncells(M);
  const double rho = M->pp[0];
  /* forward traces of Q^n (for the face-speed term) */
  size_t tsz = (size_t)C * d * 2 * V * NF;
  double* TQ = (double*)malloc(sizeof(double) * tsz);
  double* TF = (double*)malloc(sizeof(double) * tsz);
  {
    double* Qv = (double*)malloc(sizeof(double) * (size_t)V * NS);
    for (int c = 0; c < C; ++c)
      predict_cell(M, c, Qn + (size_t)c * V * NS, dt, Qv, TQ + (size_t)c * d * 2 * V * NF,
                   TF + (size_t)c * d * 2 * V * NF);
    free(Qv);
  }
  /* 1. adjoint of the surface update: face-flux adjoints from each side's own lam.
   * lamG(c, dir, side)[v][j]: side 1 is c's right face, side 0 its left face. */
  size_t gsz = (size_t)C * d * 2 * V * NF;
  double* lamG = (double*)calloc(gsz, sizeof(double));
  for (int c = 0; c < C; ++c)
    for (int dir = 0; dir < d; ++dir)
      for (int v = 0; v < V; ++v)
        for (int i = 0; i < NS; ++i) {
          int a = node_dir_index(M, i, dir), j = face_index(M, i, dir);
          double l = lam[((size_t)c * V + v) * NS + i];
          /* Q_i -= dt (psi1[a] G+ - psi0[a] G-) / (h w_a) */
          lamG[(((size_t)c * d + dir) * 2 + 1) * V * NF + v * NF + j] += -dt * M->psi1[a] / (M->h[dir] * M->w[a]) * l;
          lamG[(((size_t)c * d + dir) * 2 + 0) * V * NF + v * NF + j] += dt * M->psi0[a] / (M->h[dir] * M->w[a]) * l;
        }
  double* out = (double*)malloc(sizeof(double) * (size_t)C * V * NS);
  for (int c = 0; c < C; ++c) {
    const double* Qc = Qn + (size_t)c * V * NS;
    const double* lc = lam + (size_t)c * V * NS;
    /* forward predictor of this cell, keeping every iterate (linear flux, K = rho c^2) */
    const int I = M->picard_iters;
    double* it = (double*)malloc(sizeof(double) * (size_t)(I + 1) * n * V * NS);
    for (int k = 0; k < n; ++k)
      for (int v = 0; v < V; ++v)
        for (int i = 0; i < NS; ++i) it[((size_t)k * V + v) * NS + i] = Qc[v * NS + i];
    double* R = (double*)malloc(sizeof(double) * (size_t)n * V * NS);
    for (int r = 1; r <= I; ++r) {
      const double* qp = it + (size_t)(r - 1) * n * V * NS;
      double* qr = it + (size_t)r * n * V * NS;
      space_derivative_of_flux(M, c, qp, n, R);
      for (int v = 0; v < V; ++v)
        for (int i = 0; i < NS; ++i) {
          double rhs[OR_MAXN];
          for (int l = 0; l < n; ++l) rhs[l] = M->psi0[l] * Qc[v * NS + i] - dt * M->w[l] * R[(l * V + v) * NS + i];
          for (int k = 0; k < n; ++k) {
            double s = 0.0;
            for (int l = 0; l < n; ++l) s += M->K1inv[k][l] * rhs[l];
            qr[(k * V + v) * NS + i] = s;
          }
        }
    }
    const double* qI = it + (size_t)I * n * V * NS;
    double Qbar[OR_MAXV * 512];
    for (int j = 0; j < V * NS; ++j) Qbar[j] = 0.0;
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < V * NS; ++j) Qbar[j] += M->w[k] * qI[(size_t)k * V * NS + j];
    const double K = M->cell_c ? rho * M->cell_c[c] * M->cell_c[c] : M->pp[1];

    /* 2./3. Rusanov and trace adjoints -> lamQbar, lamFbar[dir] */
    double* lamQbar = (double*)calloc((size_t)V * NS, sizeof(double));
    double* lamFbar = (double*)calloc((size_t)d * V * NS, sizeof(double));
    for (int dir = 0; dir < d; ++dir) {
      int cl = neighbour(M, c, dir, 0), cr = neighbour(M, c, dir, 1);
      double sL = fmax(or_speed(M, cl, NULL, dir), or_speed(M, c, NULL, dir));
      double sR = fmax(or_speed(M, c, NULL, dir), or_speed(M, cr, NULL, dir));
      for (int v = 0; v < V; ++v)
        for (int j = 0; j < NF; ++j) {
          /* right face: c is the minus side; left face: c is the plus side */
          double gR = lamG[(((size_t)c * d + dir) * 2 + 1) * V * NF + v * NF + j] +
                      lamG[(((size_t)cr * d + dir) * 2 + 0) * V * NF + v * NF + j];
          double gL = lamG[(((size_t)cl * d + dir) * 2 + 1) * V * NF + v * NF + j] +
                      lamG[(((size_t)c * d + dir) * 2 + 0) * V * NF + v * NF + j];
          double lTF1 = 0.5 * gR, lTQ1 = 0.5 * sR * gR;   /* G = (Fm+Fp)/2 + s/2 (qm - qp) */
          double lTF0 = 0.5 * gL, lTQ0 = -0.5 * sL * gL;
          /* s = max(c_minus, c_plus): dG/ds = (qm - qp)/2 goes to the side holding the max
           * (half to each side on a tie); counted once per face, at its right-hand cell */
          {
            double qm = TQ[(((size_t)c * d + dir) * 2 + 1) * V * NF + v * NF + j];
            double qp = TQ[(((size_t)cr * d + dir) * 2 + 0) * V * NF + v * NF + j];
            double g = gR * 0.5 * (qm - qp);
            double cm = or_speed(M, c, NULL, dir), cp = or_speed(M, cr, NULL, dir);
            if (cm > cp) gS[c] += g;
            else if (cp > cm) gS[cr] += g;
            else {
              gS[c] += 0.5 * g;
              gS[cr] += 0.5 * g;
            }
          }
          for (int a = 0; a < n; ++a) {
            int node = 0;
            /* node with face index j and coordinate a along dir */
            for (int i = 0; i < NS; ++i)
              if (face_index(M, i, dir) == j && node_dir_index(M, i, dir) == a) { node = i; break; }
            lamQbar[v * NS + node] += M->psi1[a] * lTQ1 + M->psi0[a] * lTQ0;
            lamFbar[(dir * V + v) * NS + node] += M->psi1[a] * lTF1 + M->psi0[a] * lTF0;
          }
        }
    }
    /* 4. volume adjoint: Q_i += dt sum_dir (1/h)(1/w_{i_dir}) sum_a w_a D[a][i_dir] Fbar(i[dir<-a]) */
    for (int dir = 0; dir < d; ++dir)
      for (int v = 0; v < V; ++v)
        for (int i = 0; i < NS; ++i) {
          int id = node_dir_index(M, i, dir);
          for (int a = 0; a < n; ++a)
            lamFbar[(dir * V + v) * NS + node_with(M, i, dir, a)] +=
                dt * M->w[a] * M->D[a][id] / (M->h[dir] * M->w[id]) * lc[v * NS + i];
        }
    /* 5. Fbar_dir = A_dir Qbar: acoustic F_dir = (K v_dir, p / rho e_dir) */
    for (int dir = 0; dir < d; ++dir)
      for (int i = 0; i < NS; ++i) {
        double lp = lamFbar[(dir * V + 0) * NS + i], lv = lamFbar[(dir * V + 1 + dir) * NS + i];
        lamQbar[(1 + dir) * NS + i] += K * lp;
        lamQbar[0 * NS + i] += lv / rho;
        gK[c] += lp * Qbar[(1 + dir) * NS + i];
      }
    /* 6. time average: Qbar = sum_k w_k q_k */
    double* mu = (double*)malloc(sizeof(double) * (size_t)n * V * NS);
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < V * NS; ++j) mu[(size_t)k * V * NS + j] = M->w[k] * lamQbar[j];
    /* 7. Picard sweeps in reverse: q^r = K1inv (psi0 Q - dt w o R(q^{r-1})) */
    double* lamQ = (double*)calloc((size_t)V * NS, sizeof(double));
    double* nu = (double*)malloc(sizeof(double) * (size_t)n * V * NS);
    for (int r = I; r >= 1; --r) {
      const double* qp = it + (size_t)(r - 1) * n * V * NS;
      for (int v = 0; v < V; ++v)
        for (int i = 0; i < NS; ++i)
          for (int l = 0; l < n; ++l) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += M->K1inv[k][l] * mu[((size_t)k * V + v) * NS + i];
            lamQ[v * NS + i] += M->psi0[l] * s;
            nu[((size_t)l * V + v) * NS + i] = -dt * M->w[l] * s; /* adjoint of R_l */
          }
      /* R(q)_{k,i,v} = sum_dir (1/h) sum_a D[i_dir][a] F_dir,v(q_{k, i[dir<-a]}):
       * adjoint to q and, through K in F_dir,p = K v_dir, to K */
      for (int j = 0; j < n * V * NS; ++j) mu[j] = 0.0;
      for (int k = 0; k < n; ++k)
        for (int dir = 0; dir < d; ++dir)
          for (int i = 0; i < NS; ++i) {
            int id = node_dir_index(M, i, dir);
            for (int a = 0; a < n; ++a) {
              int m = node_with(M, i, dir, a);
              double coef = M->D[id][a] / M->h[dir];
              double np = nu[((size_t)k * V + 0) * NS + i], nv = nu[((size_t)k * V + 1 + dir) * NS + i];
              /* F_dir,p(q_m) = K v_dir(q_m), F_dir,v_dir(q_m) = p(q_m) / rho */
              mu[((size_t)k * V + 1 + dir) * NS + m] += coef * K * np;
              mu[((size_t)k * V + 0) * NS + m] += coef * nv / rho;
              gK[c] += coef * np * qp[((size_t)k * V + 1 + dir) * NS + m];
            }
          }
    }
    /* q^0 = Q at every time node */
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < V * NS; ++j) lamQ[j] += mu[(size_t)k * V * NS + j];
    /* 8. identity part of Q^{n+1} = Q^n + vol - surf */
    for (int j = 0; j < V * NS; ++j) out[(size_t)c * V * NS + j] = lc[j] + lamQ[j];
    free(it);
    free(R);
    free(lamQbar);
    free(lamFbar);
    free(mu);
    free(lamQ);
    free(nu);
  }
  memcpy(lam, out, sizeof(double) * (size_t)C * V * NS);
  free(out);
  free(lamG);
  free(TQ);
  free(TF);
}

/* J and its gradients for acoustics with per-cell c: gq0[c][NS] = dJ/dp(Q^0) at every node,
 * gc[c] = dJ/dc_c.  Forward states are all kept (small meshes only). */
double or_adjoint(const or_mesh* M, const double* Q0, int nsteps, int nrecv, const double* xyz,
                  const double* observed, double* gq0, double* gc) {
  const int V = M->nvar, NS = ipow(M->n, M->dim), C = ncells(M);
  const size_t sz = (size_t)C * V * NS;
  double* Qs = (double*)malloc(sizeof(double) * sz * (nsteps + 1));
  double* dts = (double*)malloc(sizeof(double) * (nsteps > 0 ? nsteps : 1));
  double* res = (double*)malloc(sizeof(double) * (size_t)(nsteps > 0 ? nsteps : 1) * (nrecv > 0 ? nrecv : 1));
  double* p = (double*)malloc(sizeof(double) * (nrecv > 0 ? nrecv : 1));
  memcpy(Qs, Q0, sizeof(double) * sz);
  double J = 0.0;
  for (int s = 0; s < nsteps; ++s) {
    memcpy(Qs + (size_t)(s + 1) * sz, Qs + (size_t)s * sz, sizeof(double) * sz);
    dts[s] = or_dt(M, Qs + (size_t)s * sz);
    or_step(M, Qs + (size_t)(s + 1) * sz, dts[s]);
    or_receivers_eval(M, Qs + (size_t)(s + 1) * sz, nrecv, xyz, p);
    for (int r = 0; r < nrecv; ++r) {
      double e = p[r] - observed[(size_t)s * nrecv + r];
      res[(size_t)s * nrecv + r] = e;
      J += 0.5 * e * e;
    }
  }
  double* lam = (double*)calloc(sz, sizeof(double));
  double* gK = (double*)calloc((size_t)C, sizeof(double));
  double* gS = (double*)calloc((size_t)C, sizeof(double));
  double* w = (double*)malloc(sizeof(double) * NS);
  for (int s = nsteps; s >= 1; --s) {
    /* misfit source of step s: dJ/dQ^s */
    for (int r = 0; r < nrecv; ++r) {
      int c;
      or_receiver_weights(M, xyz + (size_t)r * M->dim, &c, w);
      for (int i = 0; i < NS; ++i) lam[((size_t)c * V + 0) * NS + i] += res[(size_t)(s - 1) * nrecv + r] * w[i];
    }
    or_adjoint_step(M, Qs + (size_t)(s - 1) * sz, dts[s - 1], lam, gK, gS);
  }
  for (int c = 0; c < C; ++c) {
    for (int i = 0; i < NS; ++i) gq0[(size_t)c * NS + i] = lam[((size_t)c * V + 0) * NS + i];
    double cc = M->cell_c ? M->cell_c[c] : sqrt(M->pp[1] / M->pp[0]);
    gc[c] = gK[c] * 2.0 * M->pp[0] * cc + gS[c];
  }
  free(Qs);
  free(dts);
  free(res);
  free(p);
  free(lam);
  free(gK);
  free(gS);
  free(w);
  return J;
}
