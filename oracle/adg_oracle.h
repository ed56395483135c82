/*
 * adg_oracle.h -- plain, slow, FP64 CPU implementation of the ADER-DG step
 * (predictor by Picard iteration, Rusanov Riemann solve, volume and surface
 * integrals, CFL time step, L2 error).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Section / equation references are to Marot-Lassauzaie & Bader, "Mixed-Precision
 * in High-Order Methods: the Impact of Floating-Point Precision on the ADER-DG
 * Algorithm" (arXiv 2504.06889):
 *   Sec. 3 eq. (piecewise_solution)        nodal tensor-product GL basis
 *   Sec. 3.1 eq. (Picard)                  space-time predictor system
 *   Sec. 3.2 eq. (weak_form_volume_surface) corrector
 *   Sec. 3.2 eq. (CFL_condition)           time step
 *   Sec. 3.2 eq. (rusanov_flux)            Riemann solver
 *   Sec. 5 (acoustic, elastic, Euler, shallow water)  PDE fluxes
 *   Sec. 5.5 eq. (L2gauss)                 error norm
 *
 * Data layout (same as the exported state of the library under test, but
 * written independently): Q[cell][var][node], cell = cx + m0*(cy + m1*cz),
 * node = i0 + n*(i1 + n*i2), n = N+1, i0 the x index (fastest).
 */
#ifndef ADG_ORACLE_H
#define ADG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAXN 10 /* n = N+1 <= 10 */
#define OR_MAXV 9

/* OR_SWE: shallow water with flat bathymetry in conservative form (h, hu, hv).
 * OR_SWE_B: the paper's form of Sec. 5.4 with bathymetry, Q = (h, hu, hv, b), conservative
 * fluxes without the hydrostatic pressure and the non-conservative product B(Q) grad Q. */
enum { OR_ACOUSTIC = 0, OR_ELASTIC = 1, OR_EULER = 2, OR_SWE = 3, OR_SWE_B = 4 };
/* storage formats of Table precision_bits: significand bits p (with the hidden bit),
 * smallest normal exponent, largest exponent */
enum { OR_ST_FP64 = 0, OR_ST_FP32 = 1, OR_ST_BF16 = 2, OR_ST_FP16 = 3 };
enum {
  OR_SC_PLANAR = 0,
  OR_SC_EULER_WAVE = 1,
  OR_SC_SWE_MODES = 2,
  OR_SC_GAUSS_PULSE = 3,
  OR_SC_LAKE = 4,
  OR_SC_EULER_BELL = 5,  /* Sec. 5.3.1: advected Gaussian density bell */
  OR_SC_EULER_VORTEX = 6 /* Sec. 5.3.2: isentropic vortex */
};

typedef struct {
  int dim, N, n, nvar, pde;
  int m[3];
  double lo[3], h[3];
  double pp[8];       /* PDE parameters as given by the caller */
  double cfl;         /* C_CFL of eq. (CFL_condition) */
  int picard_iters;   /* number of Picard sweeps (the most, with a stopping tolerance) */
  double picard_tol;  /* optional stopping tolerance on max |q^(r) - q^(r-1)| per cell; 0 = off */
  int use_ck;         /* 1: Cauchy-Kowalevskaya predictor instead of Picard (linear PDEs) */
  int storage;        /* persistent-solution format (Sec. 4.1 "storage"): OR_ST_* */
  const double* cell_c; /* optional per-cell wave speed for acoustics (rho fixed); NULL = none */
  /* 1D tables on [0,1] */
  double xi[OR_MAXN], w[OR_MAXN];
  double D[OR_MAXN][OR_MAXN];   /* D[a][b] = psi_b'(xi_a) */
  double psi0[OR_MAXN], psi1[OR_MAXN];
  double K1[OR_MAXN][OR_MAXN], K1inv[OR_MAXN][OR_MAXN];
} or_mesh;

int or_nvar(int pde, int dim);
int or_setup(or_mesh* M, int dim, int N, const int* m, const double* lo, const double* hi,
             int pde, const double* params, int nparams, double cfl, int picard_iters);
void or_set_cell_c(or_mesh* M, const double* cell_c);

/* 1D tables (GL nodes/weights on [0,1], derivative matrix, boundary values) */
void or_tables(int n, double* xi, double* w, double* D, double* psi0, double* psi1,
               double* K1, double* K1inv);
double or_lagrange(int n, const double* xi, int j, double x);

/* pointwise physics */
void or_flux(const or_mesh* M, int cell, const double* q, int dir, double* F);
double or_speed(const or_mesh* M, int cell, const double* q, int dir);
/* non-conservative product B_dir(q) dq of eq. (swe_canonical) for OR_SWE_B, given the
 * derivative dq of the state along dir (zero for every other PDE) */
void or_ncp(const or_mesh* M, const double* q, int dir, const double* dq, double* out);

/* exact / initial data and error */
void or_exact(const or_mesh* M, int scen, const double* sp, int nsp, const double* x, double t,
              double* Q);
void or_interpolate(const or_mesh* M, int scen, const double* sp, int nsp, double t, double* Q);
void or_l2_error(const or_mesh* M, const double* Q, int scen, const double* sp, int nsp, double t,
                 double* out);
void or_l2_diff(const or_mesh* M, const double* Qa, const double* Qb, double* out);
void or_totals(const or_mesh* M, const double* Q, double* tot);

/* one cell's predictor: q[(k*V+v)*NS+i]; at most iters sweeps, fewer when M->picard_tol > 0
 * and the largest change of a sweep is at most that tolerance.  Returns the sweeps taken. */
int or_predictor_cell(const or_mesh* M, int cell, const double* Qc, double dt, int iters,
                      double* q);
void or_ck_cell(const or_mesh* M, int cell, const double* Qc, double dt, double* q);

/* whole step */
double or_dt(const or_mesh* M, const double* Q);
double or_step(const or_mesh* M, double* Q, double dt);
int or_run(const or_mesh* M, double* Q, int nsteps, double* t, double* dt_last);
/* the step at listed cells only: out[s][V][NS] = Q^{n+1} of cells[s] (needs full Q^n) */
void or_step_cells(const or_mesh* M, const double* Q, double dt, int nsample, const int* cells,
                   double* out);

/* receivers, misfit and the discrete adjoint (linear acoustics, per-cell c) */
void or_receiver_weights(const or_mesh* M, const double* x, int* cell, double* wts);
void or_receivers_eval(const or_mesh* M, const double* Q, int nrecv, const double* xyz, double* out);
double or_misfit(const or_mesh* M, double* Q, int nsteps, int nrecv, const double* xyz,
                 const double* observed, double* record);
void or_adjoint_step(const or_mesh* M, const double* Qn, double dt, double* lam, double* gK,
                     double* gS);
double or_adjoint(const or_mesh* M, const double* Q0, int nsteps, int nrecv, const double* xyz,
                  const double* observed, double* gq0, double* gc);

/* Rusanov flux on one face node set, exposed for unit tests (eq. rusanov_flux; for OR_SWE_B
 * the well-balanced form of eq. swe_custom_riemann without its non-conservative part) */
void or_rusanov(const or_mesh* M, int cellL, int cellR, int dir, int nface, const double* qm,
                const double* qp, const double* Fm, const double* Fp, double* G);
/* half the path integral of the non-conservative product across a face, 1/2 int_0^1
 * B_dir(q- + s (q+ - q-)) ds (q+ - q-), on the straight path (OR_SWE_B; zero otherwise):
 * the face's minus cell adds it to the flux G, the plus cell subtracts it */
void or_ncp_fluctuation(const or_mesh* M, int dir, int nface, const double* qm, const double* qp,
                        double* Dh);

/* heap handles (used by the Python wrapper) */
or_mesh* or_create(int dim, int N, const int* m, const double* lo, const double* hi, int pde,
                   const double* params, int nparams, double cfl, int picard_iters);
void or_destroy(or_mesh* M);
void or_set_ck(or_mesh* M, int use_ck);
void or_set_picard_iters(or_mesh* M, int iters);
/* Picard stopping tolerance of the oracle's reading of Sec. 3.1 (the paper fixes none): a cell
 * stops sweeping once max over k, v, i of |q^(r) - q^(r-1)| is at most tol; 0 turns it off. */
void or_set_picard_tol(or_mesh* M, double tol);
/* Persistent solution stored in format fmt (OR_ST_*) between the two grid traversals of a
 * step (Sec. 4.1, Algorithm 1): the step rounds Q after the predictor/volume pass and after
 * the corrector pass. */
void or_set_storage(or_mesh* M, int fmt);
/* x rounded to format fmt: nearest value, ties to even, overflow to +-inf. */
double or_round_format(double x, int fmt);
/* Round count values in place to format fmt. */
void or_round_array(double* x, long long count, int fmt);

#ifdef __cplusplus
}
#endif
#endif
