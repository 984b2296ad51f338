/*
 * hydro_oracle.c -- FP64 CPU oracle of the hot path of arXiv:1511.02137:
 * one SSP-RK3 time step of (3+1)D ideal relativistic hydrodynamics,
 * d_mu T^{mu nu} = S^nu (Sec. 1, Eq. 1), with EOS p = e/3 (Fig. 3 caption),
 * 7th-order WENO reconstruction and third-order Runge-Kutta time integration
 * (Sec. 1), and light-speed jets that deposit energy and momentum at their
 * position (Eq. 2) at the rate of the energy-loss law (Eq. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, plain checker of the CUDA
 * library.  Only the tests, the smoke entry point and the benchmark's CPU
 * baseline leg may load it; the product path never does.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Style: plain loops, FP64 everywhere, compiled with -ffp-contract=off (no
 * fused multiply-add) so that every expression rounds as written.  OpenMP runs
 * only over independent cells; the one cross-thread reduction is a max (exact),
 * so results do not depend on the thread count.
 *
 * Readings of points the paper leaves open:
 *  R1  Conserved vector U = (E, M^x, M^y, M^z, R) with E = T^00, M^i = T^0i and
 *      a passive charge R = n*gamma with flux R*v^j (Sec. 1 names "energy,
 *      momentum and charge densities"; no EOS uses n).
 *  R2  Conserved-to-primitive recovery is the closed form for p = e/3.
 *  R3  Temperature from e = (pi^2/30) * dof * T^4 / (hbar c)^3.
 *  R4  Eq. 3 in natural units converted with hbar c; "x" in Eq. 3 is the path
 *      length travelled since the jet started.
 *  R5  delta^3 of Eq. 2 deposits the whole source into the cell that contains
 *      the jet (nearest-grid-point), divided by the cell volume; the source is
 *      evaluated inside the right-hand side at each RK stage time.
 *  R6  Finite-difference WENO7 with Jiang-Shu weights and Balsara-Shu
 *      smoothness indicators, applied component-wise to local Lax-Friedrichs
 *      split fluxes; alpha is the max spectral radius over the 8 cells of the
 *      interface's stencil.
 *  R7  SSP-RK3 of Shu and Osher; outflow = zero-gradient ghost cells.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NG 4 /* ghost layers: an interface stencil reaches 4 cells to each side */

typedef struct {
  int32_t nx, ny, nz;
  double dx, dt, t0;
  int32_t boundary;   /* 0 = outflow (zero gradient), 1 = periodic */
  int32_t order;      /* 7 = WENO7, 5 = WENO5 */
  int32_t fluid;      /* 1 = flux divergence on, 0 = jet source only */
  int32_t nthreads;   /* OpenMP threads, <= 0: runtime default */
  double k_rad, k_coll, cr_over_cf, hbarc, dof;
  double e_floor;
  double weno_eps;
} orc_config;

typedef struct {
  double x0[3];   /* start point [fm] */
  double n[3];    /* unit direction (orc_jet_normalize) */
  double t_start; /* [fm/c] */
} orc_jet;

typedef struct {
  double dep_E;         /* RK3-weighted energy deposited by jets, sum dt*w_k*S0*dx^3 [GeV] */
  double dep_M[3];      /* same for momentum [GeV] */
  double max_speed;     /* largest spectral radius seen at the first stage of the last step */
  int64_t floor_hits;   /* cells whose primitive recovery needed a floor, summed over stages */
  int32_t jet_cell[16][3]; /* cell of each jet at the last stage evaluated, -1 if outside */
} orc_diag;

#define ORC_MAX_JETS 16

/* ------------------------------------------------------------------------ */
/* Eq. 1 with p = e/3: primitives -> conserved.                               */
/* ------------------------------------------------------------------------ */

/* u^i are the spatial components of the four-velocity, gamma = sqrt(1+u.u).
 * T^{00} = (e+p) gamma^2 - p, T^{0i} = (e+p) gamma u^i, N^0 = n gamma. */
static void prim_to_cons_cell(double e, double ux, double uy, double uz, double n,
                              double* E, double* Mx, double* My, double* Mz, double* R) {
  double p = e / 3.0;
  double g2 = 1.0 + (ux * ux + uy * uy + uz * uz);
  double g = sqrt(g2);
  double w = e + p;
  *E = w * g2 - p;
  *Mx = w * g * ux;
  *My = w * g * uy;
  *Mz = w * g * uz;
  *R = n * g;
}

/* Closed-form recovery for p = e/3.  With m = |M|/E the EOS gives
 * m = 4v/(3+v^2), whose root in [0,1) is v = 3m / (2 + sqrt(4 - 3m^2));
 * then e = E - |M| v = E (1 - m v), p = e/3, v^i = v M^i/|M|, n = R/gamma.
 * Floors act on the primitives only: E below e_floor is raised to e_floor,
 * m is capped at 1 - 1e-12.  Returns 1 when a floor was applied. */
static int cons_to_prim_cell(double E, double Mx, double My, double Mz, double R, double e_floor,
                             double* e, double* vx, double* vy, double* vz, double* p, double* n) {
  int hit = 0;
  double Mabs = sqrt(Mx * Mx + My * My + Mz * Mz);
  double Ee = E;
  if (!(Ee >= e_floor)) { /* also catches NaN */
    Ee = e_floor;
    hit = 1;
  }
  double m = Mabs / Ee;
  const double m_max = 1.0 - 1e-12;
  if (!(m <= m_max)) {
    m = m_max;
    hit = 1;
  }
  double v = 3.0 * m / (2.0 + sqrt(4.0 - 3.0 * m * m));
  *e = Ee * (1.0 - m * v);
  *p = *e / 3.0;
  if (Mabs > 0.0) {
    *vx = v * (Mx / Mabs);
    *vy = v * (My / Mabs);
    *vz = v * (Mz / Mabs);
  } else {
    *vx = 0.0;
    *vy = 0.0;
    *vz = 0.0;
  }
  *n = R * sqrt(1.0 - v * v);
  return hit;
}

/* Characteristic speeds along direction d of the ideal fluid with sound speed
 * c^2 = 1/3 (eigenvalues of the flux Jacobian; textbook relativistic form):
 * lambda_pm = [v_d (1-c^2) +- c sqrt((1-v^2)(1 - v_d^2 - (v^2 - v_d^2) c^2))] / (1 - v^2 c^2). */
static void char_speeds(double vx, double vy, double vz, int d, double* lm, double* lp) {
  const double c2 = 1.0 / 3.0;
  const double c = sqrt(c2);
  double v2 = vx * vx + vy * vy + vz * vz;
  double vd = (d == 0) ? vx : (d == 1) ? vy : vz;
  double disc = (1.0 - v2) * (1.0 - vd * vd - (v2 - vd * vd) * c2);
  if (disc < 0.0) disc = 0.0;
  double den = 1.0 - v2 * c2;
  *lp = (vd * (1.0 - c2) + c * sqrt(disc)) / den;
  *lm = (vd * (1.0 - c2) - c * sqrt(disc)) / den;
}

/* Physical flux of component q along direction d (F^d of Eq. 1):
 * (M^d, M^x v^d + p delta_xd, M^y v^d + p delta_yd, M^z v^d + p delta_zd, R v^d). */
static double phys_flux(int q, int d, const double U[5], const double v[3], double p) {
  switch (q) {
    case 0: return U[1 + d];
    case 1: return U[1] * v[d] + (d == 0 ? p : 0.0);
    case 2: return U[2] * v[d] + (d == 1 ? p : 0.0);
    case 3: return U[3] * v[d] + (d == 2 ? p : 0.0);
    default: return U[4] * v[d];
  }
}

/* ------------------------------------------------------------------------ */
/* WENO reconstruction (Sec. 1: 7th order in use, 5th order implemented).     */
/* Finite-difference form: the values f_j are treated as cell averages of a   */
/* function whose value at x_{i+1/2} is reconstructed.                        */
/* ------------------------------------------------------------------------ */

/* WENO7: candidate cubic reconstructions on stencils {i-3..i}, {i-2..i+1},
 * {i-1..i+2}, {i..i+3}; coefficients in twelfths. */
static const double W7_CAND[4][4] = {
    {-3.0, 13.0, -23.0, 25.0},
    {1.0, -5.0, 13.0, 3.0},
    {-1.0, 7.0, 7.0, -1.0},
    {3.0, 13.0, -5.0, 1.0},
};
/* Linear weights giving the 7-point upwind interpolant. */
static const double W7_D[4] = {1.0 / 35.0, 12.0 / 35.0, 18.0 / 35.0, 4.0 / 35.0};
/* Smoothness indicators beta_k = sum_{l=1..3} int h^{2l-1} (p_k^{(l)})^2 dx over
 * the cell, written as 240*beta_k = sum_{a<=b} B[k][a][b] u_a u_b with
 * u_a = f_{i-3+k+a}. */
static const double W7_B[4][4][4] = {
    {{547.0, -3882.0, 4642.0, -1854.0}, {0.0, 7043.0, -17246.0, 7042.0}, {0.0, 0.0, 11003.0, -9402.0}, {0.0, 0.0, 0.0, 2107.0}},
    {{267.0, -1642.0, 1602.0, -494.0}, {0.0, 2843.0, -5966.0, 1922.0}, {0.0, 0.0, 3443.0, -2522.0}, {0.0, 0.0, 0.0, 547.0}},
    {{547.0, -2522.0, 1922.0, -494.0}, {0.0, 3443.0, -5966.0, 1602.0}, {0.0, 0.0, 2843.0, -1642.0}, {0.0, 0.0, 0.0, 267.0}},
    {{2107.0, -9402.0, 7042.0, -1854.0}, {0.0, 11003.0, -17246.0, 4642.0}, {0.0, 0.0, 7043.0, -3882.0}, {0.0, 0.0, 0.0, 547.0}},
};

/* f[0..6] = f_{i-3..i+3}; returns the reconstruction at x_{i+1/2}.  The
 * candidate values, indicators and nonlinear weights are returned when the
 * pointers are non-NULL. */
static double weno7_point(const double f[7], double eps, double* q_out, double* b_out, double* w_out) {
  double q[4], beta[4], a[4], asum = 0.0;
  for (int k = 0; k < 4; ++k) {
    double s = 0.0;
    for (int j = 0; j < 4; ++j) s += W7_CAND[k][j] * f[k + j];
    q[k] = s / 12.0;
    double b = 0.0;
    for (int r = 0; r < 4; ++r)
      for (int c = r; c < 4; ++c) b += W7_B[k][r][c] * f[k + r] * f[k + c];
    beta[k] = b / 240.0;
    a[k] = W7_D[k] / ((eps + beta[k]) * (eps + beta[k]));
    asum += a[k];
  }
  double out = 0.0;
  for (int k = 0; k < 4; ++k) {
    double w = a[k] / asum;
    out += w * q[k];
    if (w_out) w_out[k] = w;
    if (q_out) q_out[k] = q[k];
    if (b_out) b_out[k] = beta[k];
  }
  return out;
}

/* WENO5: quadratic candidates on {i-2..i}, {i-1..i+1}, {i..i+2} (sixths),
 * linear weights (1,6,3)/10, Jiang-Shu indicators
 * beta_k = 13/12 (second difference)^2 + 1/4 (first-derivative combination)^2. */
static const double W5_CAND[3][3] = {{2.0, -7.0, 11.0}, {-1.0, 5.0, 2.0}, {2.0, 5.0, -1.0}};
static const double W5_D[3] = {1.0 / 10.0, 6.0 / 10.0, 3.0 / 10.0};

/* f[0..4] = f_{i-2..i+2}. */
static double weno5_point(const double f[5], double eps, double* q_out, double* b_out, double* w_out) {
  double q[3], beta[3], a[3], asum = 0.0;
  for (int k = 0; k < 3; ++k) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s += W5_CAND[k][j] * f[k + j];
    q[k] = s / 6.0;
  }
  double d2, d1;
  d2 = f[0] - 2.0 * f[1] + f[2];
  d1 = f[0] - 4.0 * f[1] + 3.0 * f[2];
  beta[0] = 13.0 / 12.0 * d2 * d2 + 0.25 * d1 * d1;
  d2 = f[1] - 2.0 * f[2] + f[3];
  d1 = f[1] - f[3];
  beta[1] = 13.0 / 12.0 * d2 * d2 + 0.25 * d1 * d1;
  d2 = f[2] - 2.0 * f[3] + f[4];
  d1 = 3.0 * f[2] - 4.0 * f[3] + f[4];
  beta[2] = 13.0 / 12.0 * d2 * d2 + 0.25 * d1 * d1;
  for (int k = 0; k < 3; ++k) {
    a[k] = W5_D[k] / ((eps + beta[k]) * (eps + beta[k]));
    asum += a[k];
  }
  double out = 0.0;
  for (int k = 0; k < 3; ++k) {
    double w = a[k] / asum;
    out += w * q[k];
    if (w_out) w_out[k] = w;
    if (q_out) q_out[k] = q[k];
    if (b_out) b_out[k] = beta[k];
  }
  return out;
}

/* ------------------------------------------------------------------------ */
/* Jet source (Eqs. 2-3).                                                     */
/* ------------------------------------------------------------------------ */

/* T from e = (pi^2/30) dof T^4 / (hbar c)^3; the fourth root is taken as two
 * correctly rounded square roots. */
static double temperature(const orc_config* c, double e) {
  double a = M_PI * M_PI / 30.0 * c->dof;
  double hc3 = c->hbarc * c->hbarc * c->hbarc;
  double x = e * hc3 / a;
  if (x < 0.0) x = 0.0;
  return sqrt(sqrt(x));
}

/* Cell of a jet at time t: x_J = x0 + n (t - t_start); index floor(x/dx + N/2)
 * per axis (cell centres at (i + 1/2 - N/2) dx).  Returns 1 when the jet has
 * started (t >= t_start) and lies inside the grid; *ell = t - t_start is the
 * path length at light speed. */
static int jet_cell(const orc_config* c, const orc_jet* J, double t, int32_t ijk[3], double* ell) {
  double l = t - J->t_start;
  *ell = l;
  const int32_t N[3] = {c->nx, c->ny, c->nz};
  int inside = (l >= 0.0);
  for (int a = 0; a < 3; ++a) {
    double x = J->x0[a] + J->n[a] * l;
    double s = x / c->dx + 0.5 * (double)N[a];
    double fl = floor(s);
    if (!(fl >= 0.0 && fl < (double)N[a])) {
      inside = 0;
      ijk[a] = -1;
    } else {
      ijk[a] = (int32_t)fl;
    }
  }
  if (!inside) ijk[0] = ijk[1] = ijk[2] = -1;
  return inside;
}

/* Energy given to the medium per unit time (c = 1) by a jet that has travelled
 * ell in medium of temperature T: -dE/dx of Eq. 3 in GeV/fm. */
static double jet_dEdx(const orc_config* c, double T, double ell) {
  double hc = c->hbarc;
  return c->k_rad * c->cr_over_cf * T * T * T * ell / (hc * hc) + c->k_coll * c->cr_over_cf * T * T / hc;
}

/* ------------------------------------------------------------------------ */
/* Padded grid and the right-hand side L(U) = -div F + S.                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n[3];   /* interior cells per axis */
  int p[3];   /* padded cells per axis */
  size_t pn;  /* padded cells total */
  size_t in;  /* interior cells total */
} grid_t;

static grid_t make_grid(const orc_config* c) {
  grid_t g;
  g.n[0] = c->nx; g.n[1] = c->ny; g.n[2] = c->nz;
  for (int a = 0; a < 3; ++a) g.p[a] = g.n[a] + 2 * NG;
  g.pn = (size_t)g.p[0] * g.p[1] * g.p[2];
  g.in = (size_t)g.n[0] * g.n[1] * g.n[2];
  return g;
}

static inline size_t pidx(const grid_t* g, int i, int j, int k) {
  return ((size_t)(k + NG) * g->p[1] + (size_t)(j + NG)) * g->p[0] + (size_t)(i + NG);
}
static inline size_t uidx(const grid_t* g, int i, int j, int k) {
  return ((size_t)k * g->n[1] + (size_t)j) * g->n[0] + (size_t)i;
}

/* Ghost cell -> interior cell: clamp (outflow) or wrap (periodic). */
static inline int map_index(int i, int n, int periodic) {
  if (periodic) return ((i % n) + n) % n;
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

/* Work arrays for one RHS evaluation. */
typedef struct {
  double* Up;     /* 5 x pn padded conserved */
  double* prim;   /* 6 x pn: e, vx, vy, vz, p, n */
  double* rho;    /* 3 x pn spectral radius per direction */
  double* Fhat;   /* 5 x (interfaces of one direction) */
} work_t;

static int work_alloc(work_t* w, const grid_t* g) {
  size_t fmax = 0;
  for (int d = 0; d < 3; ++d) {
    size_t f = (size_t)(g->n[d] + 1);
    for (int a = 0; a < 3; ++a)
      if (a != d) f *= (size_t)g->n[a];
    if (f > fmax) fmax = f;
  }
  w->Up = (double*)malloc(sizeof(double) * 5 * g->pn);
  w->prim = (double*)malloc(sizeof(double) * 6 * g->pn);
  w->rho = (double*)malloc(sizeof(double) * 3 * g->pn);
  w->Fhat = (double*)malloc(sizeof(double) * 5 * fmax);
  if (!w->Up || !w->prim || !w->rho || !w->Fhat) return -1;
  return 0;
}

static void work_free(work_t* w) {
  free(w->Up);
  free(w->prim);
  free(w->rho);
  free(w->Fhat);
}

typedef struct {
  double S0[ORC_MAX_JETS]; /* energy source of each jet this stage, GeV/fm^4 (0 if outside) */
  int32_t cell[ORC_MAX_JETS][3];
  int64_t floor_hits;
  double max_speed;
} rhs_info;

/* L(U) at stage time t.  U is the interior state [5][nz][ny][nx]; L has the same
 * layout. */
static void rhs_eval(const orc_config* c, const grid_t* g, work_t* w, const double* U, double t,
                     const orc_jet* jets, int njet, double* L, rhs_info* info) {
  const int periodic = (c->boundary == 1);
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const size_t pn = g->pn, in = g->in;

  /* a1: fill the padded array, ghosts by clamping (outflow) or wrapping. */
#pragma omp parallel for schedule(static)
  for (int k = -NG; k < nz + NG; ++k)
    for (int j = -NG; j < ny + NG; ++j)
      for (int i = -NG; i < nx + NG; ++i) {
        size_t src = uidx(g, map_index(i, nx, periodic), map_index(j, ny, periodic), map_index(k, nz, periodic));
        size_t dst = pidx(g, i, j, k);
        for (int q = 0; q < 5; ++q) w->Up[q * pn + dst] = U[q * in + src];
      }

  /* a2 + a3: primitives and spectral radii on every padded cell. */
  int64_t hits = 0;
  double vmax = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : hits) reduction(max : vmax)
  for (int k = -NG; k < nz + NG; ++k)
    for (int j = -NG; j < ny + NG; ++j)
      for (int i = -NG; i < nx + NG; ++i) {
        size_t s = pidx(g, i, j, k);
        double e, vx, vy, vz, p, n;
        int h = cons_to_prim_cell(w->Up[0 * pn + s], w->Up[1 * pn + s], w->Up[2 * pn + s], w->Up[3 * pn + s],
                                  w->Up[4 * pn + s], c->e_floor, &e, &vx, &vy, &vz, &p, &n);
        w->prim[0 * pn + s] = e;
        w->prim[1 * pn + s] = vx;
        w->prim[2 * pn + s] = vy;
        w->prim[3 * pn + s] = vz;
        w->prim[4 * pn + s] = p;
        w->prim[5 * pn + s] = n;
        int interior = (i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz);
        for (int d = 0; d < 3; ++d) {
          double lm, lp;
          char_speeds(vx, vy, vz, d, &lm, &lp);
          double r = fabs(lm) > fabs(lp) ? fabs(lm) : fabs(lp);
          w->rho[d * pn + s] = r;
          if (interior && r > vmax) vmax = r;
        }
        if (interior) hits += h;
      }
  info->floor_hits = hits;
  info->max_speed = vmax;

  for (size_t q = 0; q < 5 * in; ++q) L[q] = 0.0;

  if (c->fluid) {
    const int half = (c->order == 5) ? 3 : 4; /* stencil reaches cells i-half+1 .. i+half */
    const int width = 2 * half;               /* cells in one interface stencil */
    for (int d = 0; d < 3; ++d) {
      const int a1 = (d + 1) % 3, a2 = (d + 2) % 3; /* transverse axes */
      const int Nd = g->n[d], N1 = g->n[a1], N2 = g->n[a2];
      const size_t nface = (size_t)(Nd + 1);
      /* a4 + a5: numerical flux at interfaces i+1/2, i = -1 .. Nd-1. */
#pragma omp parallel for schedule(static)
      for (int t2 = 0; t2 < N2; ++t2)
        for (int t1 = 0; t1 < N1; ++t1)
          for (int i = -1; i < Nd; ++i) {
            size_t cell[8];
            for (int s = 0; s < width; ++s) {
              int idx[3];
              idx[d] = i - half + 1 + s;
              idx[a1] = t1;
              idx[a2] = t2;
              cell[s] = pidx(g, idx[0], idx[1], idx[2]);
            }
            double alpha = 0.0;
            for (int s = 0; s < width; ++s) {
              double r = w->rho[d * pn + cell[s]];
              if (r > alpha) alpha = r;
            }
            double fp[8][5], fm[8][5];
            for (int s = 0; s < width; ++s) {
              double Uc[5], v[3], p;
              for (int q = 0; q < 5; ++q) Uc[q] = w->Up[q * pn + cell[s]];
              v[0] = w->prim[1 * pn + cell[s]];
              v[1] = w->prim[2 * pn + cell[s]];
              v[2] = w->prim[3 * pn + cell[s]];
              p = w->prim[4 * pn + cell[s]];
              for (int q = 0; q < 5; ++q) {
                double F = phys_flux(q, d, Uc, v, p);
                fp[s][q] = 0.5 * (F + alpha * Uc[q]);
                fm[s][q] = 0.5 * (F - alpha * Uc[q]);
              }
            }
            size_t face = ((size_t)t2 * N1 + (size_t)t1) * nface + (size_t)(i + 1);
            for (int q = 0; q < 5; ++q) {
              double a[7], b[7];
              /* f+ from cells i-half+1 .. i+half-1; f- mirrored from i+half .. i-half+2 */
              for (int s = 0; s < width - 1; ++s) {
                a[s] = fp[s][q];
                b[s] = fm[width - 1 - s][q];
              }
              double hp, hm;
              if (c->order == 5) {
                hp = weno5_point(a, c->weno_eps, NULL, NULL, NULL);
                hm = weno5_point(b, c->weno_eps, NULL, NULL, NULL);
              } else {
                hp = weno7_point(a, c->weno_eps, NULL, NULL, NULL);
                hm = weno7_point(b, c->weno_eps, NULL, NULL, NULL);
              }
              w->Fhat[(size_t)q * N2 * N1 * nface + face] = hp + hm;
            }
          }
      /* a6: L -= (Fhat_{i+1/2} - Fhat_{i-1/2}) / dx */
#pragma omp parallel for schedule(static)
      for (int t2 = 0; t2 < N2; ++t2)
        for (int t1 = 0; t1 < N1; ++t1)
          for (int i = 0; i < Nd; ++i) {
            int idx[3];
            idx[d] = i;
            idx[a1] = t1;
            idx[a2] = t2;
            size_t u = uidx(g, idx[0], idx[1], idx[2]);
            size_t face = ((size_t)t2 * N1 + (size_t)t1) * nface + (size_t)(i + 1);
            for (int q = 0; q < 5; ++q) {
              size_t off = (size_t)q * N2 * N1 * nface;
              L[q * in + u] -= (w->Fhat[off + face] - w->Fhat[off + face - 1]) / c->dx;
            }
          }
    }
  }

  /* a7: jet sources (Eqs. 2-3), nearest-grid-point deposit. */
  double vol = c->dx * c->dx * c->dx;
  for (int jn = 0; jn < njet; ++jn) {
    int32_t ijk[3];
    double ell;
    info->S0[jn] = 0.0;
    int in_grid = jet_cell(c, &jets[jn], t, ijk, &ell);
    for (int a = 0; a < 3; ++a) info->cell[jn][a] = ijk[a];
    if (!in_grid) continue;
    size_t s = pidx(g, ijk[0], ijk[1], ijk[2]);
    double T = temperature(c, w->prim[0 * pn + s]);
    double S0 = jet_dEdx(c, T, ell) / vol;
    size_t u = uidx(g, ijk[0], ijk[1], ijk[2]);
    L[0 * in + u] += S0;
    L[1 * in + u] += jets[jn].n[0] * S0;
    L[2 * in + u] += jets[jn].n[1] * S0;
    L[3 * in + u] += jets[jn].n[2] * S0;
    info->S0[jn] = S0;
  }
}

/* ------------------------------------------------------------------------ */
/* Exported API (ctypes).                                                     */
/* ------------------------------------------------------------------------ */

static void set_threads(const orc_config* c) {
#ifdef _OPENMP
  if (c->nthreads > 0) omp_set_num_threads(c->nthreads);
#else
  (void)c;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_prim_to_cons(int64_t ncell, const double* prim5, double* cons5) {
  for (int64_t s = 0; s < ncell; ++s)
    prim_to_cons_cell(prim5[s], prim5[ncell + s], prim5[2 * ncell + s], prim5[3 * ncell + s], prim5[4 * ncell + s],
                      &cons5[s], &cons5[ncell + s], &cons5[2 * ncell + s], &cons5[3 * ncell + s], &cons5[4 * ncell + s]);
}

/* prim6 = (e, vx, vy, vz, p, n) per cell; returns the number of floor hits. */
int64_t orc_cons_to_prim(int64_t ncell, const double* cons5, double e_floor, double* prim6) {
  int64_t hits = 0;
  for (int64_t s = 0; s < ncell; ++s)
    hits += cons_to_prim_cell(cons5[s], cons5[ncell + s], cons5[2 * ncell + s], cons5[3 * ncell + s],
                              cons5[4 * ncell + s], e_floor, &prim6[s], &prim6[ncell + s], &prim6[2 * ncell + s],
                              &prim6[3 * ncell + s], &prim6[4 * ncell + s], &prim6[5 * ncell + s]);
  return hits;
}

void orc_char_speeds(const double v[3], int32_t d, double out[2]) { char_speeds(v[0], v[1], v[2], d, &out[0], &out[1]); }

double orc_weno7(const double f[7], double eps, double q[4], double beta[4], double w[4]) {
  return weno7_point(f, eps, q, beta, w);
}

double orc_weno5(const double f[5], double eps, double q[3], double beta[3], double w[3]) {
  return weno5_point(f, eps, q, beta, w);
}

double orc_temperature(const orc_config* c, double e) { return temperature(c, e); }

double orc_jet_dEdx(const orc_config* c, double T, double ell) { return jet_dEdx(c, T, ell); }

/* n = dir / |dir|, |dir| = sqrt((dx*dx + dy*dy) + dz*dz). */
int32_t orc_jet_normalize(const double dir[3], double n[3]) {
  double len = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  if (!(len > 0.0)) return -1;
  n[0] = dir[0] / len;
  n[1] = dir[1] / len;
  n[2] = dir[2] / len;
  return 0;
}

int32_t orc_jet_cell(const orc_config* c, const orc_jet* J, double t, int32_t ijk[3], double* ell) {
  return jet_cell(c, J, t, ijk, ell);
}

/* L(U) at time t (one evaluation of the spatial operator plus source). */
int32_t orc_rhs(const orc_config* c, const double* U, double t, const orc_jet* jets, int32_t njet, double* L,
                int64_t* floor_hits, double* max_speed) {
  if (njet < 0 || njet > ORC_MAX_JETS) return -1;
  set_threads(c);
  grid_t g = make_grid(c);
  work_t w;
  if (work_alloc(&w, &g)) {
    work_free(&w);
    return -2;
  }
  rhs_info info;
  rhs_eval(c, &g, &w, U, t, jets, njet, L, &info);
  if (floor_hits) *floor_hits = info.floor_hits;
  if (max_speed) *max_speed = info.max_speed;
  work_free(&w);
  return 0;
}

/* nsteps SSP-RK3 steps (Shu-Osher form) starting at step index step0:
 *   U1 = U + dt L(U, t_n)
 *   U2 = 3/4 U + 1/4 (U1 + dt L(U1, t_n + dt))
 *   U  = 1/3 U + 2/3 (U2 + dt L(U2, t_n + dt/2)),   t_n = t0 + n dt.
 * U is updated in place. */
int32_t orc_run(const orc_config* c, double* U, int64_t step0, int32_t nsteps, const orc_jet* jets, int32_t njet,
                orc_diag* diag) {
  if (njet < 0 || njet > ORC_MAX_JETS || nsteps < 0) return -1;
  set_threads(c);
  grid_t g = make_grid(c);
  const size_t n5 = 5 * g.in;
  work_t w;
  double* U0 = (double*)malloc(sizeof(double) * n5);
  double* U1 = (double*)malloc(sizeof(double) * n5);
  double* L = (double*)malloc(sizeof(double) * n5);
  if (work_alloc(&w, &g) || !U0 || !U1 || !L) {
    work_free(&w);
    free(U0);
    free(U1);
    free(L);
    return -2;
  }
  const double stage_c[3] = {0.0, 1.0, 0.5};
  const double stage_w[3] = {1.0 / 6.0, 1.0 / 6.0, 4.0 / 6.0};
  const double dt = c->dt;
  double vol = c->dx * c->dx * c->dx;
  for (int32_t s = 0; s < nsteps; ++s) {
    int64_t n = step0 + s;
    memcpy(U0, U, sizeof(double) * n5);
    for (int st = 0; st < 3; ++st) {
      double t = c->t0 + ((double)n + stage_c[st]) * dt;
      const double* Us = (st == 0) ? U0 : (st == 1 ? U1 : U);
      rhs_info info;
      rhs_eval(c, &g, &w, Us, t, jets, njet, L, &info);
      if (diag) {
        diag->floor_hits += info.floor_hits;
        if (st == 0) diag->max_speed = info.max_speed;
        for (int jn = 0; jn < njet && jn < 16; ++jn) {
          diag->dep_E += dt * stage_w[st] * info.S0[jn] * vol;
          for (int a = 0; a < 3; ++a) {
            diag->dep_M[a] += dt * stage_w[st] * jets[jn].n[a] * info.S0[jn] * vol;
            diag->jet_cell[jn][a] = info.cell[jn][a];
          }
        }
      }
      if (st == 0) {
        for (size_t q = 0; q < n5; ++q) U1[q] = U0[q] + dt * L[q];
      } else if (st == 1) {
        /* U2 is written into U (U still holds U^n's copy in U0). */
        for (size_t q = 0; q < n5; ++q) U[q] = 0.75 * U0[q] + 0.25 * (U1[q] + dt * L[q]);
      } else {
        for (size_t q = 0; q < n5; ++q) U[q] = (1.0 / 3.0) * U0[q] + (2.0 / 3.0) * (U[q] + dt * L[q]);
      }
    }
  }
  work_free(&w);
  free(U0);
  free(U1);
  free(L);
  return 0;
}
