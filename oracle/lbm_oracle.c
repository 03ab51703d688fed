/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the D2Q9 lattice Boltzmann
 * cylinder-flow step (Sahiti, Gurugubelli, Surasani, "Lattice Boltzmann
 * methodology for unconfined flows", arXiv 2605.02185).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * path.  It is written to be read against the paper, not to be fast: every
 * phase is a whole-lattice loop in the order the paper gives (Section 2.1:
 * collide, then stream, then the boundary corrections), in IEEE double
 * precision, compiled without FMA contraction.
 *
 * Readings of the paper taken here (the paper is silent or garbled on them):
 *   - Collision is BGK (Eq. 2) with the equilibrium of Eq. 3 unless the MRT
 *     model (Eq. 6, below) is selected.
 *   - Streaming is written as a pull: f_i(x) = f*_i(x - c_i).  A source that
 *     is a solid node gives the half-way bounce-back value f*_opp(i)(x)
 *     (Section 2.4 and Section 3.1: reflected within the same time step).  A
 *     source outside the lattice (non-periodic edge) gives the placeholder
 *     f*_i(x); every such value is overwritten by a boundary rule below
 *     except where a boundary rule reads it first at a corner.
 *   - Periodic top/bottom (Eq. 8) is the wrap of the pull source row modulo
 *     ny (diagonal x shift included).
 *   - Free-slip (Eq. 7) is the same-node copy of post-stream values:
 *     top f5=f3, f8=f7, f9=f6; bottom f3=f5, f7=f8, f6=f9 (paper 1-based i).
 *   - Zou-He top/bottom (Eqs. 9-10) take u = U (the inlet speed) and the
 *     wall-normal Zou-He density rho_w.
 *   - Constant-velocity bounce-back top/bottom (Eq. 11) moves both walls at
 *     (U, 0) (Section 2.3.4: the inlet velocity), reflects the node's own
 *     post-collision populations within the step, and takes rho as the
 *     density of that post-collision state.  Eq. 11b repeats "top" and the
 *     top's indices; it is read as the bottom rule with the bottom's
 *     indices (f3, f6, f7 from f*5, f*8, f*9).
 *   - The inlet (Section 3.1, "non-equilibrium bounce-back at the inlet") is
 *     the Zou-He west velocity boundary with velocity (U, 0).
 *   - The outlet (Eq. 13) copies all nine populations from column nx-2 into
 *     column nx-1 after the other boundary rules.
 *   - Boundary order: top row, bottom row (all x), inlet column, outlet
 *     column (all y).
 *   - Interpolated bounce-back (optional, Section 2.4's link-wise
 *     alternative): Bouzidi-Firdaouss-Lallemand linear interpolation with
 *     the link fraction q of the body's true surface; force by momentum
 *     exchange of the leaving and returning populations.
 *   - Momentum exchange (Eq. 14): for a resting half-way wall
 *     f_in = f_out = f*_i(x), so each fluid-to-solid link (c_i pointing into
 *     the solid) adds 2 f*_i(x) c_i; the sum is the force on the solid.
 *
 * The paper's MRT collision (Eq. 6, with its S, m_eq and M) is available as
 * the second collision model; its equilibrium moments are read as rho times
 * the printed column (the printed column lacks the density factor) with
 * j = rho u.
 *
 * A test-only Guo body force and a periodic x mode exist so that the oracle
 * can be pinned against closed forms (Poiseuille, Taylor-Green); they are not
 * part of the method.
 *
 * Population array layout: f[(k*ny + y)*nx + x], k = i-1 (paper index i).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Table 1 (Section 2.1): velocity set and weights of D2Q9, k = i - 1. */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

enum { ORC_Y_FREESLIP = 0, ORC_Y_PERIODIC = 1, ORC_Y_ZOUHE = 2, ORC_Y_MOVING = 3, ORC_Y_WALLS = 4 };
enum { ORC_X_INOUT = 0, ORC_X_PERIODIC = 1 };

/* Eq. 6: the MRT transformation matrix M as printed (rows: rho, e, epsilon,
 * j_x, q_x, j_y, q_y, p_xx, p_xy; columns: directions i = 1..9). */
static const double MM[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},         {-4, -1, -1, -1, -1, 2, 2, 2, 2}, {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},      {0, -2, 0, 2, 0, 1, -1, -1, 1},   {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},      {0, 1, -1, 1, -1, 0, 0, 0, 0},    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

enum { ORC_BGK = 0, ORC_MRT = 1 };

typedef struct {
  int nx, ny;
  int bc_y, bc_x;
  int model;            /* ORC_BGK or ORC_MRT */
  double s[9];          /* MRT relaxation rates, diagonal of S */
  double tau, U;
  double uw_top, uw_bot; /* wall speeds of the constant-velocity bounce-back (default U) */
  double gx, gy;       /* test-only body force density (Guo forcing) */
  unsigned char *solid; /* [ny][nx], 1 = solid node */
  double *f;            /* populations after stream + boundaries, f(n) */
  double *fs;           /* post-collision populations, f*(n) */
  double *rowF;         /* [ny][2] per-row force partial sums */
  double *qlink;        /* [9][ny][nx] link fractions q(x, i) (interpolated bounce-back), NULL: half-way */
} orc_t;

#define IDX(o, k, x, y) ((((size_t)(k)) * (size_t)(o)->ny + (size_t)(y)) * (size_t)(o)->nx + (size_t)(x))

/* Opposite direction: the k' with c_k' = -c_k, found by search over Table 1. */
static int opposite(int k) {
  for (int j = 0; j < 9; ++j)
    if (CX[j] == -CX[k] && CY[j] == -CY[k]) return j;
  return -1;
}

void orc_constants(int *cx, int *cy, double *w, int *opp) {
  for (int k = 0; k < 9; ++k) {
    cx[k] = CX[k];
    cy[k] = CY[k];
    w[k] = WT[k];
    opp[k] = opposite(k);
  }
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Eq. 3 with c = 1:  f_eq_i = w_i rho [1 + 3 c_i.u + 9/2 (c_i.u)^2 - 3/2 u.u]. */
void orc_feq(double rho, double ux, double uy, double *feq) {
  double uu = ux * ux + uy * uy;
  for (int k = 0; k < 9; ++k) {
    double cu = CX[k] * ux + CY[k] * uy;
    feq[k] = WT[k] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
  }
}

/* Eq. 4: rho = sum_i f_i, rho u = sum_i f_i c_i. */
void orc_moments(const double *f9, double *rho, double *ux, double *uy) {
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int k = 0; k < 9; ++k) {
    r += f9[k];
    jx += f9[k] * CX[k];
    jy += f9[k] * CY[k];
  }
  *rho = r;
  *ux = jx / r;
  *uy = jy / r;
}

/* Eq. 2 right-hand side (BGK): f*_i = f_i - (f_i - f_eq_i(rho, u)) / tau.
 * With a non-zero body force (test-only) the Guo forcing term is added and u
 * carries the half-force shift; with gx = gy = 0 this is plain Eq. 2. */
void orc_collide_node(const double *f9, double tau, double gx, double gy, double *out9) {
  double rho, ux, uy, feq[9];
  orc_moments(f9, &rho, &ux, &uy);
  if (gx == 0.0 && gy == 0.0) {
    orc_feq(rho, ux, uy, feq);
    for (int k = 0; k < 9; ++k) out9[k] = f9[k] - (f9[k] - feq[k]) / tau;
    return;
  }
  ux += 0.5 * gx / rho;
  uy += 0.5 * gy / rho;
  orc_feq(rho, ux, uy, feq);
  for (int k = 0; k < 9; ++k) {
    double cu = CX[k] * ux + CY[k] * uy;
    double cg = CX[k] * gx + CY[k] * gy;
    double s = WT[k] * (3.0 * ((CX[k] - ux) * gx + (CY[k] - uy) * gy) + 9.0 * cu * cg);
    out9[k] = f9[k] - (f9[k] - feq[k]) / tau + (1.0 - 0.5 / tau) * s;
  }
}

void orc_mrt_matrix(double *m81) {
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) m81[9 * r + c] = MM[r][c];
}

/* Eq. 6 for one node: m = M f; m_eq = rho [1, -2 + 3 u.u, 1 - 3 u.u, u, -u, v,
 * -v, u^2 - v^2, u v]; m* = m - S (m - m_eq); f* = M^-1 m*.  The rows of M are
 * mutually orthogonal, so M^-1 = M^T diag(1 / |row_k|^2). */
void orc_collide_node_mrt(const double *f9, const double *s, double *out9) {
  double m[9], meq[9], rho, ux, uy;
  orc_moments(f9, &rho, &ux, &uy);
  for (int r = 0; r < 9; ++r) {
    m[r] = 0.0;
    for (int c = 0; c < 9; ++c) m[r] += MM[r][c] * f9[c];
  }
  double uu = ux * ux + uy * uy;
  meq[0] = rho;
  meq[1] = rho * (-2.0 + 3.0 * uu);
  meq[2] = rho * (1.0 - 3.0 * uu);
  meq[3] = rho * ux;
  meq[4] = -rho * ux;
  meq[5] = rho * uy;
  meq[6] = -rho * uy;
  meq[7] = rho * (ux * ux - uy * uy);
  meq[8] = rho * ux * uy;
  double ms[9];
  for (int r = 0; r < 9; ++r) ms[r] = m[r] - s[r] * (m[r] - meq[r]);
  for (int c = 0; c < 9; ++c) {
    double acc = 0.0;
    for (int r = 0; r < 9; ++r) {
      double norm = 0.0;
      for (int q = 0; q < 9; ++q) norm += MM[r][q] * MM[r][q];
      acc += MM[r][c] * ms[r] / norm;
    }
    out9[c] = acc;
  }
}

orc_t *orc_create(int nx, int ny, double tau, double U, int bc_y, int bc_x, const unsigned char *mask) {
  if (nx < 3 || ny < 3 || !(tau > 0.5)) return NULL;
  orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
  if (!o) return NULL;
  o->nx = nx;
  o->ny = ny;
  o->tau = tau;
  o->U = U;
  o->uw_top = U;
  o->uw_bot = U;
  o->bc_y = bc_y;
  o->bc_x = bc_x;
  o->model = ORC_BGK;
  size_t n = (size_t)nx * (size_t)ny;
  o->solid = (unsigned char *)calloc(n, 1);
  o->f = (double *)malloc(9 * n * sizeof(double));
  o->fs = (double *)malloc(9 * n * sizeof(double));
  o->rowF = (double *)calloc(2 * (size_t)ny, sizeof(double));
  if (!o->solid || !o->f || !o->fs || !o->rowF) {
    free(o->solid);
    free(o->f);
    free(o->fs);
    free(o->rowF);
    free(o);
    return NULL;
  }
  if (mask)
    for (size_t c = 0; c < n; ++c) o->solid[c] = mask[c] ? 1 : 0;
  for (int k = 0; k < 9; ++k)
    for (size_t c = 0; c < n; ++c) {
      o->f[(size_t)k * n + c] = WT[k];
      o->fs[(size_t)k * n + c] = WT[k];
    }
  return o;
}

void orc_destroy(orc_t *o) {
  if (!o) return;
  free(o->solid);
  free(o->f);
  free(o->fs);
  free(o->rowF);
  free(o->qlink);
  free(o);
}

/* Select the collision: ORC_BGK (Eq. 2) or ORC_MRT (Eq. 6) with the rates
 * S = diag[1, s_e, s_eps, 1, s_q, 1, s_q, 1/tau, 1/tau] (the paper uses
 * s_e = s_eps = s_q = 1.1). */
void orc_set_collision(orc_t *o, int model, double s_e, double s_eps, double s_q) {
  o->model = model;
  const double s[9] = {1.0, s_e, s_eps, 1.0, s_q, 1.0, s_q, 1.0 / o->tau, 1.0 / o->tau};
  for (int k = 0; k < 9; ++k) o->s[k] = s[k];
}

void orc_set_body_force(orc_t *o, double gx, double gy) {
  o->gx = gx;
  o->gy = gy;
}

/* f(0) = f_eq(rho0, u0) on fluid nodes; solid nodes hold w_i. */
void orc_init_equilibrium(orc_t *o, const double *rho, const double *ux, const double *uy) {
  size_t n = (size_t)o->nx * (size_t)o->ny;
  for (size_t c = 0; c < n; ++c) {
    double feq[9];
    if (o->solid[c])
      for (int k = 0; k < 9; ++k) feq[k] = WT[k];
    else
      orc_feq(rho[c], ux[c], uy[c], feq);
    for (int k = 0; k < 9; ++k) o->f[(size_t)k * n + c] = feq[k];
  }
}

void orc_set_f(orc_t *o, const double *f) { memcpy(o->f, f, 9 * (size_t)o->nx * o->ny * sizeof(double)); }
void orc_get_f(const orc_t *o, double *f) { memcpy(f, o->f, 9 * (size_t)o->nx * o->ny * sizeof(double)); }
void orc_set_fs(orc_t *o, const double *fs) { memcpy(o->fs, fs, 9 * (size_t)o->nx * o->ny * sizeof(double)); }
void orc_get_fs(const orc_t *o, double *fs) { memcpy(fs, o->fs, 9 * (size_t)o->nx * o->ny * sizeof(double)); }

/* Neighbour (x + s*c_k) with the lattice's periodic wraps; 0 if outside. */
static int neighbour(const orc_t *o, int x, int y, int k, int s, int *nxp, int *nyp) {
  int xx = x + s * CX[k], yy = y + s * CY[k];
  if (o->bc_x == ORC_X_PERIODIC) xx = (xx % o->nx + o->nx) % o->nx;
  if (o->bc_y == ORC_Y_PERIODIC) yy = (yy % o->ny + o->ny) % o->ny;
  if (xx < 0 || xx >= o->nx || yy < 0 || yy >= o->ny) return 0;
  *nxp = xx;
  *nyp = yy;
  return 1;
}

/* Collision phase (Eq. 2 or Eq. 6, with Eq. 3 and Eq. 4) on every fluid
 * node: f -> f*. */
void orc_collide(orc_t *o) {
  int nx = o->nx, ny = o->ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = (size_t)y * nx + x;
      double f9[9], out[9];
      for (int k = 0; k < 9; ++k) f9[k] = o->f[IDX(o, k, x, y)];
      if (o->solid[c])
        for (int k = 0; k < 9; ++k) out[k] = f9[k];
      else if (o->model == ORC_MRT)
        orc_collide_node_mrt(f9, o->s, out);
      else
        orc_collide_node(f9, o->tau, o->gx, o->gy, out);
      for (int k = 0; k < 9; ++k) o->fs[IDX(o, k, x, y)] = out[k];
    }
}

/* Momentum exchange, Eq. 14: F = sum over fluid nodes x and directions i
 * with x + c_i solid of 2 f*_i(x) c_i.  Row partials are summed in row order,
 * so the result does not depend on the thread count. */
void orc_force(orc_t *o, double *F) {
  int nx = o->nx, ny = o->ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    double fx = 0.0, fy = 0.0;
    for (int x = 0; x < nx; ++x) {
      if (o->solid[(size_t)y * nx + x]) continue;
      for (int k = 1; k < 9; ++k) {
        int tx, ty;
        if (!neighbour(o, x, y, k, +1, &tx, &ty)) continue;
        if (!o->solid[(size_t)ty * nx + tx]) continue;
        double v = 2.0 * o->fs[IDX(o, k, x, y)];
        fx += v * CX[k];
        fy += v * CY[k];
      }
    }
    o->rowF[2 * y] = fx;
    o->rowF[2 * y + 1] = fy;
  }
  double fx = 0.0, fy = 0.0;
  for (int y = 0; y < ny; ++y) {
    fx += o->rowF[2 * y];
    fy += o->rowF[2 * y + 1];
  }
  F[0] = fx;
  F[1] = fy;
}

/* Interpolated bounce-back (Section 2.4: the link-wise alternative to the
 * staircase, after Bouzidi, Firdaouss and Lallemand 2001), linear form, for
 * the population arriving at fluid node x in direction k from the solid
 * side.  It left x in direction i = opp(k) and met the wall a fraction q of
 * the link from x:
 *   q <  1/2:  f_k(x) = 2q f*_i(x) + (1 - 2q) f*_i(x - c_i),
 *   q >= 1/2:  f_k(x) = f*_i(x) / (2q) + (1 - 1/(2q)) f*_k(x);
 * q = 1/2 is the half-way rule.  Where q < 1/2 and x - c_i is not a fluid
 * node of the lattice, the half-way rule is used. */
static double interpolated_bounce(const orc_t *o, int x, int y, int k) {
  int i = opposite(k);
  double q = o->qlink[IDX(o, i, x, y)];
  int bx, by;
  if (q < 0.5) {
    if (!neighbour(o, x, y, i, -1, &bx, &by) || o->solid[(size_t)by * o->nx + bx])
      return o->fs[IDX(o, i, x, y)];
    return 2.0 * q * o->fs[IDX(o, i, x, y)] + (1.0 - 2.0 * q) * o->fs[IDX(o, i, bx, by)];
  }
  return o->fs[IDX(o, i, x, y)] / (2.0 * q) + (1.0 - 1.0 / (2.0 * q)) * o->fs[IDX(o, k, x, y)];
}

/* Link fractions for interpolated bounce-back: q[(i * ny + y) * nx + x] for
 * fluid x with x + c_i solid (other entries ignored); NULL restores the
 * half-way rule. */
int orc_set_link_q(orc_t *o, const double *q) {
  size_t n = 9 * (size_t)o->nx * o->ny;
  if (!q) {
    free(o->qlink);
    o->qlink = NULL;
    return 0;
  }
  if (!o->qlink) o->qlink = (double *)malloc(n * sizeof(double));
  if (!o->qlink) return -1;
  memcpy(o->qlink, q, n * sizeof(double));
  return 0;
}

/* Copy of the link fractions (zeros under the half-way rule). */
void orc_get_link_q(const orc_t *o, double *q) {
  size_t n = 9 * (size_t)o->nx * o->ny;
  if (o->qlink)
    memcpy(q, o->qlink, n * sizeof(double));
  else
    memset(q, 0, n * sizeof(double));
}

/* Link fractions of a circular body of centre (cx, cy) and radius r: for
 * each link from fluid x along c_i into a solid node, q is the smallest
 * t in (0, 1] with |x + t c_i - c| = r (0.5 where the circle does not cross
 * the link, e.g. a solid node outside the circle). */
int orc_set_circle_q(orc_t *o, double cx, double cy, double r) {
  int nx = o->nx, ny = o->ny;
  double *q = (double *)calloc(9 * (size_t)nx * ny, sizeof(double));
  if (!q) return -1;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      if (o->solid[(size_t)y * nx + x]) continue;
      for (int i = 1; i < 9; ++i) {
        int tx, ty;
        if (!neighbour(o, x, y, i, +1, &tx, &ty) || !o->solid[(size_t)ty * nx + tx]) continue;
        double dx = x - cx, dy = y - cy;
        double a = (double)(CX[i] * CX[i] + CY[i] * CY[i]);
        double b = dx * CX[i] + dy * CY[i];
        double c = dx * dx + dy * dy - r * r;
        double disc = b * b - a * c;
        double t = disc >= 0.0 ? (-b - sqrt(disc)) / a : -1.0;
        q[IDX(o, i, x, y)] = (t > 0.0 && t <= 1.0) ? t : 0.5;
      }
    }
  int rc = orc_set_link_q(o, q);
  free(q);
  return rc;
}

/* Momentum exchange for interpolated bounce-back (Mei, Luo, Shyy 1999, as
 * cited for Eq. 14): each fluid-to-solid link adds c_i (f*_i(x, n) +
 * f_opp(i)(x, n+1)), the population that left and the one that came back;
 * called after the stream and boundary phases of step n, it returns F(n).
 * With q = 1/2 this is the 2 f*_i c_i of orc_force, summed in the same
 * order. */
void orc_force_interpolated(orc_t *o, double *F) {
  int nx = o->nx, ny = o->ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    double fx = 0.0, fy = 0.0;
    for (int x = 0; x < nx; ++x) {
      if (o->solid[(size_t)y * nx + x]) continue;
      for (int k = 1; k < 9; ++k) {
        int tx, ty;
        if (!neighbour(o, x, y, k, +1, &tx, &ty)) continue;
        if (!o->solid[(size_t)ty * nx + tx]) continue;
        double v = o->fs[IDX(o, k, x, y)] + o->f[IDX(o, opposite(k), x, y)];
        fx += v * CX[k];
        fy += v * CY[k];
      }
    }
    o->rowF[2 * y] = fx;
    o->rowF[2 * y + 1] = fy;
  }
  double fx = 0.0, fy = 0.0;
  for (int y = 0; y < ny; ++y) {
    fx += o->rowF[2 * y];
    fy += o->rowF[2 * y + 1];
  }
  F[0] = fx;
  F[1] = fy;
}

/* Streaming phase (left side of Eq. 2), pull form, with half-way bounce-back
 * on solid sources and the placeholder for sources outside the lattice. */
void orc_stream(orc_t *o) {
  int nx = o->nx, ny = o->ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      if (o->solid[(size_t)y * nx + x]) continue;
      for (int k = 0; k < 9; ++k) {
        int sx, sy;
        double v;
        if (!neighbour(o, x, y, k, -1, &sx, &sy))
          v = o->fs[IDX(o, k, x, y)];
        else if (o->solid[(size_t)sy * nx + sx])
          v = o->qlink ? interpolated_bounce(o, x, y, k) : o->fs[IDX(o, opposite(k), x, y)];
        else
          v = o->fs[IDX(o, k, sx, sy)];
        o->f[IDX(o, k, x, y)] = v;
      }
    }
}

/* Section 2.3.1, Eq. 7a (top) and Eq. 7b (bottom).  Paper indices 1-based;
 * here f[k] with k = i - 1. */
static void freeslip_top(double *f) {
  f[4] = f[2]; /* f5 = f3 */
  f[7] = f[6]; /* f8 = f7 */
  f[8] = f[5]; /* f9 = f6 */
}
static void freeslip_bottom(double *f) {
  f[2] = f[4]; /* f3 = f5 */
  f[6] = f[7]; /* f7 = f8 */
  f[5] = f[8]; /* f6 = f9 */
}

/* Section 2.3.3, Eq. 9a-c (top), wall velocity (u, 0) = (U, 0); rho is the
 * Zou-He wall density rho_w = f1 + f2 + f4 + 2 (f3 + f6 + f7). */
static void zouhe_top(double *f, double U) {
  double rho = f[0] + f[1] + f[3] + 2.0 * (f[2] + f[5] + f[6]);
  f[4] = f[2];                                         /* f5 = f3 */
  f[7] = f[5] + 0.5 * (f[1] - f[3]) - 0.5 * rho * U;  /* f8 */
  f[8] = f[6] - 0.5 * (f[1] - f[3]) + 0.5 * rho * U;  /* f9 */
}
/* Eq. 10a-c (bottom); rho_w = f1 + f2 + f4 + 2 (f5 + f8 + f9). */
static void zouhe_bottom(double *f, double U) {
  double rho = f[0] + f[1] + f[3] + 2.0 * (f[4] + f[7] + f[8]);
  f[2] = f[4];                                         /* f3 = f5 */
  f[5] = f[7] - 0.5 * (f[1] - f[3]) + 0.5 * rho * U;  /* f6 */
  f[6] = f[8] + 0.5 * (f[1] - f[3]) - 0.5 * rho * U;  /* f7 */
}

/* Inlet, Section 3.1: Zou-He (non-equilibrium bounce-back) velocity
 * boundary on the west side with velocity (U, 0); unknowns f2, f6, f9. */
static void zouhe_inlet(double *f, double U) {
  double rho = (f[0] + f[2] + f[4] + 2.0 * (f[3] + f[6] + f[7])) / (1.0 - U);
  f[1] = f[3] + (2.0 / 3.0) * rho * U;                       /* f2 */
  f[5] = f[7] - 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * rho * U; /* f6 */
  f[8] = f[6] + 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * rho * U; /* f9 */
}

/* Section 2.3.4, Eq. 11: constant-velocity (moving-wall) bounce-back.  Each
 * population that leaves the node (x, y) through the wall, f*_i(x) with c_i
 * pointing into the wall, returns in the same step as f_opp(i)(x) less
 * 2 w_i rho (c_i . u_w) / c_s^2, c_s^2 = 1/3, u_w = (uw, 0), rho the density
 * of the node's f*(x).  Top (into = +1): i = 3, 6, 7 -> 5, 8, 9 (Eq. 11a);
 * bottom (into = -1): i = 5, 8, 9 -> 3, 6, 7 (Eq. 11b, read with the bottom's
 * indices). */
static void moving_wall(const orc_t *o, int x, int y, int into, double uw, double *f) {
  double fs[9], rho = 0.0;
  for (int k = 0; k < 9; ++k) {
    fs[k] = o->fs[IDX(o, k, x, y)];
    rho += fs[k];
  }
  for (int k = 1; k < 9; ++k)
    if (CY[k] == into) f[opposite(k)] = fs[k] - 2.0 * WT[k] * rho * (CX[k] * uw) * 3.0;
}

void orc_set_wall_velocity(orc_t *o, double uw_top, double uw_bot) {
  o->uw_top = uw_top;
  o->uw_bot = uw_bot;
}

static void load9(const orc_t *o, int x, int y, double *f) {
  for (int k = 0; k < 9; ++k) f[k] = o->f[IDX(o, k, x, y)];
}
static void store9(orc_t *o, int x, int y, const double *f) {
  for (int k = 0; k < 9; ++k) o->f[IDX(o, k, x, y)] = f[k];
}

/* Boundary phase (Section 2.3, applied after streaming): top row, bottom
 * row, inlet column, outlet column (Eq. 13). */
void orc_boundaries(orc_t *o) {
  int nx = o->nx, ny = o->ny;
  double f[9];
  if (o->bc_y == ORC_Y_FREESLIP || o->bc_y == ORC_Y_ZOUHE) {
    for (int x = 0; x < nx; ++x) {
      int y = ny - 1;
      if (o->solid[(size_t)y * nx + x]) continue;
      load9(o, x, y, f);
      if (o->bc_y == ORC_Y_FREESLIP)
        freeslip_top(f);
      else
        zouhe_top(f, o->U);
      store9(o, x, y, f);
    }
    for (int x = 0; x < nx; ++x) {
      int y = 0;
      if (o->solid[(size_t)y * nx + x]) continue;
      load9(o, x, y, f);
      if (o->bc_y == ORC_Y_FREESLIP)
        freeslip_bottom(f);
      else
        zouhe_bottom(f, o->U);
      store9(o, x, y, f);
    }
  }
  if (o->bc_y == ORC_Y_MOVING) {
    for (int x = 0; x < nx; ++x) {
      if (o->solid[(size_t)(ny - 1) * nx + x]) continue;
      load9(o, x, ny - 1, f);
      moving_wall(o, x, ny - 1, +1, o->uw_top, f);
      store9(o, x, ny - 1, f);
    }
    for (int x = 0; x < nx; ++x) {
      if (o->solid[x]) continue;
      load9(o, x, 0, f);
      moving_wall(o, x, 0, -1, o->uw_bot, f);
      store9(o, x, 0, f);
    }
  }
  if (o->bc_x == ORC_X_INOUT) {
    for (int y = 0; y < ny; ++y) {
      if (o->solid[(size_t)y * nx]) continue;
      load9(o, 0, y, f);
      zouhe_inlet(f, o->U);
      store9(o, 0, y, f);
    }
    for (int y = 0; y < ny; ++y) {
      load9(o, nx - 2, y, f);
      store9(o, nx - 1, y, f);
    }
  }
}

/* One time step n -> n+1 in the paper's order (Section 2.1): collide, the
 * force of Eq. 14 from f*(n), stream, boundary corrections.  With
 * interpolated bounce-back the force of step n is taken after the stream
 * and boundary phases (it needs the returning populations).  Fhist receives
 * (Fx, Fy) of each step if not NULL. */
void orc_run(orc_t *o, long nsteps, double *Fhist) {
  for (long s = 0; s < nsteps; ++s) {
    double F[2];
    orc_collide(o);
    if (!o->qlink) orc_force(o, F);
    orc_stream(o);
    orc_boundaries(o);
    if (o->qlink) orc_force_interpolated(o, F);
    if (Fhist) {
      Fhist[2 * s] = F[0];
      Fhist[2 * s + 1] = F[1];
    }
  }
}

/* Moments of the current f (Eq. 4); solid nodes report rho = 1, u = 0.  With
 * the test-only body force the velocity carries the half-force shift. */
void orc_fields(const orc_t *o, double *rho, double *ux, double *uy) {
  int nx = o->nx, ny = o->ny;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = (size_t)y * nx + x;
      if (o->solid[c]) {
        rho[c] = 1.0;
        ux[c] = 0.0;
        uy[c] = 0.0;
        continue;
      }
      double f9[9], r, u, v;
      load9(o, x, y, f9);
      orc_moments(f9, &r, &u, &v);
      rho[c] = r;
      ux[c] = u + 0.5 * o->gx / r;
      uy[c] = v + 0.5 * o->gy / r;
    }
}

/* Brute-force list of fluid-to-solid links (x, y, k) with x + c_k solid, in
 * row-major then direction order.  Returns the number of links (all of them
 * are counted; at most cap are written). */
long orc_links(const orc_t *o, int *out, long cap) {
  long n = 0;
  for (int y = 0; y < o->ny; ++y)
    for (int x = 0; x < o->nx; ++x) {
      if (o->solid[(size_t)y * o->nx + x]) continue;
      for (int k = 1; k < 9; ++k) {
        int tx, ty;
        if (!neighbour(o, x, y, k, +1, &tx, &ty)) continue;
        if (!o->solid[(size_t)ty * o->nx + tx]) continue;
        if (n < cap) {
          out[3 * n] = x;
          out[3 * n + 1] = y;
          out[3 * n + 2] = k;
        }
        ++n;
      }
    }
  return n;
}
