/*
 * oracle.c -- plain FP64 CPU oracle for 4D space-time box screening.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Slow on purpose: every routine is
 * the textbook or paper form of what it computes, with no blocking, fusion or
 * reordering, so that it can be read against the paper.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define TWO_PI 6.283185307179586
#define PI 3.141592653589793

/* ------------------------------------------------------------------------ */
/* Dynamics: Sec. 6.1.  Eq. 1 gives nu-dot; its solution nu(t) is obtained  */
/* through Kepler's equation (mean anomaly M = M0 + n t, eccentric anomaly  */
/* E with E - e sin E = M, then nu from E).  Three rotations (argument of   */
/* perigee, inclination, RAAN) take the perifocal point to ECI.             */
/* ------------------------------------------------------------------------ */

double or_mean_motion(const double *el) {
  double a = el[0];
  return sqrt(OR_MU / (a * a * a));
}

double or_period(const double *el) {
  /* P = 2 pi sqrt(a^3 / mu), evaluated in this fixed order so that the
   * integer step count floor(P / (f dt)) is reproducible. */
  double a = el[0];
  double a3 = a * a * a;
  return TWO_PI * sqrt(a3 / OR_MU);
}

double or_max_speed(const double *el) {
  /* vis-viva at perigee r = a(1-e): v^2 = mu (2/r - 1/a) = mu/a (1+e)/(1-e) */
  double a = el[0], e = el[1];
  return sqrt(OR_MU / a * (1.0 + e) / (1.0 - e));
}

static double kepler_f(double E, double e, double M) { return E - e * sin(E) - M; }

double or_solve_kepler(double M, double e, int *iters) {
  /* Kepler's equation E - e sin E = M for M in any range.  f(E) is strictly
   * increasing (f' = 1 - e cos E > 0 for e < 1) and f(M-e) <= 0 <= f(M+e),
   * so bisection on [M-e, M+e] always brackets the root; Newton steps then
   * polish it to the last bit. */
  double lo = M - e, hi = M + e;
  int it = 0;
  if (e == 0.0) {
    if (iters) *iters = 0;
    return M;
  }
  for (; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (kepler_f(mid, e, M) > 0.0) hi = mid; else lo = mid;
  }
  double E = 0.5 * (lo + hi);
  for (int k = 0; k < 3; ++k) {
    double d = kepler_f(E, e, M) / (1.0 - e * cos(E));
    E -= d;
    ++it;
  }
  if (iters) *iters = it;
  return E;
}

double or_true_anomaly(const double *el, double t_s) {
  /* nu(t): the closed-form solution of Eq. 1.  Continuous in t (no wrap). */
  double e = el[1];
  double M = el[5] + or_mean_motion(el) * t_s;
  double E = or_solve_kepler(M, e, NULL);
  /* tan(nu/2) = sqrt((1+e)/(1-e)) tan(E/2), on the branch of E */
  double half = atan2(sqrt(1.0 + e) * sin(0.5 * E), sqrt(1.0 - e) * cos(0.5 * E));
  double nu = 2.0 * half;
  /* put nu on the same revolution as E */
  double k = floor((E - nu) / TWO_PI + 0.5);
  return nu + k * TWO_PI;
}

static void rot_z(double th, const double v[3], double out[3]) {
  double c = cos(th), s = sin(th);
  double x = v[0] * c - v[1] * s;
  double y = v[0] * s + v[1] * c;
  out[0] = x; out[1] = y; out[2] = v[2];
}

static void rot_x(double th, const double v[3], double out[3]) {
  double c = cos(th), s = sin(th);
  double y = v[1] * c - v[2] * s;
  double z = v[1] * s + v[2] * c;
  out[0] = v[0]; out[1] = y; out[2] = z;
}

/* perifocal -> ECI: rotate by the argument of perigee about z, by the
 * inclination about x, then by the RAAN about z (Sec. 6.1). */
static void perifocal_to_eci(const double *el, const double pf[3], double out[3]) {
  double t1[3], t2[3];
  rot_z(el[4], pf, t1);
  rot_x(el[2], t1, t2);
  rot_z(el[3], t2, out);
}

void or_position_from_nu(const double *el, double nu, double out[3]) {
  double a = el[0], e = el[1];
  double p = a * (1.0 - e * e);
  double r = p / (1.0 + e * cos(nu));
  double pf[3] = {r * cos(nu), r * sin(nu), 0.0};
  perifocal_to_eci(el, pf, out);
}

void or_position(const double *el, double t_s, double out[3]) {
  or_position_from_nu(el, or_true_anomaly(el, t_s), out);
}

void or_velocity_fd(const double *el, double t_s, double h_s, double out[3]) {
  double p1[3], p0[3];
  or_position(el, t_s + h_s, p1);
  or_position(el, t_s - h_s, p0);
  for (int k = 0; k < 3; ++k) out[k] = (p1[k] - p0[k]) / (2.0 * h_s);
}

static double nu_dot(const double *el, double nu) {
  /* Eq. 1: nu' = sqrt(mu / (a(1-e^2))^3) (1 + e cos nu)^2 */
  double a = el[0], e = el[1];
  double p = a * (1.0 - e * e);
  double q = 1.0 + e * cos(nu);
  return sqrt(OR_MU / (p * p * p)) * q * q;
}

double or_nu_rk4(const double *el, double t_s, double h_s) {
  /* classical Runge-Kutta integration of Eq. 1 from nu(0) to nu(t) */
  double nu = or_true_anomaly(el, 0.0);
  int64_t steps = (int64_t)ceil(fabs(t_s) / h_s);
  if (steps == 0) return nu;
  double h = t_s / (double)steps;
  for (int64_t s = 0; s < steps; ++s) {
    double k1 = nu_dot(el, nu);
    double k2 = nu_dot(el, nu + 0.5 * h * k1);
    double k3 = nu_dot(el, nu + 0.5 * h * k2);
    double k4 = nu_dot(el, nu + h * k3);
    nu += h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
  }
  return nu;
}

/* ------------------------------------------------------------------------ */
/* Per-object time step (Sec. 4.3: time is tracked per object).            */
/* ------------------------------------------------------------------------ */

int64_t or_step_ticks(const double *el, int kind, int64_t fixed_ticks,
                      double frac, const double *band_edges_km,
                      const double *band_fracs, int n_bands, double tick_s) {
  if (kind == OR_STEP_FIXED) return fixed_ticks < 1 ? 1 : fixed_ticks;
  double f = frac;
  if (kind == OR_STEP_BAND_TABLE) {
    /* bands over perigee altitude a(1-e) - R_E; n_bands-1 ascending edges */
    double hp = el[0] * (1.0 - el[1]) - OR_RE;
    int b = 0;
    while (b < n_bands - 1 && hp >= band_edges_km[b]) ++b;
    f = band_fracs[b];
  }
  double P = or_period(el);
  double k = floor(P / (f * tick_s));
  return k < 1.0 ? 1 : (int64_t)k;
}

/* ------------------------------------------------------------------------ */
/* Interval arithmetic (Sec. 4.5).  Closed intervals [lo, hi].             */
/* ------------------------------------------------------------------------ */

void or_iv_add(const double a[2], const double b[2], double out[2]) {
  out[0] = a[0] + b[0];
  out[1] = a[1] + b[1];
}

void or_iv_mul(const double a[2], const double b[2], double out[2]) {
  double p[4] = {a[0] * b[0], a[0] * b[1], a[1] * b[0], a[1] * b[1]};
  double lo = p[0], hi = p[0];
  for (int k = 1; k < 4; ++k) {
    if (p[k] < lo) lo = p[k];
    if (p[k] > hi) hi = p[k];
  }
  out[0] = lo;
  out[1] = hi;
}

void or_iv_scale(double k, const double a[2], double out[2]) {
  double x = k * a[0], y = k * a[1];
  out[0] = x < y ? x : y;
  out[1] = x < y ? y : x;
}

/* exact range of cos over [x0, x1]: the end values, widened to +-1 wherever
 * the interval contains a multiple of 2 pi (max) or an odd multiple of pi
 * (min). */
void or_iv_cos(const double x[2], double out[2]) {
  double c0 = cos(x[0]), c1 = cos(x[1]);
  double lo = c0 < c1 ? c0 : c1, hi = c0 < c1 ? c1 : c0;
  if (x[1] - x[0] >= TWO_PI) { out[0] = -1.0; out[1] = 1.0; return; }
  /* smallest multiple of pi that is >= x0 */
  double m = ceil(x[0] / PI);
  for (double k = m; k * PI <= x[1]; k += 1.0) {
    long kk = (long)k;
    if (kk % 2 == 0) hi = 1.0; else lo = -1.0;
  }
  out[0] = lo;
  out[1] = hi;
}

void or_iv_sin(const double x[2], double out[2]) {
  /* sin x = cos(x - pi/2) */
  double y[2] = {x[0] - 0.5 * PI, x[1] - 0.5 * PI};
  or_iv_cos(y, out);
}

/* ------------------------------------------------------------------------ */
/* Interval occupancy region (Def 7) and 4D occupancy region (Def 8).      */
/* ------------------------------------------------------------------------ */

static float to_float_down(double x) {
  float f = (float)x;
  if ((double)f > x) f = nextafterf(f, -INFINITY);
  return f;
}

static float to_float_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, INFINITY);
  return f;
}

static double eccentric_anomaly_at(const double *el, double t_s) {
  double M = el[5] + or_mean_motion(el) * t_s;
  return or_solve_kepler(M, el[1], NULL);
}

void or_box(const double *el, int mode, int64_t tlo, int64_t thi,
            double tick_s, float lo4[4], float hi4[4], double c_out[3],
            double *hw_out) {
  double r = el[6];
  double lo[3], hi[3];
  if (mode == OR_BOX_SPEED) {
    /* Every point of the arc over [t0, t1] lies within vmax |t - tc| of the
     * midpoint position (speed never exceeds the perigee speed), and the
     * 2-norm bounds the infinity norm, so the cube of half-width
     * r + vmax (t1 - t0)/2 around pos(tc) contains occ(w, t) for all t. */
    double tc = 0.5 * (double)(tlo + thi) * tick_s;
    double c[3];
    or_position(el, tc, c);
    double hw = r + or_max_speed(el) * (double)(thi - tlo) * tick_s * 0.5 + OR_EPS_KM;
    for (int k = 0; k < 3; ++k) { lo[k] = c[k] - hw; hi[k] = c[k] + hw; }
    if (c_out) { c_out[0] = c[0]; c_out[1] = c[1]; c_out[2] = c[2]; }
    if (hw_out) *hw_out = hw;
  } else {
    /* Sec. 4.5: the single orbital variable is monotone in time, so its
     * values at the two ends bound it over the interval; the position is
     * then bounded by interval evaluation of
     *   pos(E) = a (cos E - e) P + a sqrt(1-e^2) sin E Q,
     * P and Q the perifocal unit axes in ECI. */
    double a = el[0], e = el[1];
    double E[2] = {eccentric_anomaly_at(el, (double)tlo * tick_s),
                   eccentric_anomaly_at(el, (double)thi * tick_s)};
    double cE[2], sE[2];
    or_iv_cos(E, cE);
    or_iv_sin(E, sE);
    double ux[3] = {1.0, 0.0, 0.0}, uy[3] = {0.0, 1.0, 0.0};
    double P[3], Q[3];
    perifocal_to_eci(el, ux, P);
    perifocal_to_eci(el, uy, Q);
    double b = a * sqrt(1.0 - e * e);
    double cm[2] = {cE[0] - e, cE[1] - e};
    for (int k = 0; k < 3; ++k) {
      double t1[2], t2[2], s[2];
      or_iv_scale(a * P[k], cm, t1);
      or_iv_scale(b * Q[k], sE, t2);
      or_iv_add(t1, t2, s);
      lo[k] = s[0] - r - OR_EPS_KM;
      hi[k] = s[1] + r + OR_EPS_KM;
    }
    if (c_out) or_position(el, (double)tlo * tick_s, c_out);
    if (hw_out) *hw_out = NAN;
  }
  for (int k = 0; k < 3; ++k) {
    lo4[k] = to_float_down(lo[k]);
    hi4[k] = to_float_up(hi[k]);
  }
  lo4[3] = (float)tlo;
  hi4[3] = (float)thi;
}

int64_t or_boxes(const double *els, int64_t n, int64_t T, double tick_s,
                 const int64_t *k, int mode, float *lo4, float *hi4,
                 uint32_t *obj, int64_t cap) {
  int64_t N = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t ki = k[i];
    int64_t S = (T + 1 + ki - 1) / ki;
    for (int64_t m = 0; m < S; ++m) {
      if (N < cap) {
        int64_t tlo = m * ki;
        int64_t thi = (m + 1) * ki - 1;
        if (thi > T) thi = T;
        or_box(els + 7 * i, mode, tlo, thi, tick_s, lo4 + 4 * N, hi4 + 4 * N, NULL, NULL);
        obj[N] = (uint32_t)i;
      }
      ++N;
    }
  }
  return N;
}

/* The boxes of or_boxes whose segments start at a tick in [t0, t1), in the
 * same order: a window of the whole screen's box set (segments are cut from
 * the whole horizon [0, T], so a window's boxes are whole segments). */
int64_t or_boxes_starting(const double *els, int64_t n, int64_t T, double tick_s,
                          const int64_t *k, int mode, int64_t t0, int64_t t1, float *lo4,
                          float *hi4, uint32_t *obj, int64_t cap) {
  int64_t N = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t ki = k[i];
    int64_t S = (T + 1 + ki - 1) / ki;
    int64_t m0 = t0 > 0 ? (t0 + ki - 1) / ki : 0; /* first segment starting at or after t0 */
    for (int64_t m = m0; m < S && m * ki < t1; ++m) {
      if (N < cap) {
        int64_t tlo = m * ki;
        int64_t thi = (m + 1) * ki - 1;
        if (thi > T) thi = T;
        or_box(els + 7 * i, mode, tlo, thi, tick_s, lo4 + 4 * N, hi4 + 4 * N, NULL, NULL);
        obj[N] = (uint32_t)i;
      }
      ++N;
    }
  }
  return N;
}

/* ------------------------------------------------------------------------ */
/* Pair sets.                                                               */
/* ------------------------------------------------------------------------ */

static int boxes_overlap(const float *la, const float *ha, const float *lb, const float *hb) {
  /* closed boxes (Def 2 uses <=) overlap iff they overlap on every axis */
  for (int k = 0; k < 4; ++k)
    if (!(la[k] <= hb[k] && lb[k] <= ha[k])) return 0;
  return 1;
}

static void make_cell(const float *lo4, const float *hi4, const uint32_t *obj,
                      int64_t a, int64_t b, or_cell *c) {
  uint32_t oa = obj[a], ob = obj[b];
  c->i = oa < ob ? oa : ob;
  c->j = oa < ob ? ob : oa;
  int32_t ta0 = (int32_t)lo4[4 * a + 3], ta1 = (int32_t)hi4[4 * a + 3];
  int32_t tb0 = (int32_t)lo4[4 * b + 3], tb1 = (int32_t)hi4[4 * b + 3];
  c->tlo = ta0 > tb0 ? ta0 : tb0;
  c->thi = ta1 < tb1 ? ta1 : tb1;
}

int64_t or_raw_cells_bruteforce(const float *lo4, const float *hi4,
                                const uint32_t *obj, int64_t N,
                                or_cell *out, int64_t cap) {
  int64_t c = 0;
  for (int64_t a = 0; a < N; ++a)
    for (int64_t b = a + 1; b < N; ++b) {
      if (obj[a] == obj[b]) continue;
      if (!boxes_overlap(lo4 + 4 * a, hi4 + 4 * a, lo4 + 4 * b, hi4 + 4 * b)) continue;
      if (c < cap) make_cell(lo4, hi4, obj, a, b, out + c);
      ++c;
    }
  return c;
}

/* ------------------------------------------------------------------------ */
/* The paper's data structure (Sec. 3.2): an AABB tree built by incremental  */
/* insert under a surface-area heuristic, answering "which boxes meet this  */
/* box" by descending from the root.  Nodes link by index (parent, two      */
/* children); leaves carry a box index.  In 4D the "surface area" of a box  */
/* with extents a, b, c, d is the 3-volume of its boundary,                 */
/* 2 (abc + abd + acd + bcd).  Insertion descends to the sibling that the   */
/* heuristic prefers and refits the ancestors; no rotations (optional in    */
/* the paper), which changes the tree's shape, never its answers.           */
/* ------------------------------------------------------------------------ */

typedef struct {
  double lo[4], hi[4];
  int64_t parent, c0, c1; /* -1: none; a leaf has no children */
  int64_t box;            /* leaf: the box index */
} or_tnode;

typedef struct {
  or_tnode *n;
  int64_t count, root;
} or_tree;

static double tsurface(const double *lo, const double *hi) {
  double a = hi[0] - lo[0], b = hi[1] - lo[1], c = hi[2] - lo[2], d = hi[3] - lo[3];
  return 2.0 * (a * b * c + a * b * d + a * c * d + b * c * d);
}

static double tsurface_union(const or_tnode *x, const double *lo, const double *hi) {
  double ul[4], uh[4];
  for (int k = 0; k < 4; ++k) {
    ul[k] = x->lo[k] < lo[k] ? x->lo[k] : lo[k];
    uh[k] = x->hi[k] > hi[k] ? x->hi[k] : hi[k];
  }
  return tsurface(ul, uh);
}

static void tunion_into(or_tnode *dst, const or_tnode *a, const or_tnode *b) {
  for (int k = 0; k < 4; ++k) {
    dst->lo[k] = a->lo[k] < b->lo[k] ? a->lo[k] : b->lo[k];
    dst->hi[k] = a->hi[k] > b->hi[k] ? a->hi[k] : b->hi[k];
  }
}

static void tree_insert(or_tree *t, const float *lo4, const float *hi4, int64_t box) {
  int64_t leaf = t->count++;
  or_tnode *L = t->n + leaf;
  for (int k = 0; k < 4; ++k) {
    L->lo[k] = lo4[4 * box + k];
    L->hi[k] = hi4[4 * box + k];
  }
  L->parent = L->c0 = L->c1 = -1;
  L->box = box;
  if (t->root < 0) {
    t->root = leaf;
    return;
  }
  /* descend: pairing with node x costs its union's surface; going below x
   * adds the growth of x to whatever the child costs */
  int64_t x = t->root;
  while (t->n[x].c0 >= 0) {
    or_tnode *X = t->n + x;
    double here = tsurface_union(X, L->lo, L->hi);
    double grow = here - tsurface(X->lo, X->hi);
    double cost[2];
    for (int c = 0; c < 2; ++c) {
      const or_tnode *C = t->n + (c ? X->c1 : X->c0);
      double u = tsurface_union(C, L->lo, L->hi);
      cost[c] = grow + (C->c0 >= 0 ? u - tsurface(C->lo, C->hi) : u);
    }
    if (here <= cost[0] && here <= cost[1]) break;
    x = cost[0] <= cost[1] ? X->c0 : X->c1;
  }
  /* a new parent for x and the leaf */
  int64_t np = t->count++;
  or_tnode *P = t->n + np;
  int64_t old = t->n[x].parent;
  P->parent = old;
  P->c0 = x;
  P->c1 = leaf;
  P->box = -1;
  tunion_into(P, t->n + x, L);
  t->n[x].parent = np;
  L->parent = np;
  if (old < 0) {
    t->root = np;
  } else if (t->n[old].c0 == x) {
    t->n[old].c0 = np;
  } else {
    t->n[old].c1 = np;
  }
  /* refit the ancestors */
  for (int64_t a = old; a >= 0; a = t->n[a].parent)
    tunion_into(t->n + a, t->n + t->n[a].c0, t->n + t->n[a].c1);
}

static int tnode_meets(const or_tnode *x, const float *lo, const float *hi) {
  for (int k = 0; k < 4; ++k)
    if (x->lo[k] > (double)hi[k] || (double)lo[k] > x->hi[k]) return 0;
  return 1;
}

int64_t or_raw_cells_tree(const float *lo4, const float *hi4, const uint32_t *obj, int64_t N,
                          or_cell *out, int64_t cap) {
  or_tree t;
  t.n = (or_tnode *)malloc(sizeof(or_tnode) * (size_t)(2 * N + 1));
  t.count = 0;
  t.root = -1;
  for (int64_t b = 0; b < N; ++b) tree_insert(&t, lo4, hi4, b);
  int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * N + 1));
  int64_t c = 0;
  for (int64_t a = 0; a < N && t.root >= 0; ++a) {
    const float *ql = lo4 + 4 * a, *qh = hi4 + 4 * a;
    int64_t sp = 0;
    stack[sp++] = t.root;
    while (sp > 0) {
      const or_tnode *x = t.n + stack[--sp];
      if (!tnode_meets(x, ql, qh)) continue;
      if (x->c0 >= 0) {
        stack[sp++] = x->c0;
        stack[sp++] = x->c1;
        continue;
      }
      int64_t b = x->box; /* each pair once, from its lower box index */
      if (b <= a || obj[a] == obj[b]) continue;
      if (c < cap) make_cell(lo4, hi4, obj, a, b, out + c);
      ++c;
    }
  }
  free(stack);
  free(t.n);
  return c;
}

/* the boxes qsort's comparison reads; one per thread, so that calls from
 * several host threads do not share it */
static _Thread_local const float *g_sort_lo;
static int cmp_by_tlo(const void *x, const void *y) {
  int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
  float ta = g_sort_lo[4 * a + 3], tb = g_sort_lo[4 * b + 3];
  if (ta < tb) return -1;
  if (ta > tb) return 1;
  return (a > b) - (a < b);
}

static int64_t *sorted_by_tlo(const float *lo4, int64_t N) {
  int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  for (int64_t a = 0; a < N; ++a) ord[a] = a;
  g_sort_lo = lo4;
  qsort(ord, (size_t)N, sizeof(int64_t), cmp_by_tlo);
  return ord;
}

int64_t or_raw_cells_sweep(const float *lo4, const float *hi4,
                           const uint32_t *obj, int64_t N,
                           or_cell *out, int64_t cap) {
  int64_t *ord = sorted_by_tlo(lo4, N);
  int64_t c = 0;
  for (int64_t p = 0; p < N; ++p) {
    int64_t a = ord[p];
    float tend = hi4[4 * a + 3];
    for (int64_t q = p + 1; q < N && lo4[4 * ord[q] + 3] <= tend; ++q) {
      int64_t b = ord[q];
      if (obj[a] == obj[b]) continue;
      if (!boxes_overlap(lo4 + 4 * a, hi4 + 4 * a, lo4 + 4 * b, hi4 + 4 * b)) continue;
      if (c < cap) make_cell(lo4, hi4, obj, a, b, out + c);
      ++c;
    }
  }
  free(ord);
  return c;
}

/* or_raw_cells_sweep restricted to the pairs whose earlier box in the
 * sweep's order (by lower tick, then index) starts before tick t_end.  Over
 * windows [t0, t1) of the lower ticks, with the boxes starting in
 * [t0, t1 + longest box) as input each time, these pair sets partition the
 * whole screen's: every pair is found from its earlier box, in the window
 * where that box starts. */
int64_t or_raw_cells_sweep_before(const float *lo4, const float *hi4,
                                  const uint32_t *obj, int64_t N, int64_t t_end,
                                  or_cell *out, int64_t cap) {
  int64_t *ord = sorted_by_tlo(lo4, N);
  int64_t c = 0;
  for (int64_t p = 0; p < N && (int64_t)lo4[4 * ord[p] + 3] < t_end; ++p) {
    int64_t a = ord[p];
    float tend = hi4[4 * a + 3];
    for (int64_t q = p + 1; q < N && lo4[4 * ord[q] + 3] <= tend; ++q) {
      int64_t b = ord[q];
      if (obj[a] == obj[b]) continue;
      if (!boxes_overlap(lo4 + 4 * a, hi4 + 4 * a, lo4 + 4 * b, hi4 + 4 * b)) continue;
      if (c < cap) make_cell(lo4, hi4, obj, a, b, out + c);
      ++c;
    }
  }
  free(ord);
  return c;
}

int64_t or_raw_cells_selected(const float *lo4, const float *hi4,
                              const uint32_t *obj, int64_t N,
                              const uint8_t *sel, or_cell *out, int64_t cap) {
  int64_t *ord = sorted_by_tlo(lo4, N);
  /* longest box in ticks: a box b can meet box a only if
   * tlo_b in [tlo_a - maxlen, thi_a] */
  float maxlen = 0.0f;
  for (int64_t a = 0; a < N; ++a) {
    float L = hi4[4 * a + 3] - lo4[4 * a + 3];
    if (L > maxlen) maxlen = L;
  }
  int64_t c = 0;
  for (int64_t a = 0; a < N; ++a) {
    if (!sel[obj[a]]) continue;
    float t0 = lo4[4 * a + 3] - maxlen, t1 = hi4[4 * a + 3];
    /* first sorted position with tlo >= t0 */
    int64_t lo = 0, hi = N;
    while (lo < hi) {
      int64_t mid = (lo + hi) / 2;
      if (lo4[4 * ord[mid] + 3] < t0) lo = mid + 1; else hi = mid;
    }
    for (int64_t q = lo; q < N && lo4[4 * ord[q] + 3] <= t1; ++q) {
      int64_t b = ord[q];
      if (obj[a] == obj[b]) continue;
      if (sel[obj[b]] && b < a) continue; /* counted from b's side */
      if (!boxes_overlap(lo4 + 4 * a, hi4 + 4 * a, lo4 + 4 * b, hi4 + 4 * b)) continue;
      if (c < cap) make_cell(lo4, hi4, obj, a, b, out + c);
      ++c;
    }
  }
  free(ord);
  return c;
}

static int cmp_cell(const void *x, const void *y) {
  const or_cell *a = (const or_cell *)x, *b = (const or_cell *)y;
  if (a->i != b->i) return a->i < b->i ? -1 : 1;
  if (a->j != b->j) return a->j < b->j ? -1 : 1;
  if (a->tlo != b->tlo) return a->tlo < b->tlo ? -1 : 1;
  if (a->thi != b->thi) return a->thi < b->thi ? -1 : 1;
  return 0;
}

int64_t or_canonicalize(or_cell *cells, int64_t n) {
  if (n <= 0) return 0;
  qsort(cells, (size_t)n, sizeof(or_cell), cmp_cell);
  int64_t w = 0;
  for (int64_t r = 1; r < n; ++r) {
    or_cell *cur = cells + w;
    const or_cell *nx = cells + r;
    if (nx->i == cur->i && nx->j == cur->j && (int64_t)nx->tlo <= (int64_t)cur->thi + 1) {
      if (nx->thi > cur->thi) cur->thi = nx->thi;
    } else {
      cells[++w] = *nx;
    }
  }
  return w + 1;
}

/* ------------------------------------------------------------------------ */
/* Alg 1: brute force over every tick and every pair.                      */
/* ------------------------------------------------------------------------ */

static int occ_collide(const double *pi, double ri, const double *pj, double rj) {
  /* Def 3 with Def 2: two closed cubes meet iff their centres are within
   * r_i + r_j in the infinity norm */
  for (int k = 0; k < 3; ++k)
    if (fabs(pi[k] - pj[k]) > ri + rj) return 0;
  return 1;
}

int64_t or_alg1_witnesses(const double *els, int64_t n, int64_t T,
                          double tick_s, or_witness *out, int64_t cap) {
  double *pos = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  int64_t c = 0;
  for (int64_t t = 0; t <= T; ++t) {
    for (int64_t i = 0; i < n; ++i) or_position(els + 7 * i, (double)t * tick_s, pos + 3 * i);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = i + 1; j < n; ++j)
        if (occ_collide(pos + 3 * i, els[7 * i + 6], pos + 3 * j, els[7 * j + 6])) {
          if (c < cap) {
            out[c].i = (uint32_t)i;
            out[c].j = (uint32_t)j;
            out[c].t = (int32_t)t;
          }
          ++c;
        }
  }
  free(pos);
  return c;
}

/* ------------------------------------------------------------------------ */
/* Narrow phase: the collision witnesses (Def 4) inside a candidate list.  */
/* For each candidate (i, j, [tlo, thi]) every tick t of the interval is   */
/* tested with the same predicate as Alg 1 (Defs 2-3: centres within       */
/* r_i + r_j in the infinity norm, positions by the Sec. 6.1 propagation). */
/* Per candidate: the first witness tick (-1: none), the witness count and */
/* the smallest |d_inf - (r_i + r_j)| over its ticks (how close the        */
/* decisions came to the boundary).  Witnesses are listed in candidate     */
/* order, ticks ascending.  Returns the witness count, or -1 if a          */
/* candidate names an object >= n or has tlo > thi or tlo < 0.             */
/* ------------------------------------------------------------------------ */
int64_t or_narrow_phase(const double *els, int64_t n, const or_cell *cand, int64_t m,
                        double tick_s, int32_t *first, uint32_t *count, double *margin,
                        or_witness *out, int64_t cap) {
  int64_t c = 0;
  for (int64_t q = 0; q < m; ++q) {
    const or_cell x = cand[q];
    if ((int64_t)x.i >= n || (int64_t)x.j >= n || x.tlo < 0 || x.tlo > x.thi) return -1;
    const double *ei = els + 7 * (int64_t)x.i, *ej = els + 7 * (int64_t)x.j;
    const double R = ei[6] + ej[6];
    int32_t f = -1;
    uint32_t k = 0;
    double mg = INFINITY;
    for (int64_t t = x.tlo; t <= x.thi; ++t) {
      double pi[3], pj[3];
      or_position(ei, (double)t * tick_s, pi);
      or_position(ej, (double)t * tick_s, pj);
      double d = 0.0;
      for (int a = 0; a < 3; ++a)
        if (fabs(pi[a] - pj[a]) > d) d = fabs(pi[a] - pj[a]);
      if (fabs(d - R) < mg) mg = fabs(d - R);
      if (!occ_collide(pi, ei[6], pj, ej[6])) continue;
      if (f < 0) f = (int32_t)t;
      ++k;
      if (out && c < cap) {
        out[c].i = x.i;
        out[c].j = x.j;
        out[c].t = (int32_t)t;
      }
      ++c;
    }
    if (first) first[q] = f;
    if (count) count[q] = k;
    if (margin) margin[q] = mg;
  }
  return c;
}

/* Alg 1 over ticks t0..t1 (inclusive) with the pairs restricted by a sweep
 * along x: two objects can only meet (Def 3) if their x centres are within
 * r_i + r_j <= 2 max r, so after sorting by x only pairs inside that window
 * are tested, with the same predicate.  Each witness also gets the
 * Euclidean distance of the two centres (dist[k]).  Witnesses come in tick
 * order; within a tick in sweep order (i < j in each). */
typedef struct {
  double x;
  int64_t i;
} or_xkey;

static int cmp_xkey(const void *a, const void *b) {
  double xa = ((const or_xkey *)a)->x, xb = ((const or_xkey *)b)->x;
  return (xa > xb) - (xa < xb);
}

int64_t or_alg1_sweep(const double *els, int64_t n, int64_t t0, int64_t t1, double tick_s,
                      or_witness *out, double *dist, int64_t cap) {
  double *pos = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  or_xkey *key = (or_xkey *)malloc(sizeof(or_xkey) * (size_t)(n > 0 ? n : 1));
  double rmax = 0.0;
  for (int64_t i = 0; i < n; ++i)
    if (els[7 * i + 6] > rmax) rmax = els[7 * i + 6];
  int64_t c = 0;
  for (int64_t t = t0; t <= t1; ++t) {
    for (int64_t i = 0; i < n; ++i) {
      or_position(els + 7 * i, (double)t * tick_s, pos + 3 * i);
      key[i].x = pos[3 * i];
      key[i].i = i;
    }
    qsort(key, (size_t)n, sizeof(or_xkey), cmp_xkey);
    for (int64_t a = 0; a < n; ++a)
      for (int64_t b = a + 1; b < n && key[b].x - key[a].x <= 2.0 * rmax; ++b) {
        int64_t i = key[a].i < key[b].i ? key[a].i : key[b].i;
        int64_t j = key[a].i < key[b].i ? key[b].i : key[a].i;
        if (!occ_collide(pos + 3 * i, els[7 * i + 6], pos + 3 * j, els[7 * j + 6])) continue;
        if (c < cap) {
          double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1],
                 dz = pos[3 * i + 2] - pos[3 * j + 2];
          out[c].i = (uint32_t)i;
          out[c].j = (uint32_t)j;
          out[c].t = (int32_t)t;
          dist[c] = sqrt(dx * dx + dy * dy + dz * dz);
        }
        ++c;
      }
  }
  free(key);
  free(pos);
  return c;
}

/* ------------------------------------------------------------------------ */
/* Alg 3 with Alg 4 (initializeTree), getSmallestMaxTimeObject, Alg 5      */
/* (advanceTime) and Alg 6 (resolveCollisions).  The AABB tree's job is to  */
/* answer "which boxes meet this box"; a flat list answers the same query. */
/* ------------------------------------------------------------------------ */

typedef struct {
  const double *els;
  int64_t n;
  double tick_s;
  int mode;
  int64_t *tmin, *tmax;
  float *lo, *hi; /* current occ-4d box of each object */
} alg3_state;

static void a3_update(alg3_state *s, int64_t w) {
  or_box(s->els + 7 * w, s->mode, s->tmin[w], s->tmax[w], s->tick_s,
         s->lo + 4 * w, s->hi + 4 * w, NULL, NULL);
}

static int a3_meet(const alg3_state *s, int64_t a, int64_t b) {
  return boxes_overlap(s->lo + 4 * a, s->hi + 4 * a, s->lo + 4 * b, s->hi + 4 * b);
}

/* queryObject: all objects whose box meets v's box, v excluded */
static int64_t a3_query(const alg3_state *s, int64_t v, int64_t *out) {
  int64_t c = 0;
  for (int64_t y = 0; y < s->n; ++y)
    if (y != v && a3_meet(s, v, y)) out[c++] = y;
  return c;
}

int or_alg3(const double *els, int64_t n, int64_t T, double tick_s, int mode,
            int64_t t_first, uint32_t *wi, uint32_t *wj, int64_t *wt,
            int64_t *iterations) {
  alg3_state s;
  s.els = els; s.n = n; s.tick_s = tick_s; s.mode = mode;
  s.tmin = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  s.tmax = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  s.lo = (float *)malloc(sizeof(float) * 4 * (size_t)n);
  s.hi = (float *)malloc(sizeof(float) * 4 * (size_t)n);
  int64_t *l = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int rc = 0;
  int64_t iters = 0;

  /* Alg 4: insert every object at [0, 0]; an overlap is a collision at 0 */
  for (int64_t i = 0; i < n; ++i) {
    s.tmin[i] = 0; s.tmax[i] = 0;
    a3_update(&s, i);
    for (int64_t y = 0; y < i; ++y)
      if (a3_meet(&s, i, y)) {
        *wi = (uint32_t)y; *wj = (uint32_t)i; *wt = 0;
        rc = 1;
        goto done;
      }
  }

  for (;;) {
    /* getSmallestMaxTimeObject: ties go to the lowest index */
    int64_t v = 0;
    for (int64_t z = 1; z < n; ++z)
      if (s.tmax[z] < s.tmax[v]) v = z;
    int64_t tp = s.tmax[v];
    /* Loop Invariant 1: every t_min <= t' + delta */
    for (int64_t z = 0; z < n; ++z)
      if (s.tmin[z] > tp + 1) { rc = -1; goto done; }
    /* Loop Invariant 2: no actual collision up to t' */
    if (t_first >= 0 && t_first <= tp) { rc = -2; goto done; }
    if (tp >= T) break;
    if (++iters > 100000000) { rc = -3; goto done; }

    /* Alg 5: advanceTime */
    int64_t prev = s.tmax[v] - s.tmin[v];
    int64_t next = prev > 0 ? 2 * prev : 1;
    s.tmin[v] = s.tmax[v] + 1;
    s.tmax[v] = s.tmin[v] + next;
    if (s.tmax[v] > T) s.tmax[v] = T;
    a3_update(&s, v);

    /* Alg 6: resolveCollisions */
    int64_t nl = a3_query(&s, v, l);
    while (nl > 0) {
      for (int64_t q = 0; q < nl; ++q) {
        int64_t y = l[q];
        if (!a3_meet(&s, y, v)) continue;
        int64_t sy = s.tmax[y] - s.tmin[y];
        int64_t sv = s.tmax[v] - s.tmin[v];
        if (sy == 0 && sv == 0) {
          *wi = (uint32_t)(v < y ? v : y);
          *wj = (uint32_t)(v < y ? y : v);
          *wt = s.tmin[v];
          rc = 1;
          goto done;
        } else if (s.tmin[y] < s.tmin[v]) {
          /* the branch raises y's t_min to v's (the text of Sec. 4.4) */
          s.tmin[y] = s.tmin[v];
          a3_update(&s, y);
        } else if (sv <= sy) {
          s.tmax[y] = s.tmin[y] + sy / 2;
          a3_update(&s, y);
        } else {
          s.tmax[v] = s.tmin[v] + sv / 2;
          a3_update(&s, v);
        }
      }
      nl = a3_query(&s, v, l);
    }
  }
done:
  if (iterations) *iterations = iters;
  free(s.tmin); free(s.tmax); free(s.lo); free(s.hi); free(l);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Adaptive refinement in bulk-synchronous rounds: the interval doubling    */
/* and halving of Alg 5 and Alg 6 taken top-down over all objects at once. */
/* Every object starts with the whole horizon, or with it cut into        */
/* intervals of a bounded length (or_refine_start_ticks).  In a round      */
/* every active interval gets its 4D box (Def 8); a box that meets no box  */
/* of another object proves its object collision-free over the interval    */
/* (every other object's position at those times lies in one of this       */
/* round's boxes, or was proven free of collisions in an earlier round),   */
/* so the interval is done; an interval whose box meets another is halved, */
/* as Alg 6 halves the longer of two overlapping intervals.  Property 2    */
/* keeps the halves inside the parent box.                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t obj, t0, t1;
} or_seg;

static void *grow(void *p, int64_t *cap, int64_t need, size_t elem) {
  if (need <= *cap) return p;
  int64_t c = *cap > 0 ? *cap : 64;
  while (c < need) c *= 2;
  *cap = c;
  return realloc(p, (size_t)c * elem);
}

static int cmp_witness_alg1(const void *x, const void *y) {
  const or_witness *a = (const or_witness *)x, *b = (const or_witness *)y;
  if (a->t != b->t) return a->t < b->t ? -1 : 1;
  if (a->i != b->i) return a->i < b->i ? -1 : 1;
  if (a->j != b->j) return a->j < b->j ? -1 : 1;
  return 0;
}

int64_t or_refine_start_ticks(const double *el, int64_t T, double tick_s, double fraction) {
  if (!(fraction > 0.0)) return T + 1;
  const double q = floor(or_period(el) / (fraction * tick_s));
  int64_t L = 1;
  while (L <= T && (double)(2 * L) <= q) L *= 2; /* beyond T the length is T + 1 anyway */
  return L > T ? T + 1 : L;
}

int64_t or_refine_discrete(const double *els, int64_t n, int64_t T, double tick_s, int mode,
                           double start_fraction, or_witness *out, int64_t cap,
                           int64_t *round_boxes, int *rounds, int64_t *n_tick_candidates) {
  int64_t m = 0, scap = 0, ncap = 0, ccap = 0, nc = 0;
  or_seg *S = NULL;
  or_seg *next = NULL;
  or_witness *cand = NULL;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t L = or_refine_start_ticks(els + 7 * i, T, tick_s, start_fraction);
    for (int64_t t0 = 0; t0 <= T; t0 += L) {
      S = (or_seg *)grow(S, &scap, m + 1, sizeof(or_seg));
      S[m].obj = i;
      S[m].t0 = t0;
      S[m].t1 = t0 + L - 1 < T ? t0 + L - 1 : T;
      ++m;
    }
  }
  if (!S) S = (or_seg *)grow(NULL, &scap, 1, sizeof(or_seg));
  int r = 0;
  while (m > 0 && r < 64) {
    if (round_boxes) round_boxes[r] = m;
    float *lo = (float *)malloc(sizeof(float) * 4 * (size_t)m);
    float *hi = (float *)malloc(sizeof(float) * 4 * (size_t)m);
    char *hit = (char *)calloc((size_t)m, 1), *hit_long = (char *)calloc((size_t)m, 1);
    for (int64_t a = 0; a < m; ++a)
      or_box(els + 7 * S[a].obj, mode, S[a].t0, S[a].t1, tick_s, lo + 4 * a, hi + 4 * a, NULL,
             NULL);
    for (int64_t a = 0; a < m; ++a)
      for (int64_t b = a + 1; b < m; ++b) {
        if (S[a].obj == S[b].obj) continue;
        if (!boxes_overlap(lo + 4 * a, hi + 4 * a, lo + 4 * b, hi + 4 * b)) continue;
        hit[a] = hit[b] = 1;
        const int la = S[a].t1 > S[a].t0, lb = S[b].t1 > S[b].t0;
        if (lb) hit_long[a] = 1;
        if (la) hit_long[b] = 1;
        if (!la && !lb) { /* two single ticks (the same tick: the boxes meet in time) */
          cand = (or_witness *)grow(cand, &ccap, nc + 1, sizeof(or_witness));
          cand[nc].i = (uint32_t)(S[a].obj < S[b].obj ? S[a].obj : S[b].obj);
          cand[nc].j = (uint32_t)(S[a].obj < S[b].obj ? S[b].obj : S[a].obj);
          cand[nc].t = (int32_t)S[a].t0;
          ++nc;
        }
      }
    int64_t mn = 0;
    for (int64_t a = 0; a < m; ++a) {
      if (!hit[a]) continue; /* proven free of collisions over [t0, t1] */
      if (S[a].t1 > S[a].t0) {
        const int64_t mid = S[a].t0 + (S[a].t1 - S[a].t0) / 2;
        next = (or_seg *)grow(next, &ncap, mn + 2, sizeof(or_seg));
        next[mn].obj = S[a].obj;
        next[mn].t0 = S[a].t0;
        next[mn].t1 = mid;
        next[mn + 1].obj = S[a].obj;
        next[mn + 1].t0 = mid + 1;
        next[mn + 1].t1 = S[a].t1;
        mn += 2;
      } else if (hit_long[a]) { /* wait for the longer intervals it meets to halve */
        next = (or_seg *)grow(next, &ncap, mn + 1, sizeof(or_seg));
        next[mn++] = S[a];
      }
    }
    free(lo);
    free(hi);
    free(hit);
    free(hit_long);
    or_seg *tmp = S;
    int64_t tcap = scap;
    S = next;
    scap = ncap;
    next = tmp;
    ncap = tcap;
    m = mn;
    ++r;
  }
  if (rounds) *rounds = r;
  /* tick candidates, once each, then Alg 1's test at the tick */
  if (nc > 0) qsort(cand, (size_t)nc, sizeof(or_witness), cmp_witness_alg1);
  int64_t u = 0;
  for (int64_t q = 0; q < nc; ++q)
    if (u == 0 || cmp_witness_alg1(&cand[u - 1], &cand[q]) != 0) cand[u++] = cand[q];
  if (n_tick_candidates) *n_tick_candidates = u;
  int64_t c = 0;
  for (int64_t q = 0; q < u; ++q) {
    const double *ei = els + 7 * (int64_t)cand[q].i, *ej = els + 7 * (int64_t)cand[q].j;
    double pi[3], pj[3];
    or_position(ei, (double)cand[q].t * tick_s, pi);
    or_position(ej, (double)cand[q].t * tick_s, pj);
    if (!occ_collide(pi, ei[6], pj, ej[6])) continue;
    if (c < cap) out[c] = cand[q];
    ++c;
  }
  free(S);
  free(next);
  free(cand);
  return c;
}

/* The continuous-time variant (Sec. 4.6): the same rounds over closed real
 * intervals, halved down to length eps_s; consecutive halves share their
 * endpoint (t_min of the second = t_max of the first).  At the finest
 * level every pair of meeting boxes is reported with the intersection of
 * the two intervals: any collision at any real time lies in a reported
 * span (sound without a time step), and with interval boxes the spans'
 * boxes shrink to the occupancy regions as eps_s goes to 0. */
static int cmp_span(const void *x, const void *y) {
  const or_span *a = (const or_span *)x, *b = (const or_span *)y;
  if (a->i != b->i) return a->i < b->i ? -1 : 1;
  if (a->j != b->j) return a->j < b->j ? -1 : 1;
  if (a->t0 != b->t0) return a->t0 < b->t0 ? -1 : 1;
  if (a->t1 != b->t1) return a->t1 < b->t1 ? -1 : 1;
  return 0;
}

/* One round of the refinement applied to given boxes: m active intervals
 * with their FP32 boxes lo4/hi4 (the interval's first and last unit in the
 * w lane) and objects.  An interval is met when its box overlaps, closed on
 * all four axes, the box of an interval of another object (every pair
 * tested).  Discrete rule (cont == 0, Alg 5-6 in rounds): a met interval
 * [t0, t1] with t1 > t0 becomes [t0, mid] and [mid + 1, t1], mid = t0 +
 * (t1 - t0) / 2; a met single tick stays when one of the boxes it meets is
 * longer than one tick.  Continuous rule (cont == 1, Sec. 4.6): a met
 * interval [k, k + 1] becomes [2k, 2k + 1] and [2k + 1, 2k + 2].  The next
 * intervals go to nobj, nt0, nt1 (up to cap; in input order); returns how
 * many there are. */
int64_t or_refine_round(const float *lo4, const float *hi4, const uint32_t *obj, int64_t m,
                        int cont, uint32_t *nobj, int32_t *nt0, int32_t *nt1, int64_t cap) {
  char *hit = (char *)calloc((size_t)(m > 0 ? m : 1), 1);
  char *hit_long = (char *)calloc((size_t)(m > 0 ? m : 1), 1);
  for (int64_t a = 0; a < m; ++a)
    for (int64_t b = a + 1; b < m; ++b) {
      if (obj[a] == obj[b]) continue;
      if (!boxes_overlap(lo4 + 4 * a, hi4 + 4 * a, lo4 + 4 * b, hi4 + 4 * b)) continue;
      hit[a] = hit[b] = 1;
      if (hi4[4 * b + 3] > lo4[4 * b + 3]) hit_long[a] = 1;
      if (hi4[4 * a + 3] > lo4[4 * a + 3]) hit_long[b] = 1;
    }
  int64_t mn = 0;
  for (int64_t a = 0; a < m; ++a) {
    if (!hit[a]) continue;
    const int32_t t0 = (int32_t)lo4[4 * a + 3], t1 = (int32_t)hi4[4 * a + 3];
    int32_t u[2][2];
    int k = 0;
    if (cont) {
      u[0][0] = 2 * t0;
      u[0][1] = 2 * t0 + 1;
      u[1][0] = 2 * t0 + 1;
      u[1][1] = 2 * t0 + 2;
      k = 2;
    } else if (t1 > t0) {
      const int32_t mid = t0 + (t1 - t0) / 2;
      u[0][0] = t0;
      u[0][1] = mid;
      u[1][0] = mid + 1;
      u[1][1] = t1;
      k = 2;
    } else if (hit_long[a]) {
      u[0][0] = t0;
      u[0][1] = t1;
      k = 1;
    }
    for (int q = 0; q < k; ++q) {
      if (mn < cap) {
        nobj[mn] = obj[a];
        nt0[mn] = u[q][0];
        nt1[mn] = u[q][1];
      }
      ++mn;
    }
  }
  free(hit);
  free(hit_long);
  return mn;
}

int64_t or_refine_continuous(const double *els, int64_t n, double T_s, double eps_s, int mode,
                             or_span *out, int64_t cap, int64_t *round_boxes, int *rounds) {
  int L = 0;
  while (L < 40 && ldexp(T_s, -L) > eps_s) ++L;
  int64_t m = n, scap = 0, ncap = 0, ocap = 0, no = 0;
  or_seg *S = (or_seg *)grow(NULL, &scap, n > 0 ? n : 1, sizeof(or_seg));
  or_seg *next = NULL;
  or_span *o = NULL;
  for (int64_t i = 0; i < n; ++i) {
    S[i].obj = i;
    S[i].t0 = 0; /* interval [t0, t0 + 1] in units of T_s / 2^level */
    S[i].t1 = 1;
  }
  int r = 0;
  for (int level = 0; level <= L && m > 0; ++level) {
    if (round_boxes) round_boxes[r] = m;
    ++r;
    const double unit = ldexp(T_s, -level);
    float *lo = (float *)malloc(sizeof(float) * 4 * (size_t)m);
    float *hi = (float *)malloc(sizeof(float) * 4 * (size_t)m);
    char *hit = (char *)calloc((size_t)m, 1);
    for (int64_t a = 0; a < m; ++a)
      or_box(els + 7 * S[a].obj, mode, S[a].t0, S[a].t1, unit, lo + 4 * a, hi + 4 * a, NULL,
             NULL);
    for (int64_t a = 0; a < m; ++a)
      for (int64_t b = a + 1; b < m; ++b) {
        if (S[a].obj == S[b].obj) continue;
        if (!boxes_overlap(lo + 4 * a, hi + 4 * a, lo + 4 * b, hi + 4 * b)) continue;
        hit[a] = hit[b] = 1;
        if (level == L) {
          o = (or_span *)grow(o, &ocap, no + 1, sizeof(or_span));
          o[no].i = (uint32_t)(S[a].obj < S[b].obj ? S[a].obj : S[b].obj);
          o[no].j = (uint32_t)(S[a].obj < S[b].obj ? S[b].obj : S[a].obj);
          o[no].t0 = (double)(S[a].t0 > S[b].t0 ? S[a].t0 : S[b].t0) * unit;
          o[no].t1 = (double)(S[a].t1 < S[b].t1 ? S[a].t1 : S[b].t1) * unit;
          ++no;
        }
      }
    int64_t mn = 0;
    if (level < L)
      for (int64_t a = 0; a < m; ++a) {
        if (!hit[a]) continue;
        next = (or_seg *)grow(next, &ncap, mn + 2, sizeof(or_seg));
        next[mn].obj = next[mn + 1].obj = S[a].obj;
        next[mn].t0 = 2 * S[a].t0;
        next[mn].t1 = 2 * S[a].t0 + 1;
        next[mn + 1].t0 = 2 * S[a].t0 + 1;
        next[mn + 1].t1 = 2 * S[a].t0 + 2;
        mn += 2;
      }
    free(lo);
    free(hi);
    free(hit);
    or_seg *tmp = S;
    int64_t tcap = scap;
    S = next;
    scap = ncap;
    next = tmp;
    ncap = tcap;
    m = mn;
  }
  if (rounds) *rounds = r;
  if (no > 0) qsort(o, (size_t)no, sizeof(or_span), cmp_span);
  int64_t u = 0;
  for (int64_t q = 0; q < no; ++q)
    if (u == 0 || cmp_span(&o[u - 1], &o[q]) != 0) o[u++] = o[q];
  for (int64_t q = 0; q < u && q < cap; ++q) out[q] = o[q];
  free(S);
  free(next);
  free(o);
  return u;
}

/* ------------------------------------------------------------------------ */
/* Static decomposition: potential-collision graph from perigee/apogee      */
/* (Sec. 6.1) and altitude bands from every (n/p)-th sorted semi-major axis.*/
/* ------------------------------------------------------------------------ */

void or_radial_range(const double *el, double out[2]) {
  /* a true collision needs ||dpos||_inf <= r_i + r_j, hence
   * | |pos_i| - |pos_j| | <= sqrt(3) (r_i + r_j): padding each object's
   * [perigee, apogee] radius range by sqrt(3) r keeps every such pair. */
  double a = el[0], e = el[1], r = el[6];
  double pad = sqrt(3.0) * r;
  out[0] = a * (1.0 - e) - pad;
  out[1] = a * (1.0 + e) + pad;
}

static int cmp_double(const void *x, const void *y) {
  double a = *(const double *)x, b = *(const double *)y;
  return (a > b) - (a < b);
}

void or_band_edges(const double *els, int64_t n, int p, double *edges) {
  double *a = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) a[i] = els[7 * i];
  qsort(a, (size_t)n, sizeof(double), cmp_double);
  int64_t d = n / p;
  for (int k = 1; k < p; ++k) edges[k - 1] = a[(int64_t)k * d];
  free(a);
}

void or_band_counts(const double *els, int64_t n, int p, int64_t *counts) {
  double *edges = (double *)malloc(sizeof(double) * (size_t)(p > 1 ? p - 1 : 1));
  if (p > 1) or_band_edges(els, n, p, edges);
  for (int k = 0; k < p; ++k) counts[k] = 0;
  for (int64_t i = 0; i < n; ++i) {
    double rr[2];
    or_radial_range(els + 7 * i, rr);
    for (int k = 0; k < p; ++k) {
      double lo = k == 0 ? -INFINITY : edges[k - 1];
      double hi = k == p - 1 ? INFINITY : edges[k];
      /* [rr0, rr1] meets [lo, hi) */
      if (rr[0] < hi && rr[1] >= lo) counts[k]++;
    }
  }
  free(edges);
}
