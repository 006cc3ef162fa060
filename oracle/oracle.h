/*
 * oracle.h -- plain FP64 CPU oracle for 4D space-time box screening
 * (Bak & Hobbs, "Efficient n-to-n Collision Detection for Space Debris using
 * 4D AABB Trees").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this code: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, constant or table with the
 * CUDA library; the two meet only through plain arrays.
 *
 * Every function is the slow, obviously correct form of one definition or
 * algorithm of the paper, cited beside it.  Element layout: 7 doubles per
 * object, in this order: a [km], e, i [rad], RAAN [rad], argument of perigee
 * [rad], mean anomaly at t=0 [rad], radius [km] (Def 1: the object's fixed
 * infinity-norm radius r).  Time is integer ticks of length tick_s seconds
 * (Def 6, discrete-time problem); the horizon T is a tick count and ticks
 * 0..T inclusive are checked (Alg 1 runs t from 0 to T).
 */
#ifndef SCD_ORACLE_H
#define SCD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* geocentric gravitational parameter [km^3/s^2] and Earth radius [km]; the
 * paper names mu in Eq. 1 without a value, these are the WGS-84 figures. */
#define OR_MU 398600.4418
#define OR_RE 6378.137
/* margin added to every half-width before rounding outward to FP32 [km] */
#define OR_EPS_KM 1e-6

#define OR_STEP_FIXED 0
#define OR_STEP_PERIOD_FRACTION 1
#define OR_STEP_BAND_TABLE 2
#define OR_BOX_SPEED 0
#define OR_BOX_INTERVAL 1

/* one candidate: objects i<j may collide at some tick of [tlo, thi] */
typedef struct { uint32_t i, j; int32_t tlo, thi; } or_cell;
/* one collision witness (Def 4): objects i<j collide at tick t */
typedef struct { uint32_t i, j; int32_t t; } or_witness;

/* --- dynamics (Sec. 6.1, Eq. 1) --------------------------------------- */
double or_mean_motion(const double *el);                  /* sqrt(mu/a^3) */
double or_period(const double *el);                       /* 2 pi / n     */
double or_max_speed(const double *el);                    /* perigee speed */
double or_solve_kepler(double M, double e, int *iters);   /* E - e sinE = M */
double or_true_anomaly(const double *el, double t_s);     /* nu(t), continuous */
void   or_position(const double *el, double t_s, double out[3]);
void   or_position_from_nu(const double *el, double nu, double out[3]);
void   or_velocity_fd(const double *el, double t_s, double h_s, double out[3]);
double or_nu_rk4(const double *el, double t_s, double h_s);  /* integrate Eq. 1 */

/* --- step policy (per-object time step, Sec. 4.3) ---------------------- */
int64_t or_step_ticks(const double *el, int kind, int64_t fixed_ticks,
                      double frac, const double *band_edges_km,
                      const double *band_fracs, int n_bands, double tick_s);

/* --- interval arithmetic (Sec. 4.5) ------------------------------------ */
void or_iv_add(const double a[2], const double b[2], double out[2]);
void or_iv_mul(const double a[2], const double b[2], double out[2]);
void or_iv_scale(double k, const double a[2], double out[2]);
void or_iv_cos(const double x[2], double out[2]);
void or_iv_sin(const double x[2], double out[2]);

/* --- interval occupancy region, Def 7/8 -------------------------------- */
/* 4D box of object el over ticks [tlo, thi]: the spatial part is FP64, then
 * rounded outward to FP32; the time part holds the ticks exactly. */
void or_box(const double *el, int mode, int64_t tlo, int64_t thi,
            double tick_s, float lo4[4], float hi4[4], double c_out[3],
            double *hw_out);
/* all boxes of a population: object i is cut into ceil((T+1)/k_i) segments
 * of k_i ticks (the last one clipped to T).  Box order: object-major,
 * segment-minor.  Returns the number of boxes written (or needed, if cap
 * is too small). */
int64_t or_boxes(const double *els, int64_t n, int64_t T, double tick_s,
                 const int64_t *k, int mode, float *lo4, float *hi4,
                 uint32_t *obj, int64_t cap);
/* the boxes of or_boxes whose segments start at a tick in [t0, t1), in the
 * same order (whole segments of the horizon [0, T]) */
int64_t or_boxes_starting(const double *els, int64_t n, int64_t T, double tick_s,
                          const int64_t *k, int mode, int64_t t0, int64_t t1, float *lo4,
                          float *hi4, uint32_t *obj, int64_t cap);

/* --- pair sets ------------------------------------------------------------ */
/* every pair of boxes of different objects that overlap, closed, on all four
 * axes, as (min obj, max obj, tick intersection).  Plain O(N^2) loop. */
int64_t or_raw_cells_bruteforce(const float *lo4, const float *hi4,
                                const uint32_t *obj, int64_t N,
                                or_cell *out, int64_t cap);
/* the same set: boxes sorted by tlo, each box tested against the boxes that
 * start inside its time span.  Only a restriction of the brute force loop. */
int64_t or_raw_cells_sweep(const float *lo4, const float *hi4,
                           const uint32_t *obj, int64_t N,
                           or_cell *out, int64_t cap);
/* the sweep's pairs whose earlier box in its order starts before t_end
 * (windows of the lower tick partition the whole set) */
int64_t or_raw_cells_sweep_before(const float *lo4, const float *hi4,
                                  const uint32_t *obj, int64_t N, int64_t t_end,
                                  or_cell *out, int64_t cap);
/* the same set restricted to pairs with at least one object in `sel`
 * (sel[obj] != 0), for spot checks on large populations. */
int64_t or_raw_cells_selected(const float *lo4, const float *hi4,
                              const uint32_t *obj, int64_t N,
                              const uint8_t *sel, or_cell *out, int64_t cap);
/* sort by (i,j,tlo,thi) and merge intervals of one (i,j) that overlap or
 * touch (next.tlo <= cur.thi + 1).  In place; returns the new length. */
/* The same cell set as or_raw_cells_bruteforce, found through an AABB tree
 * built by incremental insertion under a surface-area heuristic (Sec. 3.2);
 * cells come in query order. */
int64_t or_raw_cells_tree(const float *lo4, const float *hi4, const uint32_t *obj, int64_t N,
                          or_cell *out, int64_t cap);
int64_t or_canonicalize(or_cell *cells, int64_t n);

/* --- the paper's algorithms ---------------------------------------------- */
/* Alg 1: every witness (i<j, t) with ||pos_i(t) - pos_j(t)||_inf <= r_i+r_j
 * for t = 0..T, in (t, i, j) order. */
int64_t or_alg1_witnesses(const double *els, int64_t n, int64_t T,
                          double tick_s, or_witness *out, int64_t cap);
/* Alg 1 on ticks t0..t1 with pairs restricted by an x sweep (same witness
 * set as or_alg1_witnesses on that range); dist[k] = Euclidean distance of
 * witness k's centres.  Returns the witness count (only cap are written). */
int64_t or_alg1_sweep(const double *els, int64_t n, int64_t t0, int64_t t1, double tick_s,
                      or_witness *out, double *dist, int64_t cap);
/* Narrow phase over m candidates (i < j < n, 0 <= tlo <= thi): every tick
 * of each interval tested as in Alg 1.  first[q] = first witness tick or -1,
 * count[q] = witness ticks, margin[q] = min |d_inf - (r_i + r_j)| over the
 * ticks; witnesses (candidate order, ticks ascending) go to out (cap
 * entries, out may be NULL).  Returns the witness count, -1 on a bad
 * candidate. */
int64_t or_narrow_phase(const double *els, int64_t n, const or_cell *cand, int64_t m,
                        double tick_s, int32_t *first, uint32_t *count, double *margin,
                        or_witness *out, int64_t cap);
/* Alg 3 with Algs 4-6: the serial 4D search.  Returns 1 and the first
 * witness, 0 for None, or a negative code if a loop invariant (Sec. 7.2)
 * failed: -1 invariant 1, -2 invariant 2 (needs t_first, the earliest Alg 1
 * witness tick, or -1 if none), -3 iteration guard. */
int or_alg3(const double *els, int64_t n, int64_t T, double tick_s, int mode,
            int64_t t_first, uint32_t *wi, uint32_t *wj, int64_t *wt,
            int64_t *iterations);

/* --- adaptive refinement (Alg 5-6 in rounds; Sec. 4.6) ------------------- */
/* one span of the continuous-time variant: objects i < j may meet at some
 * real time in [t0, t1] seconds */
typedef struct { uint32_t i, j; double t0, t1; } or_span;
/* Rounds over all objects' intervals: a box that meets no other object's
 * box is done, one that meets another is halved (ticks [t0, mid],
 * [mid+1, t1]); two single-tick boxes that meet are a tick candidate.  The
 * first round holds object i's ticks cut into intervals of L_i ticks from
 * tick 0 (the last one clipped at T), L_i the largest power of two not
 * above max(1, floor(P_i / (f tick_s))) for the start fraction f > 0 (P_i
 * the period, or_period), or [0, T] when L_i > T or f = 0: a bounded first
 * interval, as Alg 5's intervals start at one step and grow up to a bound.
 * Returns the witnesses among the tick
 * candidates (Alg 1's test at the tick), in Alg 1's order (t, i, j);
 * round_boxes[r] = active intervals of round r (up to 64 rounds), *rounds
 * the rounds taken, *n_tick_candidates the distinct tick candidates. */
int64_t or_refine_discrete(const double *els, int64_t n, int64_t T, double tick_s, int mode,
                           double start_fraction, or_witness *out, int64_t cap,
                           int64_t *round_boxes, int *rounds, int64_t *n_tick_candidates);
/* the first-interval length L_i for the start fraction f, in ticks */
int64_t or_refine_start_ticks(const double *el, int64_t T, double tick_s, double fraction);
/* The continuous-time variant (Sec. 4.6): closed real intervals halved
 * down to length <= eps_s, halves sharing their endpoint; every meeting
 * pair of boxes at that level as (i < j, intersection of the intervals),
 * sorted, each once.  Returns the span count (only cap written). */
/* one refinement round on given boxes: the next round's intervals by the
 * discrete (cont = 0) or continuous (cont = 1) halving rule */
int64_t or_refine_round(const float *lo4, const float *hi4, const uint32_t *obj, int64_t m,
                        int cont, uint32_t *nobj, int32_t *nt0, int32_t *nt1, int64_t cap);
int64_t or_refine_continuous(const double *els, int64_t n, double T_s, double eps_s, int mode,
                             or_span *out, int64_t cap, int64_t *round_boxes, int *rounds);

/* --- static decomposition (Sec. 5, Sec. 6.1) ----------------------------- */
/* padded radial range [a(1-e) - sqrt(3) r, a(1+e) + sqrt(3) r] */
void or_radial_range(const double *el, double out[2]);
/* band edges e_1..e_{p-1} from the sorted semi-major axes */
void or_band_edges(const double *els, int64_t n, int p, double *edges);
/* object counts per band (an object sits in every band its range meets) */
void or_band_counts(const double *els, int64_t n, int p, int64_t *counts);

#ifdef __cplusplus
}
#endif
#endif
