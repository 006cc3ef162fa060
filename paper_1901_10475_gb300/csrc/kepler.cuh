// kepler.cuh -- the FP64 two-body propagation of Sec. 6.1 (Eq. 1 solved
// through Kepler's equation) shared by the box build, the stand-alone
// propagation and the narrow phase, so that all three evaluate the same
// positions.
#pragma once

#include <math.h>

#include "scd_internal.cuh"

namespace scd {

// ---------------------------------------------------------------------------
// FP64 sine and cosine of the eccentric anomaly by table and Taylor series.
// x = k (2 pi / 256) + r with |r| <= pi / 256; sin x and cos x from the
// table's sin and cos of k (2 pi / 256) and the Taylor series of sin r (to
// r^5) and cos r (to r^6), whose truncation errors are below 1e-17 and
// 1e-20.  The table is built at compile time: each entry by the Taylor
// series of its angle within a quarter turn (16 terms), then turned by whole
// quarters.  Checked on the host against long-double sinl / cosl (the same
// operations, k picked in FP32): table entries within 2.6e-16, sin and cos
// over [-4, 4] within 3.7e-16.  The argument reduction
// takes 2 pi as a double-double (its double and the remainder 2.449e-16),
// each product subtracted with one rounding (fma).  One table load and a
// dozen FP64 multiply-adds, in place of a general sincos, in the Kepler
// solve's FP64 steps (once per box).
// ---------------------------------------------------------------------------
constexpr int kSinTab = 256;
struct SinCosTab {
  double v[2 * kSinTab];  // sin, cos of k (2 pi / 256)
};
constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int n = 1; n < 16; ++n) {
    t *= -x * x / (double)((2 * n) * (2 * n + 1));
    s += t;
  }
  return s;
}
constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int n = 1; n < 16; ++n) {
    t *= -x * x / (double)((2 * n - 1) * (2 * n));
    s += t;
  }
  return s;
}
constexpr SinCosTab make_sincos_tab() {
  SinCosTab t{};
  for (int k = 0; k < kSinTab; ++k) {
    const int q = k / (kSinTab / 4), m = k % (kSinTab / 4);
    const double th = (double)m * (kTwoPi / kSinTab);
    const double s = taylor_sin(th), c = taylor_cos(th);
    double S = s, C = c;
    if (q == 1) { S = c; C = -s; }
    if (q == 2) { S = -s; C = -c; }
    if (q == 3) { S = -c; C = s; }
    t.v[2 * k] = S;
    t.v[2 * k + 1] = C;
  }
  return t;
}
static __device__ const SinCosTab g_sincos_tab = make_sincos_tab();

// xf: x in FP32 (or any float within a few ulp of it), from which the table
// step k is picked in FP32: near a half step the two roundings may pick
// neighbouring k, either of which leaves |r| within half a step and a hair
__device__ __forceinline__ void sincos_tab(double x, float xf, double &s, double &c) {
  constexpr double kStepHi = kTwoPi / kSinTab;                 // exact: a power-of-2 division
  constexpr double kStepLo = 2.4492935982947064e-16 / kSinTab;  // 2 pi - fl(2 pi), divided
  const float kf = rintf(xf * (float)(kSinTab / kTwoPi));
  const double k = (double)kf;
  double r = fma(-k, kStepHi, x);
  r = fma(-k, kStepLo, r);
  const int idx = ((int)kf) & (kSinTab - 1);
  const double sk = __ldg(&g_sincos_tab.v[2 * idx]), ck = __ldg(&g_sincos_tab.v[2 * idx + 1]);
  const double r2 = r * r;
  // |r| <= pi / 256 (and a hair): the first omitted terms, r^7 / 7! and
  // r^8 / 8!, are below 1e-17 and 1e-20
  const double sr = r * fma(r2, fma(r2, 1.0 / 120.0, -1.0 / 6.0), 1.0);
  const double cr = fma(r2, fma(r2, fma(r2, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
  s = fma(sk, cr, ck * sr);
  c = fma(ck, cr, -(sk * sr));
}

// The Newton correction d = (E - e sin E - M) / (1 - e cos E): the residual
// in FP64 (it cancels), the quotient in FP32 (d is a correction of at most
// 1e-5 rad, so its relative error of 1e-7 leaves E within 1e-12 rad)
__device__ __forceinline__ float newton_step(double Ed, double s, double c, double M, double e) {
  const double f = fma(-e, s, Ed - M);
  const double fp = fma(-e, c, 1.0);
  return (float)f / (float)fp;
}

// ---------------------------------------------------------------------------
// Kepler's equation E - e sin E = M by Newton's method.  The start is
// M + e sin M for moderate e and Danby's M + 0.85 e sign(sin M) above
// e = 0.5; both converge for the e < 1 of closed orbits.
// ---------------------------------------------------------------------------
constexpr int kKeplerMaxIter = 40;

__device__ __forceinline__ double reduce_2pi(double M) {
  double k = rint(M * (1.0 / kTwoPi));
  return fma(-k, kTwoPi, M);
}

// Kepler's equation, mixed precision: Newton in FP32 to about 3e-7 rad (at
// most 12 steps: by perigee at e near 1 the FP32 residual cancels and stalls
// near 1e-5 rad), then FP64 Newton steps.  Each FP64 step squares the error
// (times |f''/2f'| = e|sin E| / 2(1 - e cos E), at most e / 2(1 - e): 1.5 for
// e <= 0.75), so one step usually suffices: below 2e-13 rad, i.e. below
// 1e-8 km of position at GEO distance.  Steps continue while that bound on
// the error left exceeds a quarter of the object's tolerance (1e-7 km / a),
// i.e. while the last correction's square exceeds the object's dmax2, or the
// correction exceeds 1e-5 rad; both compared in FP32 (the test needs no FP64
// arithmetic); after kFp64Steps without that, iters reports non-convergence.
// Returns E with sin E and cos E, corrected to second order in the last step
// (third-order error below 2e-16), so the caller needs no further sincos.
constexpr int kFp32Steps = 12, kFp64Steps = 8;

// The rare further FP64 steps: take the pending correction d, then step until
// the test passes; on return (Ed, s, c, d) describe the last step.
__device__ __forceinline__ bool newton_more(float d, float dmax2) {
  return d * d > dmax2 || fabsf(d) > 1e-5f;
}

static __device__ __noinline__ void kepler_more_fp64(double M, double e, float dmax2, double &Ed,
                                                     double &s, double &c, float &d,
                                                     int &iters) {
  for (int step = 1; step < kFp64Steps; ++step) {
    Ed -= (double)d;
    sincos_tab(Ed, (float)Ed, s, c);
    d = newton_step(Ed, s, c, M, e);
    iters += 1;
    if (!newton_more(d, dmax2)) return;
  }
  iters = kKeplerMaxIter;  // no convergence
}

// ef: e in FP32 (precomputed per object)
__device__ __forceinline__ double kepler_E_sc(double M, double e, float ef, float dmax2,
                                              double &sE, double &cE, int &iters) {
  const float Mf = (float)M;
  if (e == 0.0) {
    sincos_tab(M, Mf, sE, cE);
    iters = 0;
    return M;
  }
  float E = (ef <= 0.5f) ? Mf + ef * sinf(Mf)
                         : Mf + 0.85f * ef * (sinf(Mf) >= 0.f ? 1.f : -1.f);
  int it = 0;
  for (; it < kFp32Steps; ++it) {
    float s, c;
    sincosf(E, &s, &c);
    float d = (E - ef * s - Mf) / (1.0f - ef * c);
    E -= d;
    if (fabsf(d) <= 1e-6f) break;
  }
  double Ed = (double)E, s, c;
  sincos_tab(Ed, E, s, c);
  float df = newton_step(Ed, s, c, M, e);
  iters = it + 1;
  if (newton_more(df, dmax2)) kepler_more_fp64(M, e, dmax2, Ed, s, c, df, iters);
  // sin(E - d), cos(E - d) to second order in d
  const double d = (double)df;
  const double h = 0.5 * d * d;
  sE = s - d * c - h * s;
  cE = c + d * s - h * c;
  return Ed - d;
}

// position at time t [s] from the per-object constants
__device__ __forceinline__ void position_at(const ObjParams &p, double t, double out[3],
                                            int &iters) {
  double M = reduce_2pi(p.M0 + p.n * t);
  double s, c;
  kepler_E_sc(M, p.e, p.ef, p.dmax2, s, c, iters);
  double ce = c - p.e;
#pragma unroll
  for (int k = 0; k < 3; ++k) out[k] = fma(p.A[k], ce, p.B[k] * s);
}

// exact ranges of cos and sin over [x0, x1] (x1 >= x0) from the end values
// c0 = cos x0, c1 = cos x1, s0 = sin x0, s1 = sin x1: each widened to its
// extremum wherever a multiple m of a quarter turn lies inside (m = 0 mod 4:
// cos = 1, 1: sin = 1, 2: cos = -1, 3: sin = -1); the whole range once the
// interval spans a full turn.  The multiples inside are the integers from
// ceil(x0 / (pi/2)) to floor(x1 / (pi/2)): six FP64 operations for both
// ranges, the rest integer work (the multiples are at most four).
__device__ __forceinline__ void cos_sin_range(double x0, double x1, double c0, double c1,
                                              double s0, double s1, double &clo, double &chi,
                                              double &slo, double &shi) {
  clo = fmin(c0, c1);
  chi = fmax(c0, c1);
  slo = fmin(s0, s1);
  shi = fmax(s0, s1);
  if (x1 - x0 >= kTwoPi) {
    clo = slo = -1.0;
    chi = shi = 1.0;
    return;
  }
  constexpr double kQuarter = 2.0 / kPi;
  const long long m0 = (long long)ceil(x0 * kQuarter), m1 = (long long)floor(x1 * kQuarter);
  for (long long m = m0; m <= m1; ++m) {
    switch ((int)(m & 3)) {
      case 0: chi = 1.0; break;
      case 1: shi = 1.0; break;
      case 2: clo = -1.0; break;
      default: slo = -1.0; break;
    }
  }
}

// The interval occupancy box (Def 7) of one object over the ticks [tlo, thi]
// (tick length tick_s seconds), before outward FP32 rounding:
//  SPEED     every point of the arc lies within vmax |t - tc| of pos(tc):
//            the cube of half-width r + vmax (thi - tlo) tick_s / 2 + eps
//            around the position at the midpoint tc
//  INTERVAL  interval evaluation of A (cos E - e) + B sin E over
//            [E(tlo), E(thi)] (Sec. 4.5: E is monotone in t, so its ends
//            bound it), widened by r + eps
// `iters` receives the Kepler iterations (kKeplerMaxIter: no convergence).
__device__ __forceinline__ void segment_box(const ObjParams &p, int mode, int64_t tlo, int64_t thi,
                                            double tick_s, double lo[3], double hi[3],
                                            int &iters) {
  if (mode == SCD_BOX_SPEED) {
    double tc = 0.5 * (double)(tlo + thi) * tick_s;
    double c[3];
    position_at(p, tc, c, iters);
    double hw = p.r + p.vmax * (double)(thi - tlo) * tick_s * 0.5 + kEpsKm;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      lo[q] = c[q] - hw;
      hi[q] = c[q] + hw;
    }
    return;
  }
  double M0 = p.M0 + p.n * ((double)tlo * tick_s);
  double M1 = p.M0 + p.n * ((double)thi * tick_s);
  double kk = rint(M0 * (1.0 / kTwoPi));
  double Mr0 = fma(-kk, kTwoPi, M0), Mr1 = fma(-kk, kTwoPi, M1);
  // both ends by the mixed-precision solve, which also gives sin E, cos E
  // (E within 1e-7 km / a: far inside the 1e-6 km margin)
  int i0 = 0, i1 = 0;
  double s0, c0, s1, c1;
  double E0 = kepler_E_sc(Mr0, p.e, p.ef, p.dmax2, s0, c0, i0);
  double E1 = kepler_E_sc(Mr1, p.e, p.ef, p.dmax2, s1, c1, i1);
  iters = max(i0, i1);
  double clo, chi, slo, shi;
  cos_sin_range(E0, E1, c0, c1, s0, s1, clo, chi, slo, shi);
  const double w = p.r + kEpsKm, cl = clo - p.e, ch = chi - p.e;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    // interval products by the coefficient's sign (rounding is monotone, so
    // these are the two products' minimum and maximum, bit for bit)
    const bool ap = __double_as_longlong(p.A[q]) >= 0, bp = __double_as_longlong(p.B[q]) >= 0;
    const double ulo = __dmul_rn(p.A[q], ap ? cl : ch), uhi = __dmul_rn(p.A[q], ap ? ch : cl);
    const double vlo = __dmul_rn(p.B[q], bp ? slo : shi), vhi = __dmul_rn(p.B[q], bp ? shi : slo);
    lo[q] = __dsub_rn(__dadd_rn(ulo, vlo), w);
    hi[q] = __dadd_rn(__dadd_rn(uhi, vhi), w);
  }
}

}  // namespace scd
