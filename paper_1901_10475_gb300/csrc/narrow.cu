// narrow.cu -- the narrow phase: the collision witnesses (Def 4) inside a
// screen's candidate list, and the earliest of them, which is the answer of
// the discrete-time n-to-n problem (Def 5, Def 6) in Alg 1's order.
//
// For a candidate (i < j, [tlo, thi]) a tick t is a witness iff the two
// centres are within R = r_i + r_j in the infinity norm (Defs 2-3, the test
// of Alg 1), with positions from the Sec. 6.1 propagation in FP64.
//
// Two tiers decide a tick.  An FP32 evaluation (FP32 Kepler solve, FP32
// position and velocity) comes with a bound on its position error, from the
// residual of Kepler's equation at the FP32 solution: with f(E) = E - e sin E
// - M and f' >= 1 - e, the solution is within (|f| + rounding) / (1 - e) of
// the true eccentric anomaly, and the position A (cos E - e) + B sin E moves
// by at most |A| + |B| <= 2a per radian of E (taken four times over, plus
// the FP32 rounding of the position).  When the FP32 distance is farther
// from R than the two objects' bounds, that decides the tick; only ticks in
// the thin shell between go to the FP64 evaluation, which decides exactly as
// Alg 1 does.
//
// Ticks are visited in increasing order; a tick may be skipped only when no
// witness can lie there, by a bound on how fast the infinity-norm distance d
// can shrink.  From tick t, s seconds later
//   d(t + s) >= d(t) - min(V s, w s + A s^2 / 2),
// where V = vmax_i + vmax_j (perigee speeds: the largest speed on each
// orbit, vis-viva), w bounds |v_i(t) - v_j(t)|_inf (FP32 velocity plus its
// error bound) and A = mu / rp_i^2 + mu / rp_j^2 bounds the relative
// acceleration (gravity is largest at perigee rp).  While that lower bound
// stays above R, the ticks are skipped.  So the witness count and first
// witness of each candidate are those of testing every tick in FP64.
#include <math.h>

#include <algorithm>

#include "kepler.cuh"
#include "scd_internal.cuh"

namespace scd {

constexpr int kNpThreads = 256, kNpBlocksPerSm = 3;
// margin of the FP64 skip bound [km] (the FP64 propagation is good to
// 1e-7 km)
constexpr double kNpMarginKm = 1e-5;
// slack of the FP32 tier's decisions beyond the two position bounds [km],
// plus this fraction of R (FP32 rounding of R and of the distance)
constexpr float kNpSlackKm = 1e-4f, kNpSlackRel = 1e-6f;
// the skip length is computed in FP32 and shortened by this factor, far
// more than the rounding of the few FP32 operations it takes
constexpr float kNpSkipShrink = 1.0f - 1e-4f;
// rounding allowance added to the Kepler residual [rad]: FP32 rounding of
// M, of e and of the residual's own terms (sinf within 2 ulp), together
// below 2e-6 rad for |E|, |M| < 2 pi
constexpr float kNpResidualSlack = 3.5e-6f;

// narrow-phase state words (device): earliest witness as t << 32 | candidate,
// next candidate to claim, error bits, tick evaluations, FP64 evaluations
enum { NP_EARLIEST = 0, NP_NEXT = 1, NP_ERR = 2, NP_EVALS = 3, NP_EVALS64 = 4, NP_WORDS = 5 };
enum : unsigned long long { NP_ERR_PAIR = 1, NP_ERR_KEPLER = 2 };

// Per-object FP32 constants of the narrow phase (80 bytes, five 16-byte
// loads): perifocal axes, mean motion, eccentricity, the mean anomaly at
// t = 0 and per tick as unevaluated float pairs (hi + lo, 48 significant
// bits), the coefficients of the FP32 error bounds and the bounds of the
// skip rule.
struct __align__(16) NpObj {
  float A[3], n;                 // n: mean motion [rad/s]
  float B[3], e;
  float M0hi, M0lo, nthi, ntlo;  // M0 reduced to [-pi, pi]; n * tick_s [rad]
  float errA;   // position bound per radian of residual: 8 a / (1 - e) [km]
  float errB;   // FP32 rounding of the position: 4e-6 a + 1e-3 [km]
  float vErrA;  // velocity bound per radian of residual: 8 a n / (1 - e)^3 [km/s]
  float vErrB;  // FP32 rounding of the velocity: 1e-5 vmax + 1e-6 [km/s]
  float vmax;   // perigee speed x 1.001 [km/s]
  float acc;    // mu / rp^2 x 1.001 [km/s^2]
  float r;      // radius [km]
  float pad;
};
static_assert(sizeof(NpObj) == 80, "five 16-byte loads per object");

struct NarrowArgs {
  const ObjParams *par;
  const NpObj *obj;
  const scd_pair *pairs;
  int64_t m;  // candidates
  int64_t n;  // objects
  int64_t T;  // last tick a candidate may name
  double tick_s;
  float inv_tick;
  int32_t *first;   // per candidate, may be null
  uint32_t *count;  // per candidate, may be null
  unsigned long long *state;
};

// The velocity bound: v = (B cos E - A sin E) n / (1 - e cos E) changes by
// at most 2 a n / (1 - e)^2 per radian of E, and the FP32 solution's E is
// within (residual) / (1 - e) of the true one; four times over.
__global__ void k_np_objects(const ObjParams *__restrict__ par, int64_t n, double tick_s,
                             NpObj *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ObjParams p = par[i];
  const double a = sqrt(p.A[0] * p.A[0] + p.A[1] * p.A[1] + p.A[2] * p.A[2]);  // |A| = a
  const double om = 1.0 - p.e, rp = a * om;
  NpObj o;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    o.A[k] = (float)p.A[k];
    o.B[k] = (float)p.B[k];
  }
  o.n = (float)p.n;
  o.e = (float)p.e;
  const double M0 = reduce_2pi(p.M0), nt = p.n * tick_s;
  o.M0hi = (float)M0;
  o.M0lo = (float)(M0 - (double)o.M0hi);
  o.nthi = (float)nt;
  o.ntlo = (float)(nt - (double)o.nthi);
  o.errA = (float)(8.0 * a / om);
  o.errB = (float)(4e-6 * a + 1e-3);
  o.vErrA = (float)(8.0 * a * p.n / (om * om * om));
  o.vErrB = (float)(1e-5 * p.vmax + 1e-6);
  o.vmax = (float)(p.vmax * 1.001);
  o.acc = (float)(kMu / (rp * rp) * 1.001);
  o.r = (float)p.r;
  o.pad = 0.f;
  out[i] = o;
}

// the per-tick part of an object's constants (its first four 16-byte words)
struct NpTick {
  float4 a, b, m, err;
};

__device__ __forceinline__ NpTick load_tick(const NpObj *p) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
  return {__ldg(q), __ldg(q + 1), __ldg(q + 2), __ldg(q + 3)};
}

// 2 pi as a float pair, and 1 / (2 pi)
constexpr float kTwoPiHiF = (float)kTwoPi;
constexpr float kTwoPiLoF = (float)(kTwoPi - (double)(float)kTwoPi);
constexpr float kInvTwoPiF = (float)(1.0 / kTwoPi);

// Mean anomaly M0 + n t tick_s at tick t (< 2^24, exact in FP32), reduced
// by whole turns, in FP32 arithmetic only: the product and the sum are split
// exactly (an FMA gives the product's rounding error, Knuth's two-sum the
// sum's), the turns are taken off the high part exactly (the result is a
// multiple of the high part's last place and below 2^24 of them), and the
// low parts are added last.  Within 1.3e-7 rad of the exact value while
// |n t tick_s| < 2^14 rad.  The explicitly rounded intrinsics keep the
// compiler from fusing the splits.
__device__ __forceinline__ float mean_anomaly32(const float4 m, float tf) {
  const float p = __fmul_rn(m.z, tf);
  const float pe = fmaf(m.z, tf, -p);  // exact: m.z tf - p
  const float s = __fadd_rn(m.x, p);
  const float bb = __fsub_rn(s, m.x);
  const float se = __fadd_rn(__fsub_rn(m.x, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float lo = __fadd_rn(__fadd_rn(se, pe), fmaf(m.w, tf, m.y));
  const float k = rintf(s * kInvTwoPiF);
  const float rh = fmaf(-k, kTwoPiHiF, s);  // exact
  return __fadd_rn(rh, fmaf(-k, kTwoPiLoF, lo));
}

// FP32 position [km] and velocity [km/s] at tick t with bounds of their
// errors.  The Newton steps start as the FP32 stage of kepler_E_sc and use
// the fast hardware sine, cosine and division: their accuracy does not
// matter, because the bounds come from the residual of Kepler's equation at
// the final E, evaluated with the accurate sincosf (within 2 ulp).
__device__ __forceinline__ void pv32(const NpTick &o, float tf, float x[3], float v[3],
                                     float &perr, float &verr) {
  const float Mf = mean_anomaly32(o.m, tf), ef = o.b.w;
  float E = (ef <= 0.5f) ? Mf + ef * sinf(Mf)
                         : Mf + 0.85f * ef * (sinf(Mf) >= 0.f ? 1.f : -1.f);
  for (int it = 0; it < kFp32Steps; ++it) {
    const float d = __fdividef(E - ef * __sinf(E) - Mf, 1.0f - ef * __cosf(E));
    E -= d;
    if (fabsf(d) <= 1e-6f) break;
  }
  float s, c;
  sincosf(E, &s, &c);
  const float r = fabsf(E - ef * s - Mf) + kNpResidualSlack;
  perr = fmaf(o.err.x, r, o.err.y);
  verr = fmaf(o.err.z, r, o.err.w);
  const float ce = c - ef;
  const float edot = o.a.w / (1.0f - ef * c);
  const float A[3] = {o.a.x, o.a.y, o.a.z}, B[3] = {o.b.x, o.b.y, o.b.z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    x[k] = fmaf(A[k], ce, B[k] * s);
    v[k] = (B[k] * c - A[k] * s) * edot;
  }
}

// one lane's candidate
struct NpLane {
  int64_t q = -1;
  int32_t t = 0, thi = 0;  // ticks (T < 2^24)
  uint32_t oi = 0, oj = 0, cnt = 0;
  int32_t f = -1;
  float Rf = 0.f, slack = 0.f, V = 0.f, Acc = 0.f;  // r_i + r_j [km], decision slack, skip bounds
};

// One tick of a lane's candidate: the FP32 tier, the FP64 tier in the shell
// around R, then the next tick that can hold a witness; at the end of the
// interval the results are written and the lane goes idle (q = -1).
__device__ __forceinline__ void np_tick(const NarrowArgs &a, NpLane &L,
                                        unsigned long long &evals, unsigned long long &evals64,
                                        unsigned long long &err) {
  const NpTick oi = load_tick(a.obj + L.oi), oj = load_tick(a.obj + L.oj);
  const float tf = (float)L.t;
  float xi[3], xj[3], vi[3], vj[3], ei, ej, wi, wj;
  pv32(oi, tf, xi, vi, ei, wi);
  pv32(oj, tf, xj, vj, ej, wj);
  ++evals;
  float d32 = 0.f, w = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d32 = fmaxf(d32, fabsf(xi[k] - xj[k]));
    w = fmaxf(w, fabsf(vi[k] - vj[k]));
  }
  const float band = ei + ej + L.slack;  // the FP64 distance lies within d32 +- band
  bool hit;
  float D = 0.f;  // a lower bound of d - R over this tick, when positive
  if (d32 - L.Rf > band) {
    hit = false;
    D = d32 - L.Rf - band;
  } else if (d32 - L.Rf < -band) {
    hit = true;
  } else {  // the shell around R: decide in FP64 as Alg 1 does
    const ObjParams &pi = a.par[L.oi], &pj = a.par[L.oj];
    const double ts = (double)L.t * a.tick_s, R = pi.r + pj.r;
    double X[3], Y[3];
    int it_i = 0, it_j = 0;
    position_at(pi, ts, X, it_i);
    position_at(pj, ts, Y, it_j);
    if (it_i >= kKeplerMaxIter || it_j >= kKeplerMaxIter) err |= NP_ERR_KEPLER;
    ++evals64;
    double d = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) d = fmax(d, fabs(X[k] - Y[k]));
    hit = d <= R;
    if (!hit) D = (float)(d - R - kNpMarginKm);
  }
  int32_t next = L.t + 1;
  if (hit) {  // a witness at tick t
    if (L.f < 0) L.f = L.t;
    ++L.cnt;
  } else if (D > 0.f) {
    // the largest s with min(V s, w s + Acc s^2 / 2) < D, in whole ticks
    const float wm = w + wi + wj + 1e-5f;
    const float s1 = D / L.V;
    const float s2 = 2.f * D / (wm + sqrtf(wm * wm + 2.f * L.Acc * D));
    const float ks = floorf(fmaxf(s1, s2) * a.inv_tick * kNpSkipShrink);
    if (ks >= 1.f) next = L.t + 1 + (int32_t)fminf(ks, (float)(L.thi - L.t));
  }
  L.t = next;
  if (L.t > L.thi) {
    if (a.first) a.first[L.q] = L.f;
    if (a.count) a.count[L.q] = L.cnt;
    if (L.f >= 0)
      atomicMin(&a.state[NP_EARLIEST],
                ((unsigned long long)L.f << 32) | (unsigned long long)L.q);
    L.q = -1;
  }
}

// Persistent: every lane holds one candidate and walks its ticks; lanes that
// finish claim the next candidates (one atomic per warp and refill), so
// consecutive lanes share object i and its constants stay in L1.  Claims run
// from the end of the list: candidates of the highest object indices, which
// in catalog order are the eccentric and geosynchronous orbits with the
// longest intervals, start first instead of forming a tail.
__global__ void __launch_bounds__(kNpThreads, kNpBlocksPerSm) k_narrow(NarrowArgs a) {
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  NpLane L;
  bool drained = false;
  unsigned long long evals = 0, evals64 = 0, err = 0;
  for (;;) {
    const unsigned idle = __ballot_sync(kFull, L.q < 0);
    if (idle && !drained) {
      const int leader = __ffs(idle) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(&a.state[NP_NEXT], (unsigned long long)__popc(idle));
      base = __shfl_sync(kFull, base, leader);
      if (base + (unsigned long long)__popc(idle) >= (unsigned long long)a.m) drained = true;
      if (L.q < 0) {
        const unsigned long long mine =
            base + (unsigned long long)__popc(idle & ((1u << lane) - 1u));
        if (mine < (unsigned long long)a.m) {
          const int64_t qq = a.m - 1 - (int64_t)mine;
          const scd_pair c = a.pairs[qq];
          if ((int64_t)c.i >= a.n || (int64_t)c.j >= a.n || c.tlo < 0 || c.tlo > c.thi ||
              (int64_t)c.thi > a.T) {
            err |= NP_ERR_PAIR;
            if (a.first) a.first[qq] = -1;
            if (a.count) a.count[qq] = 0;
          } else {
            L.q = qq;
            L.oi = c.i;
            L.oj = c.j;
            L.t = c.tlo;
            L.thi = c.thi;
            L.f = -1;
            L.cnt = 0;
            const float4 si = __ldg(reinterpret_cast<const float4 *>(a.obj + c.i) + 4);
            const float4 sj = __ldg(reinterpret_cast<const float4 *>(a.obj + c.j) + 4);
            L.V = si.x + sj.x;
            L.Acc = si.y + sj.y;
            L.Rf = si.z + sj.z;
            L.slack = kNpSlackKm + kNpSlackRel * L.Rf;
          }
        }
      }
    }
    if (__ballot_sync(kFull, L.q >= 0) == 0) {
      if (drained) break;
      continue;  // uniform: every lane of the warp is idle
    }
    if (L.q >= 0) np_tick(a, L, evals, evals64, err);
  }
  // per-warp totals
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    evals += __shfl_xor_sync(kFull, evals, o);
    evals64 += __shfl_xor_sync(kFull, evals64, o);
    err |= __shfl_xor_sync(kFull, err, o);
  }
  if (lane == 0) {
    if (evals) atomicAdd(&a.state[NP_EVALS], evals);
    if (evals64) atomicAdd(&a.state[NP_EVALS64], evals64);
    if (err) atomicOr(&a.state[NP_ERR], err);
  }
}

__global__ void k_narrow_init(unsigned long long *state) {
  if (threadIdx.x == 0) {
    state[NP_EARLIEST] = ~0ull;
    state[NP_NEXT] = 0;
    state[NP_ERR] = 0;
    state[NP_EVALS] = 0;
    state[NP_EVALS64] = 0;
  }
}

}  // namespace scd

using namespace scd;

extern "C" SCD_API int scd_narrow_phase(scd_scene *s, const scd_pair *d_pairs, int64_t n_pairs,
                                        int32_t *d_first, uint32_t *d_count,
                                        scd_witness *earliest) {
  if (!s || n_pairs < 0 || (n_pairs > 0 && !d_pairs)) return SCD_ERR_INVALID_ARG;
  if (!s->boxes_built) return SCD_ERR_STATE;
  if (n_pairs > (int64_t)0xffffffffll) return SCD_ERR_CAPACITY;
  if (!s->d_narrow.ensure(NP_WORDS, s->stream)) return SCD_ERR_OOM;
  if (!s->d_npobj.ensure((size_t)s->n * sizeof(NpObj), s->stream)) return SCD_ERR_OOM;
  NpObj *obj = reinterpret_cast<NpObj *>(s->d_npobj.p);
  k_narrow_init<<<1, 32, 0, s->stream>>>(s->d_narrow.p);
  note_launch();
  if (n_pairs > 0) {
    k_np_objects<<<(unsigned)((s->n + 255) / 256), 256, 0, s->stream>>>(s->d_par.p, s->n,
                                                                         s->tick_s, obj);
    note_launch();
    static int per_sm = 0, sms = 0;
    if (!per_sm) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_narrow, kNpThreads, 0);
    if (!sms) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    int64_t blocks = (int64_t)std::max(sms, 1) * std::max(per_sm, 1);
    const int64_t need = (n_pairs + kNpThreads - 1) / kNpThreads;
    if (need < blocks) blocks = need;
    NarrowArgs a;
    a.par = s->d_par.p;
    a.obj = obj;
    a.pairs = d_pairs;
    a.m = n_pairs;
    a.n = s->n;
    a.T = s->T;
    a.tick_s = s->tick_s;
    a.inv_tick = (float)(1.0 / s->tick_s);
    a.first = d_first;
    a.count = d_count;
    a.state = s->d_narrow.p;
    k_narrow<<<(unsigned)blocks, kNpThreads, 0, s->stream>>>(a);
    note_launch();
  }
  if (cudaGetLastError() != cudaSuccess) return SCD_ERR_CUDA;
  unsigned long long h[NP_WORDS];
  if (cudaMemcpyAsync(h, s->d_narrow.p, sizeof(h), cudaMemcpyDeviceToHost, s->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return SCD_ERR_CUDA;
  s->last_np_evals = h[NP_EVALS];
  s->last_np_evals64 = h[NP_EVALS64];
  if (h[NP_ERR] & NP_ERR_PAIR) return SCD_ERR_INVALID_ARG;
  if (h[NP_ERR] & NP_ERR_KEPLER) return SCD_ERR_KEPLER_NOCONV;
  if (earliest) {
    earliest->i = 0;
    earliest->j = 0;
    earliest->t = -1;
    if (h[NP_EARLIEST] != ~0ull) {
      scd_pair p;
      const int64_t q = (int64_t)(h[NP_EARLIEST] & 0xffffffffull);
      if (cudaMemcpyAsync(&p, d_pairs + q, sizeof(p), cudaMemcpyDeviceToHost, s->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(s->stream) != cudaSuccess)
        return SCD_ERR_CUDA;
      earliest->i = p.i;
      earliest->j = p.j;
      earliest->t = (int32_t)(h[NP_EARLIEST] >> 32);
    }
  }
  return SCD_OK;
}
