// narrow.cu -- the narrow phase: the collision witnesses (Def 4) inside a
// screen's candidate list, and the earliest of them, which is the answer of
// the discrete-time n-to-n problem (Def 5, Def 6) in Alg 1's order.
//
// For a candidate (i < j, [tlo, thi]) a tick t is a witness iff the two
// centres are within r_i + r_j in the infinity norm (Defs 2-3, the test of
// Alg 1), with positions from the Sec. 6.1 propagation in FP64.  Ticks are
// visited in increasing order; a tick may be skipped only when no witness
// can lie there, by a bound on how fast the infinity-norm distance d of the
// two centres can shrink.  From tick t, s seconds later
//   d(t + s) >= d(t) - min(V s, w s + A s^2 / 2),
// where V = vmax_i + vmax_j (perigee speeds: the largest speed on each
// orbit, vis-viva), w = |v_i(t) - v_j(t)|_inf and A = mu / rp_i^2 +
// mu / rp_j^2 bounds the relative acceleration (gravity is largest at
// perigee rp).  So while that lower bound stays above r_i + r_j, plus a
// margin far above the position error of the propagation, the ticks are
// skipped.  Every tick that is not skipped is decided exactly as Alg 1
// decides it, so the witness count and first witness of each candidate are
// those of testing every tick.
#include <math.h>

#include <algorithm>

#include "kepler.cuh"
#include "scd_internal.cuh"

namespace scd {

constexpr int kNpThreads = 256;
// margin of the skip bound [km] (the propagation is good to 1e-7 km), and
// speed margin [km/s] added to w (the FP32 relative velocity below is good
// to about 1e-5 km/s, and an error there grows with the skipped time)
constexpr double kNpMarginKm = 1e-5;
constexpr float kNpMarginKmS = 1e-4f;
// the skip length is computed in FP32 and shortened by this factor, far
// more than the rounding of the few FP32 operations it takes
constexpr float kNpSkipShrink = 1.0f - 1e-4f;

// narrow-phase state words (device): earliest witness as t << 32 | candidate,
// next candidate to claim, error bits, tick evaluations
enum { NP_EARLIEST = 0, NP_NEXT = 1, NP_ERR = 2, NP_EVALS = 3, NP_WORDS = 4 };
enum : unsigned long long { NP_ERR_PAIR = 1, NP_ERR_KEPLER = 2 };

struct NarrowArgs {
  const ObjParams *par;
  const scd_pair *pairs;
  int64_t m;  // candidates
  int64_t n;  // objects
  int64_t T;  // last tick a candidate may name
  double tick_s;
  int32_t *first;   // per candidate, may be null
  uint32_t *count;  // per candidate, may be null
  unsigned long long *state;
};

// Position [km] at t [s], computed exactly as position_at, and velocity
// [km/s]: d/dt of A (cos E - e) + B sin E with dE/dt = n / (1 - e cos E)
// (Kepler's equation differentiated), the reciprocal in FP32.
__device__ __forceinline__ void pos_vel(const ObjParams &p, double t, double x[3], float v[3],
                                        int &iters) {
  const double M = reduce_2pi(p.M0 + p.n * t);
  double s, c;
  kepler_E_sc(M, p.e, p.tolE, s, c, iters);
  const double ce = c - p.e;
#pragma unroll
  for (int k = 0; k < 3; ++k) x[k] = fma(p.A[k], ce, p.B[k] * s);
  const float edot = (float)p.n * __frcp_rn((float)(1.0 - p.e * c));
  const float sf = (float)s, cf = (float)c;
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = ((float)p.B[k] * cf - (float)p.A[k] * sf) * edot;
}

// largest relative acceleration bound of one object: mu / rp^2 [km/s^2]
__device__ __forceinline__ float accel_bound(const ObjParams &p) {
  const double a = sqrt(p.A[0] * p.A[0] + p.A[1] * p.A[1] + p.A[2] * p.A[2]);  // |A| = a
  const double rp = a * (1.0 - p.e);
  return (float)(kMu / (rp * rp));
}

// One tick of a lane's candidate: Alg 1's test at tick t, then the next tick
// that can hold a witness; at the end of the interval the results are
// written and the lane goes idle (q = -1).
__device__ __forceinline__ void np_tick(const NarrowArgs &a, int64_t &q, int64_t &t, int64_t thi,
                                        uint32_t oi, uint32_t oj, int32_t &f, uint32_t &cnt,
                                        double R, float V, float Acc, float inv_tick,
                                        unsigned long long &evals, unsigned long long &err) {
  double xi[3], xj[3];
  float vi[3], vj[3];
  int it_i = 0, it_j = 0;
  const double ts = (double)t * a.tick_s;
  pos_vel(a.par[oi], ts, xi, vi, it_i);
  pos_vel(a.par[oj], ts, xj, vj, it_j);
  if (it_i >= kKeplerMaxIter || it_j >= kKeplerMaxIter) err |= NP_ERR_KEPLER;
  ++evals;
  double d = 0.0;
  float w = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d = fmax(d, fabs(xi[k] - xj[k]));
    w = fmaxf(w, fabsf(vi[k] - vj[k]));
  }
  int64_t next = t + 1;
  if (d <= R) {  // a witness at tick t
    if (f < 0) f = (int32_t)t;
    ++cnt;
  } else {
    const double D = d - R - kNpMarginKm;
    if (D > 0.0) {
      // the largest s with min(V s, w s + Acc s^2 / 2) < D, in whole ticks
      const float Df = (float)D;
      const float wm = w + kNpMarginKmS;
      const float s1 = Df / V;
      const float s2 = 2.f * Df / (wm + sqrtf(wm * wm + 2.f * Acc * Df));
      const float ks = floorf(fmaxf(s1, s2) * inv_tick * kNpSkipShrink);
      if (ks >= 1.f) next = t + 1 + (int64_t)fminf(ks, (float)(thi - t));
    }
  }
  t = next;
  if (t > thi) {
    if (a.first) a.first[q] = f;
    if (a.count) a.count[q] = cnt;
    if (f >= 0)
      atomicMin(&a.state[NP_EARLIEST], ((unsigned long long)f << 32) | (unsigned long long)q);
    q = -1;
  }
}

// Persistent: every lane holds one candidate and walks its ticks; lanes that
// finish claim the next candidates in list order (one atomic per warp and
// refill), so consecutive lanes share object i and its constants stay in L1.
__global__ void __launch_bounds__(kNpThreads) k_narrow(NarrowArgs a) {
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int64_t q = -1, t = 0, thi = 0;
  uint32_t oi = 0, oj = 0, cnt = 0;
  int32_t f = -1;
  double R = 0.0;
  float V = 0.f, Acc = 0.f, inv_tick = 0.f;
  bool drained = false;
  unsigned long long evals = 0, err = 0;
  for (;;) {
    const unsigned idle = __ballot_sync(kFull, q < 0);
    if (idle && !drained) {
      const int leader = __ffs(idle) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(&a.state[NP_NEXT], (unsigned long long)__popc(idle));
      base = __shfl_sync(kFull, base, leader);
      if (base + (unsigned long long)__popc(idle) >= (unsigned long long)a.m) drained = true;
      if (q < 0) {
        const unsigned long long mine = base + (unsigned long long)__popc(idle & ((1u << lane) - 1u));
        if (mine < (unsigned long long)a.m) {
          const scd_pair c = a.pairs[mine];
          if ((int64_t)c.i >= a.n || (int64_t)c.j >= a.n || c.tlo < 0 || c.tlo > c.thi ||
              (int64_t)c.thi > a.T) {
            err |= NP_ERR_PAIR;
            if (a.first) a.first[mine] = -1;
            if (a.count) a.count[mine] = 0;
          } else {
            q = (int64_t)mine;
            oi = c.i;
            oj = c.j;
            t = c.tlo;
            thi = c.thi;
            f = -1;
            cnt = 0;
            const ObjParams &pi = a.par[oi], &pj = a.par[oj];
            R = pi.r + pj.r;
            V = (float)((pi.vmax + pj.vmax) * 1.001);
            Acc = (accel_bound(pi) + accel_bound(pj)) * 1.001f;
            inv_tick = (float)(1.0 / a.tick_s);
          }
        }
      }
    }
    if (__ballot_sync(kFull, q >= 0) == 0) {
      if (drained) break;
      continue;  // uniform: every lane of the warp is idle
    }
    if (q >= 0) np_tick(a, q, t, thi, oi, oj, f, cnt, R, V, Acc, inv_tick, evals, err);
  }
  // per-warp totals
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    evals += __shfl_xor_sync(kFull, evals, o);
    err |= __shfl_xor_sync(kFull, err, o);
  }
  if (lane == 0) {
    if (evals) atomicAdd(&a.state[NP_EVALS], evals);
    if (err) atomicOr(&a.state[NP_ERR], err);
  }
}

__global__ void k_narrow_init(unsigned long long *state) {
  if (threadIdx.x == 0) {
    state[NP_EARLIEST] = ~0ull;
    state[NP_NEXT] = 0;
    state[NP_ERR] = 0;
    state[NP_EVALS] = 0;
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
  k_narrow_init<<<1, 32, 0, s->stream>>>(s->d_narrow.p);
  note_launch();
  if (n_pairs > 0) {
    static int per_sm = 0, sms = 0;
    if (!per_sm) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_narrow, kNpThreads, 0);
    if (!sms) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    int64_t blocks = (int64_t)std::max(sms, 1) * std::max(per_sm, 1);
    const int64_t need = (n_pairs + kNpThreads - 1) / kNpThreads;
    if (need < blocks) blocks = need;
    NarrowArgs a;
    a.par = s->d_par.p;
    a.pairs = d_pairs;
    a.m = n_pairs;
    a.n = s->n;
    a.T = s->T;
    a.tick_s = s->tick_s;
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
