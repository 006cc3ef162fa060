// refine.cu -- adaptive refinement: the interval growing and halving of
// Alg 5 and Alg 6 as data-parallel rounds over all objects at once.
//
// Every object starts with the whole horizon [0, T] as its interval.  A round
// builds the 4D box of every active interval (Def 8), finds the boxes that
// meet a box of another object, and then
//   - drops an interval whose box meets none: its object is proven free of
//     collisions over it (every other object's position at those times lies
//     in one of this round's boxes, or was proven free in an earlier round);
//   - halves an interval whose box meets another, into ticks [t0, mid] and
//     [mid + 1, t1] (t_min of the second half = t_max of the first + one
//     tick, as Alg 5 advances), as Alg 6 halves an interval that meets;
//   - keeps a single tick whose box still meets a longer interval, until
//     that one is halved;
//   - collects every pair of single-tick boxes that meet (the same tick) as
//     a tick candidate.
// The narrow phase then decides each tick candidate with Alg 1's test, so
// the result is exactly the set of collision witnesses (Def 4).
//
// The continuous-time variant (Sec. 4.6) runs the same rounds over closed
// real intervals: the interval [k, k + 1] of a level, in units of
// T / 2^level seconds, is halved into [2k, 2k + 1] and [2k + 1, 2k + 2] of
// the next level (the halves share their endpoint), down to a length of at
// most eps; every pair of meeting boxes at that level is reported as a span,
// the intersection of the two intervals.  The box, sort and sweep kernels
// serve both: with t0 = k, t1 = k + 1 and the level's unit as the tick, the
// SPEED box covers the real interval.
//
// Boxes are SPEED boxes (position at the interval's midpoint, half-width
// r + vmax span / 2, rounded outward to FP32), the screen's formula.  The
// meeting boxes of a round are found by sorting the boxes on their lower x
// face and sweeping: box a is tested against the boxes after it in that
// order whose lower x face is at most a's upper x face.  The sweep suits
// rounds of up to some 1e5 boxes; larger populations want the screen's
// hierarchy.
#include <math.h>

#include <algorithm>

#include "kepler.cuh"
#include "scd_internal.cuh"

namespace scd {

constexpr int kRfThreads = 256;
constexpr int kRfMaxRounds = 64;
// object indices take 20 bits and ticks 24 in a packed candidate key
constexpr int64_t kRfMaxObjects = 1ll << 20;
// device state words: tick candidates, next intervals, error bits, unique
// candidates, witnesses
enum { RF_NCAND = 0, RF_NNEXT = 1, RF_ERR = 2, RF_NUNIQ = 3, RF_NWIT = 4, RF_WORDS = 5 };
constexpr uint32_t RF_HIT = 1u, RF_HIT_LONG = 2u;  // per-interval flags of a round

// packed tick candidate: t (24 bits) | i (20) | j (20): sorts in Alg 1's order
__host__ __device__ inline unsigned long long rf_key(uint32_t t, uint32_t i, uint32_t j) {
  return ((unsigned long long)t << 40) | ((unsigned long long)i << 20) | (unsigned long long)j;
}

// order-preserving map of a float to an unsigned key
__device__ __forceinline__ uint32_t rf_float_key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k_rf_init(int64_t n, int32_t T, uint32_t *obj, int32_t *t0, int32_t *t1) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  obj[i] = (uint32_t)i;
  t0[i] = 0;
  t1[i] = T;
}

struct RfBoxArgs {
  const ObjParams *par;
  const uint32_t *obj;
  const int32_t *t0, *t1;
  int64_t M;
  double tick_s;
  float4 *lo, *hi;
  uint32_t *key, *idx;
  unsigned long long *state;
};

__global__ void __launch_bounds__(kRfThreads) k_rf_boxes(RfBoxArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.M) return;
  const ObjParams &p = a.par[a.obj[i]];
  const int32_t t0 = a.t0[i], t1 = a.t1[i];
  // every point of the arc lies within vmax |t - tc| of pos(tc)
  const double tc = 0.5 * ((double)t0 + (double)t1) * a.tick_s;
  double c[3];
  int iters = 0;
  position_at(p, tc, c, iters);
  if (iters >= kKeplerMaxIter) atomicOr(&a.state[RF_ERR], 1ull);
  const double hw = p.r + p.vmax * (double)(t1 - t0) * a.tick_s * 0.5 + kEpsKm;
  float4 L, H;
  L.x = __double2float_rd(c[0] - hw);
  L.y = __double2float_rd(c[1] - hw);
  L.z = __double2float_rd(c[2] - hw);
  H.x = __double2float_ru(c[0] + hw);
  H.y = __double2float_ru(c[1] + hw);
  H.z = __double2float_ru(c[2] + hw);
  L.w = (float)t0;  // ticks < 2^24: exact
  H.w = (float)t1;
  a.lo[i] = L;
  a.hi[i] = H;
  a.key[i] = rf_float_key(L.x);
  a.idx[i] = (uint32_t)i;
}

struct RfSweepArgs {
  const float4 *lo, *hi;
  const uint32_t *obj;
  const int32_t *t0, *t1;
  const uint32_t *idx;  // intervals in order of their lower x face
  int64_t M;
  uint32_t *flags;
  unsigned long long *cand;
  int64_t cap;
  unsigned long long *state;
  int spans;  // continuous variant, finest level: every meeting pair is a span
};

// span key of two meeting intervals [ka, ka + 1], [kb, kb + 1] of one level:
// i (20 bits) | j (20) | the later start (22) | whether the starts agree (1);
// sorts by (i, j, t0, t1) of the intersection
__device__ __forceinline__ unsigned long long rf_span_key(uint32_t i, uint32_t j, int32_t ka,
                                                          int32_t kb) {
  const uint32_t km = (uint32_t)max(ka, kb), same = ka == kb ? 1u : 0u;
  return ((unsigned long long)i << 44) | ((unsigned long long)j << 24) |
         ((unsigned long long)km << 1) | same;
}

// One thread per interval a (in sorted order): every interval after it
// whose lower x face is at most a's upper x face meets a on x (a's lower
// face is not above its own), so only y, z and the tick range are tested.
__global__ void __launch_bounds__(kRfThreads) k_rf_sweep(RfSweepArgs a) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.M) return;
  const uint32_t ia = a.idx[s];
  const float4 la = a.lo[ia], ha = a.hi[ia];
  const uint32_t oa = a.obj[ia];
  const int32_t ta = a.t0[ia];
  const bool longa = a.t1[ia] > ta;
  uint32_t fa = 0;
  for (int64_t u = s + 1; u < a.M; ++u) {
    const uint32_t ib = a.idx[u];
    const float4 lb = a.lo[ib];
    if (!(lb.x <= ha.x)) break;  // sorted: no later box reaches a on x
    const uint32_t ob = a.obj[ib];
    if (ob == oa) continue;
    const float4 hb = a.hi[ib];
    if (!(la.y <= hb.y && lb.y <= ha.y && la.z <= hb.z && lb.z <= ha.z && la.w <= hb.w &&
          lb.w <= ha.w))
      continue;
    const bool longb = a.t1[ib] > a.t0[ib];
    fa |= RF_HIT | (longb ? RF_HIT_LONG : 0u);
    atomicOr(&a.flags[ib], RF_HIT | (longa ? RF_HIT_LONG : 0u));
    if (a.spans) {
      const unsigned long long q = atomicAdd(&a.state[RF_NCAND], 1ull);
      if (q < (unsigned long long)a.cap)
        a.cand[q] = rf_span_key(min(oa, ob), max(oa, ob), ta, a.t0[ib]);
    } else if (!longa && !longb) {  // two single ticks meet: the same tick
      const unsigned long long q = atomicAdd(&a.state[RF_NCAND], 1ull);
      if (q < (unsigned long long)a.cap)
        a.cand[q] = rf_key((uint32_t)ta, min(oa, ob), max(oa, ob));
    }
  }
  if (fa) atomicOr(&a.flags[ia], fa);
}

// next round's intervals (order is free: appended by atomics); the buffers
// hold 2 M entries, so nothing overflows
__global__ void __launch_bounds__(kRfThreads) k_rf_split(const uint32_t *__restrict__ obj,
                                                         const int32_t *__restrict__ t0,
                                                         const int32_t *__restrict__ t1,
                                                         const uint32_t *__restrict__ flags,
                                                         int64_t M, uint32_t *nobj, int32_t *nt0,
                                                         int32_t *nt1,
                                                         unsigned long long *state) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const uint32_t f = flags[i];
  if (!(f & RF_HIT)) return;  // proven free of collisions over [t0, t1]
  const int32_t a0 = t0[i], a1 = t1[i];
  if (a1 > a0) {
    const unsigned long long q = atomicAdd(&state[RF_NNEXT], 2ull);
    const int32_t mid = a0 + (a1 - a0) / 2;
    nobj[q] = obj[i];
    nt0[q] = a0;
    nt1[q] = mid;
    nobj[q + 1] = obj[i];
    nt0[q + 1] = mid + 1;
    nt1[q + 1] = a1;
  } else if (f & RF_HIT_LONG) {  // wait for the longer intervals it meets
    const unsigned long long q = atomicAdd(&state[RF_NNEXT], 1ull);
    nobj[q] = obj[i];
    nt0[q] = a0;
    nt1[q] = a1;
  }
}

// continuous variant: both halves of an interval [k, k + 1] that met, as
// [2k, 2k + 1] and [2k + 1, 2k + 2] in units of the next level
__global__ void __launch_bounds__(kRfThreads) k_rf_split_cont(const uint32_t *__restrict__ obj,
                                                              const int32_t *__restrict__ t0,
                                                              const uint32_t *__restrict__ flags,
                                                              int64_t M, uint32_t *nobj,
                                                              int32_t *nt0, int32_t *nt1,
                                                              unsigned long long *state) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M || !(flags[i] & RF_HIT)) return;
  const unsigned long long q = atomicAdd(&state[RF_NNEXT], 2ull);
  const int32_t k = t0[i];
  nobj[q] = obj[i];
  nt0[q] = 2 * k;
  nt1[q] = 2 * k + 1;
  nobj[q + 1] = obj[i];
  nt0[q + 1] = 2 * k + 1;
  nt1[q + 1] = 2 * k + 2;
}

// distinct span keys (sorted) appended to out (in any order)
__global__ void k_rf_distinct(const unsigned long long *__restrict__ key, int64_t n,
                              unsigned long long *out, unsigned long long *state) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  if (q > 0 && key[q - 1] == key[q]) return;
  out[atomicAdd(&state[RF_NUNIQ], 1ull)] = key[q];
}

__global__ void k_rf_span_decode(const unsigned long long *__restrict__ key, int64_t n,
                                 double unit, scd_span *out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const unsigned long long k = key[q];
  const uint32_t km = (uint32_t)((k >> 1) & 0x3fffffull);
  scd_span sp;
  sp.i = (uint32_t)(k >> 44);
  sp.j = (uint32_t)((k >> 24) & 0xfffffull);
  sp.t0 = (double)km * unit;
  sp.t1 = (double)(km + (uint32_t)(k & 1ull)) * unit;
  out[q] = sp;
}

// distinct tick candidates (sorted keys) as one-tick candidate pairs
__global__ void k_rf_unique(const unsigned long long *__restrict__ key, int64_t n, scd_pair *out,
                            unsigned long long *state) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const unsigned long long k = key[q];
  if (q > 0 && key[q - 1] == k) return;
  const unsigned long long w = atomicAdd(&state[RF_NUNIQ], 1ull);
  scd_pair p;
  p.i = (uint32_t)((k >> 20) & 0xfffffull);
  p.j = (uint32_t)(k & 0xfffffull);
  p.tlo = p.thi = (int32_t)(k >> 40);
  out[w] = p;
}

// the candidates the narrow phase found a witness at
__global__ void k_rf_witness_keys(const scd_pair *__restrict__ p, const int32_t *__restrict__ first,
                                  int64_t n, unsigned long long *wkey,
                                  unsigned long long *state) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n || first[q] < 0) return;
  const unsigned long long w = atomicAdd(&state[RF_NWIT], 1ull);
  wkey[w] = rf_key((uint32_t)p[q].tlo, p[q].i, p[q].j);
}

__global__ void k_rf_decode(const unsigned long long *__restrict__ wkey, int64_t n,
                            scd_witness *out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const unsigned long long k = wkey[q];
  scd_witness w;
  w.i = (uint32_t)((k >> 20) & 0xfffffull);
  w.j = (uint32_t)(k & 0xfffffull);
  w.t = (int32_t)(k >> 40);
  out[q] = w;
}

// device buffers of one call, released on every return path
struct RfBuffers {
  cudaStream_t st;
  DevBuf<uint32_t> obj[2], key, idx, flags;
  DevBuf<int32_t> t0[2], t1[2], first;
  DevBuf<float4> lo, hi;
  DevBuf<unsigned long long> cand, state, wkey;
  DevBuf<uint32_t> count, sort_err;
  DevBuf<scd_pair> pairs;
  DevBuf<scd_witness> wit;
  DevBuf<scd_span> span;
  SortScratch sc;
  explicit RfBuffers(cudaStream_t s) : st(s) {}
  ~RfBuffers() {
    for (int b = 0; b < 2; ++b) {
      obj[b].release(st);
      t0[b].release(st);
      t1[b].release(st);
    }
    key.release(st); idx.release(st); flags.release(st); first.release(st);
    lo.release(st); hi.release(st); cand.release(st); state.release(st); wkey.release(st);
    count.release(st); sort_err.release(st); pairs.release(st); wit.release(st);
    span.release(st);
    sc.release(st);
  }
};

static unsigned grid_of(int64_t n) { return (unsigned)((n + kRfThreads - 1) / kRfThreads); }

static int rf_read_state(RfBuffers &B, unsigned long long h[RF_WORDS]) {
  if (cudaMemcpyAsync(h, B.state.p, sizeof(unsigned long long) * RF_WORDS, cudaMemcpyDeviceToHost,
                      B.st) != cudaSuccess ||
      cudaStreamSynchronize(B.st) != cudaSuccess)
    return SCD_ERR_CUDA;
  return SCD_OK;
}

}  // namespace scd

using namespace scd;

extern "C" SCD_API int scd_refine_witnesses(scd_scene *s, scd_witness *host_out, int64_t cap,
                                            int64_t *n_out, int64_t *round_boxes,
                                            int *rounds) {
  if (!s || !n_out || cap < 0 || (cap > 0 && !host_out)) return SCD_ERR_INVALID_ARG;
  if (!s->boxes_built) return SCD_ERR_STATE;
  if (s->n_scenes > 0) return SCD_ERR_INVALID_ARG;  // one horizon for all objects
  if (s->n > kRfMaxObjects) return SCD_ERR_CAPACITY;
  cudaStream_t st = s->stream;
  RfBuffers B(st);
  const int64_t n = s->n;
  if (!B.state.ensure(RF_WORDS, st) || !B.sort_err.ensure(1, st)) return SCD_ERR_OOM;
  if (cudaMemsetAsync(B.state.p, 0, sizeof(unsigned long long) * RF_WORDS, st) != cudaSuccess ||
      cudaMemsetAsync(B.sort_err.p, 0, sizeof(uint32_t), st) != cudaSuccess)
    return SCD_ERR_CUDA;
  B.sc.err = B.sort_err.p;
  int cur = 0;
  if (!B.obj[0].ensure(n, st) || !B.t0[0].ensure(n, st) || !B.t1[0].ensure(n, st))
    return SCD_ERR_OOM;
  k_rf_init<<<grid_of(n), kRfThreads, 0, st>>>(n, (int32_t)s->T, B.obj[0].p, B.t0[0].p,
                                                B.t1[0].p);
  note_launch();
  int64_t M = n, ncand = 0, ccap = 1 << 16;
  if (!B.cand.ensure(ccap, st)) return SCD_ERR_OOM;
  int r = 0;
  unsigned long long h[RF_WORDS];
  for (; r < kRfMaxRounds && M > 0; ++r) {
    if (round_boxes) round_boxes[r] = M;
    const int nx = cur ^ 1;
    if (!B.lo.ensure(M, st) || !B.hi.ensure(M, st) || !B.key.ensure(M, st) ||
        !B.idx.ensure(M, st) || !B.flags.ensure(M, st) || !B.obj[nx].ensure(2 * M, st) ||
        !B.t0[nx].ensure(2 * M, st) || !B.t1[nx].ensure(2 * M, st))
      return SCD_ERR_OOM;
    RfBoxArgs ba{s->d_par.p, B.obj[cur].p, B.t0[cur].p, B.t1[cur].p, M, s->tick_s,
                 B.lo.p, B.hi.p, B.key.p, B.idx.p, B.state.p};
    k_rf_boxes<<<grid_of(M), kRfThreads, 0, st>>>(ba);
    note_launch();
    int rc = radix_sort_u32(B.key.p, B.idx.p, M, 32, B.sc, st);
    if (rc != SCD_OK) return rc;
    // the sweep, again with a larger candidate buffer if this round's
    // candidates did not fit
    for (;;) {
      if (cudaMemsetAsync(B.flags.p, 0, sizeof(uint32_t) * (size_t)M, st) != cudaSuccess)
        return SCD_ERR_CUDA;
      const unsigned long long nc0 = (unsigned long long)ncand;
      if (cudaMemcpyAsync(B.state.p + RF_NCAND, &nc0, sizeof(nc0), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
        return SCD_ERR_CUDA;
      RfSweepArgs sa{B.lo.p, B.hi.p, B.obj[cur].p, B.t0[cur].p, B.t1[cur].p, B.idx.p, M,
                     B.flags.p, B.cand.p, ccap, B.state.p, 0};
      k_rf_sweep<<<grid_of(M), kRfThreads, 0, st>>>(sa);
      note_launch();
      if ((rc = rf_read_state(B, h)) != SCD_OK) return rc;
      if ((int64_t)h[RF_NCAND] <= ccap) break;
      const int64_t want = (int64_t)h[RF_NCAND] * 2;
      if (!B.cand.grow_keep(want, ncand, st)) return SCD_ERR_OOM;
      ccap = want;
    }
    ncand = (int64_t)h[RF_NCAND];
    const unsigned long long zero = 0;
    if (cudaMemcpyAsync(B.state.p + RF_NNEXT, &zero, sizeof(zero), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return SCD_ERR_CUDA;
    k_rf_split<<<grid_of(M), kRfThreads, 0, st>>>(B.obj[cur].p, B.t0[cur].p, B.t1[cur].p,
                                                 B.flags.p, M, B.obj[nx].p, B.t0[nx].p,
                                                 B.t1[nx].p, B.state.p);
    note_launch();
    if ((rc = rf_read_state(B, h)) != SCD_OK) return rc;
    M = (int64_t)h[RF_NNEXT];
    cur = nx;
  }
  if (rounds) *rounds = r;
  if (M > 0) return SCD_ERR_INTERNAL;  // more rounds than the halvings of [0, T] allow
  if (h[RF_ERR]) return SCD_ERR_KEPLER_NOCONV;
  // distinct tick candidates, then Alg 1's test at each tick
  int64_t nw = 0;
  if (ncand > 0) {
    int rc = radix_sort_u64(B.cand.p, nullptr, ncand, 64, B.sc, st);
    if (rc != SCD_OK) return rc;
    if (!B.pairs.ensure(ncand, st) || !B.first.ensure(ncand, st)) return SCD_ERR_OOM;
    k_rf_unique<<<grid_of(ncand), kRfThreads, 0, st>>>(B.cand.p, ncand, B.pairs.p, B.state.p);
    note_launch();
    if ((rc = rf_read_state(B, h)) != SCD_OK) return rc;
    const int64_t nu = (int64_t)h[RF_NUNIQ];
    rc = scd_narrow_phase(s, B.pairs.p, nu, B.first.p, nullptr, nullptr);
    if (rc != SCD_OK) return rc;
    if (!B.wkey.ensure(nu, st)) return SCD_ERR_OOM;
    k_rf_witness_keys<<<grid_of(nu), kRfThreads, 0, st>>>(B.pairs.p, B.first.p, nu, B.wkey.p,
                                                         B.state.p);
    note_launch();
    if ((rc = rf_read_state(B, h)) != SCD_OK) return rc;
    nw = (int64_t)h[RF_NWIT];
    if (nw > 0) {
      if ((rc = radix_sort_u64(B.wkey.p, nullptr, nw, 64, B.sc, st)) != SCD_OK) return rc;
      if (!B.wit.ensure(nw, st)) return SCD_ERR_OOM;
      k_rf_decode<<<grid_of(nw), kRfThreads, 0, st>>>(B.wkey.p, nw, B.wit.p);
      note_launch();
    }
  }
  uint32_t serr = 0;
  if (cudaMemcpyAsync(&serr, B.sort_err.p, sizeof(serr), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SCD_ERR_CUDA;
  if (serr) return SCD_ERR_TIMEOUT;
  *n_out = nw;
  if (nw > cap) return SCD_ERR_BUFFER_TOO_SMALL;
  if (nw > 0 &&
      (cudaMemcpyAsync(host_out, B.wit.p, sizeof(scd_witness) * (size_t)nw, cudaMemcpyDeviceToHost,
                       st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    return SCD_ERR_CUDA;
  return SCD_OK;
}

namespace scd {
// levels of the continuous variant: interval starts take 22 bits of a span key
constexpr int kRfMaxLevels = 22;

// boxes, sort and sweep of one round (with a larger candidate buffer when
// the round's candidates do not fit); h receives the state words
static int rf_round(scd_scene *s, RfBuffers &B, int cur, int64_t M, double tick_s, int spans,
                    int64_t &ncand, int64_t &ccap, unsigned long long h[RF_WORDS]) {
  cudaStream_t st = B.st;
  RfBoxArgs ba{s->d_par.p, B.obj[cur].p, B.t0[cur].p, B.t1[cur].p, M, tick_s,
               B.lo.p, B.hi.p, B.key.p, B.idx.p, B.state.p};
  k_rf_boxes<<<grid_of(M), kRfThreads, 0, st>>>(ba);
  note_launch();
  int rc = radix_sort_u32(B.key.p, B.idx.p, M, 32, B.sc, st);
  if (rc != SCD_OK) return rc;
  for (;;) {
    if (cudaMemsetAsync(B.flags.p, 0, sizeof(uint32_t) * (size_t)M, st) != cudaSuccess)
      return SCD_ERR_CUDA;
    const unsigned long long nc0 = (unsigned long long)ncand;
    if (cudaMemcpyAsync(B.state.p + RF_NCAND, &nc0, sizeof(nc0), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return SCD_ERR_CUDA;
    RfSweepArgs sa{B.lo.p, B.hi.p, B.obj[cur].p, B.t0[cur].p, B.t1[cur].p, B.idx.p, M,
                   B.flags.p, B.cand.p, ccap, B.state.p, spans};
    k_rf_sweep<<<grid_of(M), kRfThreads, 0, st>>>(sa);
    note_launch();
    if ((rc = rf_read_state(B, h)) != SCD_OK) return rc;
    if ((int64_t)h[RF_NCAND] <= ccap) break;
    const int64_t want = (int64_t)h[RF_NCAND] * 2;
    if (!B.cand.grow_keep(want, ncand, st)) return SCD_ERR_OOM;
    ccap = want;
  }
  ncand = (int64_t)h[RF_NCAND];
  return SCD_OK;
}
}  // namespace scd

extern "C" SCD_API int scd_refine_continuous(scd_scene *s, double eps_s, scd_span *host_out,
                                             int64_t cap, int64_t *n_out, int64_t *round_boxes,
                                             int *rounds) {
  if (!s || !n_out || cap < 0 || (cap > 0 && !host_out) || !(eps_s > 0.0))
    return SCD_ERR_INVALID_ARG;
  if (!s->boxes_built) return SCD_ERR_STATE;
  if (s->n_scenes > 0) return SCD_ERR_INVALID_ARG;
  if (s->n > kRfMaxObjects) return SCD_ERR_CAPACITY;
  const double T_s = (double)s->T * s->tick_s;
  int L = 0;
  while (L <= kRfMaxLevels && ldexp(T_s, -L) > eps_s) ++L;
  if (L > kRfMaxLevels) return SCD_ERR_CAPACITY;  // eps_s below T / 2^22
  cudaStream_t st = s->stream;
  RfBuffers B(st);
  const int64_t n = s->n;
  if (!B.state.ensure(RF_WORDS, st) || !B.sort_err.ensure(1, st)) return SCD_ERR_OOM;
  if (cudaMemsetAsync(B.state.p, 0, sizeof(unsigned long long) * RF_WORDS, st) != cudaSuccess ||
      cudaMemsetAsync(B.sort_err.p, 0, sizeof(uint32_t), st) != cudaSuccess)
    return SCD_ERR_CUDA;
  B.sc.err = B.sort_err.p;
  int cur = 0;
  if (!B.obj[0].ensure(n, st) || !B.t0[0].ensure(n, st) || !B.t1[0].ensure(n, st))
    return SCD_ERR_OOM;
  k_rf_init<<<grid_of(n), kRfThreads, 0, st>>>(n, 1, B.obj[0].p, B.t0[0].p, B.t1[0].p);
  note_launch();
  int64_t M = n, ncand = 0, ccap = 1 << 16;
  if (!B.cand.ensure(ccap, st)) return SCD_ERR_OOM;
  unsigned long long h[RF_WORDS] = {};
  int r = 0;
  for (int level = 0; level <= L && M > 0; ++level, ++r) {
    if (round_boxes) round_boxes[r] = M;
    const int nx = cur ^ 1;
    if (!B.lo.ensure(M, st) || !B.hi.ensure(M, st) || !B.key.ensure(M, st) ||
        !B.idx.ensure(M, st) || !B.flags.ensure(M, st) || !B.obj[nx].ensure(2 * M, st) ||
        !B.t0[nx].ensure(2 * M, st) || !B.t1[nx].ensure(2 * M, st))
      return SCD_ERR_OOM;
    int rc = rf_round(s, B, cur, M, ldexp(T_s, -level), level == L, ncand, ccap, h);
    if (rc != SCD_OK) return rc;
    if (level == L) {
      ++r;
      break;
    }
    const unsigned long long zero = 0;
    if (cudaMemcpyAsync(B.state.p + RF_NNEXT, &zero, sizeof(zero), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return SCD_ERR_CUDA;
    k_rf_split_cont<<<grid_of(M), kRfThreads, 0, st>>>(B.obj[cur].p, B.t0[cur].p, B.flags.p, M,
                                                      B.obj[nx].p, B.t0[nx].p, B.t1[nx].p,
                                                      B.state.p);
    note_launch();
    if ((rc = rf_read_state(B, h)) != SCD_OK) return rc;
    M = (int64_t)h[RF_NNEXT];
    cur = nx;
  }
  if (rounds) *rounds = r;
  if (h[RF_ERR]) return SCD_ERR_KEPLER_NOCONV;
  int64_t nu = 0;
  if (ncand > 0) {  // spans of the finest level: distinct, in (i, j, t0, t1) order
    int rc = radix_sort_u64(B.cand.p, nullptr, ncand, 64, B.sc, st);
    if (rc != SCD_OK) return rc;
    if (!B.wkey.ensure(ncand, st)) return SCD_ERR_OOM;
    k_rf_distinct<<<grid_of(ncand), kRfThreads, 0, st>>>(B.cand.p, ncand, B.wkey.p, B.state.p);
    note_launch();
    if ((rc = rf_read_state(B, h)) != SCD_OK) return rc;
    nu = (int64_t)h[RF_NUNIQ];
    if ((rc = radix_sort_u64(B.wkey.p, nullptr, nu, 64, B.sc, st)) != SCD_OK) return rc;
    if (!B.span.ensure(nu, st)) return SCD_ERR_OOM;
    k_rf_span_decode<<<grid_of(nu), kRfThreads, 0, st>>>(B.wkey.p, nu, ldexp(T_s, -L), B.span.p);
    note_launch();
  }
  uint32_t serr = 0;
  if (cudaMemcpyAsync(&serr, B.sort_err.p, sizeof(serr), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SCD_ERR_CUDA;
  if (serr) return SCD_ERR_TIMEOUT;
  *n_out = nu;
  if (nu > cap) return SCD_ERR_BUFFER_TOO_SMALL;
  if (nu > 0 &&
      (cudaMemcpyAsync(host_out, B.span.p, sizeof(scd_span) * (size_t)nu, cudaMemcpyDeviceToHost,
                       st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    return SCD_ERR_CUDA;
  return SCD_OK;
}
