// refine.cu -- adaptive refinement: the interval growing and halving of
// Alg 5 and Alg 6 as data-parallel rounds over all objects at once.
//
// Object i starts with its ticks [0, T] cut into intervals of L_i ticks
// (the last one shorter), L_i the largest power of two not above
// max(1, floor(P_i / (f tick))), P_i its period and f the scene's start
// fraction, or the whole horizon when that is longer or f = 0: Alg 5 grows
// an interval from one step up to a bound, and a box over more than a few
// hundredths of an orbit meets nearly every other box of a crowded catalog,
// so the rounds with longer intervals would halve nearly everything at full
// cost and decide nothing.  A round builds the 4D box of every active
// interval (Def 8, in the scene's box mode), finds the boxes that meet a
// box of another object, and then
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
// the intersection of the two intervals.  The box kernel serves both: with
// t0 = k, t1 = k + 1 and the level's unit as the tick, a box covers the real
// interval.
//
// The meeting boxes of a round are found with the screen's machinery: the
// boxes are sorted along a 4D Morton curve, a binary radix tree with
// compact quantised nodes is built over them, and the persistent traversal
// (in its refinement mode) flags both intervals of every meeting pair and
// collects the candidates.  The rounds run without the host: every kernel
// reads the round's interval count from device memory, and the host queues
// all rounds at once (ceil(log2(L)) + 2 of them, L the longest first
// interval, or the levels of the continuous variant) and reads the counts once at the end.  The
// buffers are sized for a capacity of intervals per round; a round that
// would exceed it is cut short and flagged, and the call runs again with a
// larger capacity (kept on the scene for the next call).
#include <math.h>

#include <algorithm>

#include "kepler.cuh"
#include <cstring>

#include "scd_internal.cuh"

namespace scd {

constexpr int kRfThreads = 256;
constexpr int kRfMaxRounds = 64;
// object indices take 20 bits and ticks 24 in a packed candidate key
constexpr int64_t kRfMaxObjects = 1ll << 20;
// device state words: tick candidates, next intervals, error bits, unique
// candidates, witnesses, this round's intervals, the largest next-round
// count asked for
enum {
  RF_NCAND = 0, RF_NNEXT = 1, RF_ERR = 2, RF_NUNIQ = 3, RF_NWIT = 4, RF_M = 5, RF_OVER = 6,
  RF_LMAX = 7, RF_WORDS = 8
};
// the rounds' 4D Morton keys: 10 bits per axis, time weighed 4x against
// space (24 h catalog rounds 552 -> 522 ms against equal weights; 12-bit axes
// with weight 8, the screen's choice, 519 ms but slower on small rounds)
constexpr int kRfMortonBits = 10;
constexpr float kRfTimeScale = 4.0f;

__device__ __forceinline__ int64_t rf_count(const unsigned long long *state, int64_t cap) {
  const unsigned long long m = state[RF_M];
  return m < (unsigned long long)cap ? (int64_t)m : cap;
}

// The first interval length of an object in ticks: the largest power of
// two not above max(1, floor(P / unit)), unit = f tick for the start
// fraction f, or T + 1 when longer or f = 0 (a bounded first interval:
// Alg 5's intervals grow from one step up to a bound; the rounds before, in
// which nearly every box meets another, are skipped).  The division is
// rounded as the oracle's.
__device__ __forceinline__ int32_t rf_start_ticks(const ObjParams &p, int32_t T, double unit) {
  if (!(unit > 0.0)) return T + 1;
  const double q = floor(__ddiv_rn(p.P, unit));
  int64_t L = 1;
  while (L <= T && (double)(2 * L) <= q) L *= 2;  // past T the answer is T + 1
  return L > T ? T + 1 : (int32_t)L;
}

// per object its first round's intervals, and the longest first interval
__global__ void k_rf_start_count(const ObjParams *__restrict__ par, int64_t n, int32_t T,
                                 double unit, int64_t *__restrict__ cnt,
                                 unsigned long long *__restrict__ state) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const int32_t L = rf_start_ticks(par[o], T, unit);
  cnt[o] = ((int64_t)T + L) / L;  // ceil((T + 1) / L)
  atomicMax(&state[RF_LMAX], (unsigned long long)L);
}

// The first round's intervals, object-major: [k L, min((k + 1) L - 1, T)],
// one warp per object; at most cap of them written, the count asked for
// noted for the retry.
__global__ void k_rf_init_start(const ObjParams *__restrict__ par, int64_t n, int32_t T,
                                double unit, const int64_t *__restrict__ off, int64_t cap,
                                uint32_t *obj, int32_t *t0, int32_t *t1,
                                unsigned long long *state) {
  const int64_t total = off[n];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    state[RF_M] = (unsigned long long)(total < cap ? total : cap);
    if (total > cap) atomicMax(&state[RF_OVER], (unsigned long long)total);
  }
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; o < n; o += nw) {
    const int64_t L = rf_start_ticks(par[o], T, unit);
    const int64_t b0 = off[o], c = off[o + 1] - b0;
    for (int64_t k = lane; k < c && b0 + k < cap; k += 32) {
      const int64_t a = k * L, b = a + L - 1;
      obj[b0 + k] = (uint32_t)o;
      t0[b0 + k] = (int32_t)a;
      t1[b0 + k] = (int32_t)(b < T ? b : T);
    }
  }
}

__global__ void k_rf_init(int64_t n, int32_t T, uint32_t *obj, int32_t *t0, int32_t *t1,
                          unsigned long long *state) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) state[RF_M] = (unsigned long long)n;
  if (i >= n) return;
  obj[i] = (uint32_t)i;
  t0[i] = 0;
  t1[i] = T;
}

struct RfBoxArgs {
  const ObjParams *par;
  int mode;                     // SPEED or INTERVAL boxes
  const uint32_t *obj;
  const int32_t *t0, *t1;
  int64_t cap;
  const unsigned long long *state;
  unsigned long long *round_count;  // this round's entry of the per-round counts
  double tick_s;                // the length of one unit of t0, t1 [s]
  const DevCounters *ctr;       // the scene's extent (key frame)
  int64_t Tf;                   // the time extent of the key frame [units]
  float split_km;
  float4 *lo, *hi;
  unsigned long long *key;
  uint32_t *idx;
  unsigned long long *err;
};

// the box, Morton key and index of interval i
__device__ __forceinline__ void rf_box(const RfBoxArgs &a, int64_t i) {
  const ObjParams &p = a.par[a.obj[i]];
  const int32_t t0 = a.t0[i], t1 = a.t1[i];
  double lo[3], hi[3];
  int iters = 0;
  segment_box(p, a.mode, t0, t1, a.tick_s, lo, hi, iters);
  if (iters >= kKeplerMaxIter) atomicOr(a.err, 1ull);
  float4 L, H;
  L.x = __double2float_rd(lo[0]);
  L.y = __double2float_rd(lo[1]);
  L.z = __double2float_rd(lo[2]);
  H.x = __double2float_ru(hi[0]);
  H.y = __double2float_ru(hi[1]);
  H.z = __double2float_ru(hi[2]);
  L.w = (float)t0;  // < 2^24: exact
  H.w = (float)t1;
  a.lo[i] = L;
  a.hi[i] = H;
  const float R = (float)__longlong_as_double((long long)a.ctr->extent_bits);
  unsigned long long k =
      box_morton(L, H, R, (float)(a.Tf + 1), kRfMortonBits, kRfTimeScale, 0);
  k |= (unsigned long long)split_bit(L, H, a.split_km) << (4 * kRfMortonBits);
  a.key[i] = k;
  a.idx[i] = (uint32_t)i;
}

__global__ void __launch_bounds__(kRfThreads) k_rf_boxes(RfBoxArgs a) {
  const int64_t M = rf_count(a.state, a.cap);
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i0 == 0) *a.round_count = (unsigned long long)M;
  for (int64_t i = i0; i < M; i += (int64_t)gridDim.x * blockDim.x) rf_box(a, i);
}

// the sorted boxes (32-byte records) and their objects
__global__ void __launch_bounds__(kRfThreads) k_rf_gather(const uint32_t *__restrict__ idx,
                                                          const float4 *__restrict__ lo,
                                                          const float4 *__restrict__ hi,
                                                          const uint32_t *__restrict__ obj,
                                                          int64_t cap,
                                                          const unsigned long long *state,
                                                          SBox *sbox, uint32_t *sobj) {
  const int64_t M = rf_count(state, cap);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < M;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = idx[p];
    sbox[p].lo = lo[i];
    sbox[p].hi = hi[i];
    sobj[p] = obj[i];
  }
}

// Slots for `need` next-round intervals of each lane of a warp: one atomic
// on the next-round count per warp (the lanes' slots follow one another).
// Every lane of the warp calls it.
__device__ __forceinline__ unsigned long long rf_claim(unsigned long long *nnext,
                                                       uint32_t need) {
  const int lane = threadIdx.x & 31;
  uint32_t incl = need;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && total) base = atomicAdd(nnext, (unsigned long long)total);
  base = __shfl_sync(0xffffffffu, base, 31);
  return base + (incl - need);
}

// next round's intervals (order is free: appended by atomics); entries past
// the capacity are not written, and the count asked for shows it
__global__ void __launch_bounds__(kRfThreads) k_rf_split(const uint32_t *__restrict__ obj,
                                                         const int32_t *__restrict__ t0,
                                                         const int32_t *__restrict__ t1,
                                                         const uint32_t *__restrict__ flags,
                                                         int64_t cap, uint32_t *nobj,
                                                         int32_t *nt0, int32_t *nt1,
                                                         unsigned long long *state) {
  const int64_t M = rf_count(state, cap);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // whole warps walk the intervals (rf_claim needs every lane)
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < M;
       base += stride) {
    const int64_t i = base + (threadIdx.x & 31);
    uint32_t need = 0, o = 0;
    int32_t a0 = 0, a1 = 0;
    if (i < M) {
      const uint32_t f = flags[i];
      if (f & kRfHit) {  // else proven free of collisions over [t0, t1]
        a0 = t0[i];
        a1 = t1[i];
        o = obj[i];
        // halved, or a single tick waiting for the longer intervals it meets
        need = a1 > a0 ? 2u : ((f & kRfHitLong) ? 1u : 0u);
      }
    }
    const unsigned long long q = rf_claim(&state[RF_NNEXT], need);
    // every slot below the capacity is written, also by the lane whose two
    // slots straddle it: a round cut short still reads all of its intervals
    if (need == 0 || q >= (unsigned long long)cap) continue;
    const int32_t mid = need == 2 ? a0 + (a1 - a0) / 2 : a1;
    nobj[q] = o;
    nt0[q] = a0;
    nt1[q] = mid;
    if (need == 2 && q + 1 < (unsigned long long)cap) {
      nobj[q + 1] = o;
      nt0[q + 1] = mid + 1;
      nt1[q + 1] = a1;
    }
  }
}

// continuous variant: both halves of an interval [k, k + 1] that met, as
// [2k, 2k + 1] and [2k + 1, 2k + 2] in units of the next level
__global__ void __launch_bounds__(kRfThreads) k_rf_split_cont(const uint32_t *__restrict__ obj,
                                                              const int32_t *__restrict__ t0,
                                                              const uint32_t *__restrict__ flags,
                                                              int64_t cap, uint32_t *nobj,
                                                              int32_t *nt0, int32_t *nt1,
                                                              unsigned long long *state) {
  const int64_t M = rf_count(state, cap);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < M;
       base += stride) {
    const int64_t i = base + (threadIdx.x & 31);
    const uint32_t need = (i < M && (flags[i] & kRfHit)) ? 2u : 0u;
    const unsigned long long q = rf_claim(&state[RF_NNEXT], need);
    if (need == 0 || q >= (unsigned long long)cap) continue;  // (slots below cap all written)
    const int32_t k = t0[i];
    nobj[q] = obj[i];
    nt0[q] = 2 * k;
    nt1[q] = 2 * k + 1;
    if (q + 1 < (unsigned long long)cap) {
      nobj[q + 1] = obj[i];
      nt0[q + 1] = 2 * k + 1;
      nt1[q + 1] = 2 * k + 2;
    }
  }
}

// a copy of round r's boxes and objects after those of the rounds before it
// (the trace of scd_refine_trace), if they fit in tcap entries
__global__ void __launch_bounds__(kRfThreads) k_rf_trace(const float4 *__restrict__ lo,
                                                         const float4 *__restrict__ hi,
                                                         const uint32_t *__restrict__ obj,
                                                         int64_t cap,
                                                         const unsigned long long *state,
                                                         const unsigned long long *rounds, int r,
                                                         float4 *tlo, float4 *thi,
                                                         uint32_t *tobj, int64_t tcap) {
  const int64_t M = rf_count(state, cap);
  unsigned long long off = 0;
  for (int q = 0; q < r; ++q) off += rounds[q];
  if (off + (unsigned long long)M > (unsigned long long)tcap) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    tlo[off + i] = lo[i];
    thi[off + i] = hi[i];
    tobj[off + i] = obj[i];
  }
}

// the next round's count becomes the current one (at most the capacity; the
// largest count asked for is kept)
__global__ void k_rf_advance(unsigned long long *state, int64_t cap) {
  const unsigned long long nx = state[RF_NNEXT];
  if (nx > state[RF_OVER]) state[RF_OVER] = nx;
  state[RF_M] = nx < (unsigned long long)cap ? nx : (unsigned long long)cap;
  state[RF_NNEXT] = 0;
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
  wkey[w] = rf_tick_key((uint32_t)p[q].tlo, p[q].i, p[q].j);
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
  DevBuf<uint32_t> obj[2], idx, flags, sobj, qlink, arrive;
  DevBuf<int32_t> t0[2], t1[2], first, parent_int, parent_leaf;
  DevBuf<float4> lo, hi;
  DevBuf<unsigned long long> key, cand, state, wkey, rounds;
  DevBuf<SBox> sbox;
  DevBuf<TravNode> nodes;
  DevBuf<QBox> nq, qbox;
  DevBuf<DevCounters> ctr;
  DevBuf<uint32_t> sort_err;
  DevBuf<scd_pair> pairs;
  DevBuf<scd_witness> wit;
  DevBuf<scd_span> span;
  DevBuf<float4> tlo, thi;  // trace (scd_refine_trace): every round's boxes
  DevBuf<uint32_t> tobj;
  int64_t tcap = 0;
  // discrete rounds: per object its first intervals and their offsets
  DevBuf<int64_t> scnt, soff, stmp;
  int64_t start_total = 0;
  // the rounds' sort scratch (inside a captured graph: sized only by size())
  // and the scratch of the sorts after the rounds
  SortScratch sc, sc_post;
  explicit RfBuffers(cudaStream_t s) : st(s) {}
  ~RfBuffers() {
    for (int b = 0; b < 2; ++b) {
      obj[b].release(st);
      t0[b].release(st);
      t1[b].release(st);
    }
    idx.release(st); flags.release(st); sobj.release(st); qlink.release(st);
    arrive.release(st); first.release(st); parent_int.release(st); parent_leaf.release(st);
    lo.release(st); hi.release(st); key.release(st); cand.release(st); state.release(st);
    wkey.release(st); rounds.release(st); sbox.release(st); nodes.release(st); nq.release(st);
    qbox.release(st); ctr.release(st); sort_err.release(st); pairs.release(st);
    wit.release(st); span.release(st); tlo.release(st); thi.release(st); tobj.release(st);
    scnt.release(st); soff.release(st); stmp.release(st);
    sc.release(st);
    sc_post.release(st);
  }
  // every per-interval buffer for `cap` intervals a round, and `ccap`
  // candidates
  bool size(int64_t cap, int64_t ccap) {
    const size_t c = (size_t)cap;
    for (int b = 0; b < 2; ++b)
      if (!obj[b].ensure(c, st) || !t0[b].ensure(c, st) || !t1[b].ensure(c, st)) return false;
    return idx.ensure(c, st) && flags.ensure(c, st) && sobj.ensure(c, st) &&
           qlink.ensure(c, st) && arrive.ensure(c, st) && parent_int.ensure(c, st) &&
           parent_leaf.ensure(c, st) && lo.ensure(c, st) && hi.ensure(c, st) &&
           key.ensure(c, st) && sbox.ensure(c, st) && nodes.ensure(c, st) && nq.ensure(c, st) &&
           qbox.ensure(2 * c, st) && cand.ensure((size_t)ccap, st) &&
           sort_reserve(sc, cap, sizeof(unsigned long long), true, st) == SCD_OK;
  }
};

static unsigned grid_of(int64_t n) { return (unsigned)((n + kRfThreads - 1) / kRfThreads); }

// the grid of a round kernel over up to n items: the blocks that are
// resident at once, or fewer (its threads loop over the round's count, read
// on the device, so an almost empty round costs one short wave)
static unsigned wave_of(int64_t n) {
  static int wave = 0;
  if (!wave) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    wave = std::max(1, sms) * (2048 / kRfThreads);
  }
  return std::min<unsigned>(grid_of(std::max<int64_t>(n, 1)), (unsigned)wave);
}

static int rf_read_state(RfBuffers &B, unsigned long long h[RF_WORDS]) {
  if (cudaMemcpyAsync(h, B.state.p, sizeof(unsigned long long) * RF_WORDS, cudaMemcpyDeviceToHost,
                      B.st) != cudaSuccess ||
      cudaStreamSynchronize(B.st) != cudaSuccess)
    return SCD_ERR_CUDA;
  return SCD_OK;
}

// the unit of rf_start_ticks: the scene's start fraction of a period times
// the tick [s], 0 for whole-horizon first intervals
static double rf_start_unit(const scd_scene *s) {
  return s->tune.refine_start > 0.0f ? (double)s->tune.refine_start * s->tick_s : 0.0;
}

// The first intervals of the discrete rounds (rf_start_ticks): their counts
// per object, the offsets, and on the host their total and the number of
// rounds that halve the longest down to single ticks and decide them.
static int rf_start(scd_scene *s, RfBuffers &B, int &rounds) {
  cudaStream_t st = B.st;
  const int64_t n = s->n;
  if (!B.scnt.ensure((size_t)n, st) || !B.soff.ensure((size_t)n + 1, st)) return SCD_ERR_OOM;
  if (cudaMemsetAsync(B.state.p, 0, sizeof(unsigned long long) * RF_WORDS, st) != cudaSuccess)
    return SCD_ERR_CUDA;
  if (n > 0) {
    k_rf_start_count<<<grid_of(n), kRfThreads, 0, st>>>(s->d_par.p, n, (int32_t)s->T,
                                                        rf_start_unit(s), B.scnt.p, B.state.p);
    note_launch();
  }
  int rc = scan_exclusive_i64(B.scnt.p, B.soff.p, n, B.stmp, st);
  if (rc != SCD_OK) return rc;
  int64_t total = 0;
  unsigned long long lmax = 0;
  if (cudaMemcpyAsync(&total, B.soff.p + n, sizeof(total), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(&lmax, B.state.p + RF_LMAX, sizeof(lmax), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SCD_ERR_CUDA;
  B.start_total = total;
  rounds = 2;
  while ((1ull << (rounds - 2)) < lmax) ++rounds;
  return SCD_OK;
}

// The rounds of one call, queued at once.  Discrete: rounds from the first
// intervals (rf_start) until nothing is left (at most `rounds` of them).  Continuous
// (levels >= 0): level l = 0 .. levels in units of T_s / 2^l, spans at the
// last.  On return h holds the state words and round_counts the intervals
// of every round; the caller checks capacity, candidates and the stack.
static int rf_queue(scd_scene *s, RfBuffers &B, int64_t cap, int64_t ccap, int deep,
                    int rounds, int levels) {
  cudaStream_t st = B.st;
  const int64_t n = s->n;
  if (cudaMemsetAsync(B.state.p, 0, sizeof(unsigned long long) * RF_WORDS, st) != cudaSuccess ||
      cudaMemsetAsync(B.rounds.p, 0, sizeof(unsigned long long) * kRfMaxRounds, st) !=
          cudaSuccess ||
      cudaMemsetAsync(B.sort_err.p, 0, sizeof(uint32_t), st) != cudaSuccess ||
      cudaMemsetAsync(B.ctr.p, 0, sizeof(DevCounters), st) != cudaSuccess ||
      cudaMemcpyAsync(&B.ctr.p->extent_bits, &s->d_ctr.p->extent_bits, sizeof(unsigned long long),
                      cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SCD_ERR_CUDA;
  const bool cont = levels >= 0;
  const double T_s = (double)s->T * s->tick_s;
  if (cont)
    k_rf_init<<<grid_of(n), kRfThreads, 0, st>>>(n, 1, B.obj[0].p, B.t0[0].p, B.t1[0].p,
                                                  B.state.p);
  else
    k_rf_init_start<<<wave_of(32 * n), kRfThreads, 0, st>>>(s->d_par.p, n, (int32_t)s->T,
                                                             rf_start_unit(s), B.soff.p, cap,
                                                             B.obj[0].p, B.t0[0].p, B.t1[0].p,
                                                             B.state.p);
  note_launch();
  const float split = split_of(s->tune);
  const int kb = 4 * kRfMortonBits + (split != 0.0f);
  unsigned long long *dM = B.state.p + RF_M;
  const int nr = cont ? levels + 1 : rounds;
  int cur = 0;
  for (int r = 0; r < nr; ++r) {
    const int nx = cur ^ 1;
    // the unit of t0, t1 and the time extent of the key frame
    const double unit = cont ? ldexp(T_s, -r) : s->tick_s;
    const int64_t Tf = cont ? (1ll << r) : s->T;
    RfBoxArgs ba{s->d_par.p, s->box_mode, B.obj[cur].p, B.t0[cur].p, B.t1[cur].p, cap,
                 B.state.p, B.rounds.p + r, unit, B.ctr.p, Tf, split, B.lo.p, B.hi.p,
                 B.key.p, B.idx.p, B.state.p + RF_ERR};
    k_rf_boxes<<<wave_of(cap), kRfThreads, 0, st>>>(ba);
    note_launch();
    if (B.tcap > 0) {
      k_rf_trace<<<wave_of(cap), kRfThreads, 0, st>>>(B.lo.p, B.hi.p, B.obj[cur].p, cap, B.state.p,
                                                     B.rounds.p, r, B.tlo.p, B.thi.p, B.tobj.p,
                                                     B.tcap);
      note_launch();
    }
    int rc = radix_sort_u64_dev(B.key.p, B.idx.p, cap, dM, 0, kb, B.sc, st);
    if (rc != SCD_OK) return rc;
    k_rf_gather<<<wave_of(cap), kRfThreads, 0, st>>>(B.idx.p, B.lo.p, B.hi.p, B.obj[cur].p, cap,
                                                     B.state.p, B.sbox.p, B.sobj.p);
    note_launch();
    rc = build_round_tree(B.key.p, B.sbox.p, cap, dM, B.nodes.p, B.parent_int.p,
                          B.parent_leaf.p, B.arrive.p, B.nq.p, B.qbox.p, B.qlink.p, B.ctr.p, Tf,
                          st);
    if (rc != SCD_OK) return rc;
    // the flags, and the traversal's counters (its error bits, which follow
    // them, stay set across the rounds)
    if (cudaMemsetAsync(B.flags.p, 0, sizeof(uint32_t) * (size_t)cap, st) != cudaSuccess ||
        cudaMemsetAsync(B.ctr.p, 0, offsetof(DevCounters, trav_flags), st) != cudaSuccess)
      return SCD_ERR_CUDA;
    const int spans = cont && r == levels;
    rc = traverse_round(B.qbox.p, B.qlink.p, B.sbox.p, B.sobj.p, B.idx.p, cap, dM, Tf, B.ctr.p,
                        B.flags.p, B.cand.p, B.state.p + RF_NCAND, (unsigned long long)ccap,
                        spans, deep, st);
    if (rc != SCD_OK) return rc;
    if (spans) break;
    if (cont)
      k_rf_split_cont<<<wave_of(cap), kRfThreads, 0, st>>>(B.obj[cur].p, B.t0[cur].p, B.flags.p,
                                                          cap, B.obj[nx].p, B.t0[nx].p,
                                                          B.t1[nx].p, B.state.p);
    else
      k_rf_split<<<wave_of(cap), kRfThreads, 0, st>>>(B.obj[cur].p, B.t0[cur].p, B.t1[cur].p,
                                                     B.flags.p, cap, B.obj[nx].p, B.t0[nx].p,
                                                     B.t1[nx].p, B.state.p);
    k_rf_advance<<<1, 1, 0, st>>>(B.state.p, cap);
    note_launch(2);
    cur = nx;
  }
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

// the rounds' sizes, the traversal flags and the state words, after the queue
static int rf_collect(RfBuffers &B, unsigned long long h[RF_WORDS],
                      unsigned long long *round_counts, unsigned int &trav_flags) {
  if (cudaMemcpyAsync(round_counts, B.rounds.p, sizeof(unsigned long long) * kRfMaxRounds,
                      cudaMemcpyDeviceToHost, B.st) != cudaSuccess ||
      cudaMemcpyAsync(&trav_flags, &B.ctr.p->trav_flags, sizeof(unsigned int),
                      cudaMemcpyDeviceToHost, B.st) != cudaSuccess)
    return SCD_ERR_CUDA;
  return rf_read_state(B, h);
}

// The rounds' queue captured as one CUDA graph, replayed while the call's
// shape (sizes, capacities, rounds) and the scene's buffers stay the same:
// the small cases are launch-bound (about 30 launches a round).  The
// buffers live with the scene so that the graph's pointers stay valid.
struct RfCache {
  RfBuffers B;
  cudaStream_t gst = nullptr;
  cudaEvent_t in = nullptr, out = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t key[11] = {};
  unsigned long long nlaunch = 0;  // kernels in the graph
  explicit RfCache(cudaStream_t st) : B(st) {}
  ~RfCache() {
    if (exec) cudaGraphExecDestroy(exec);
    if (gst) {
      cudaStreamSynchronize(gst);
      cudaStreamDestroy(gst);
    }
    if (in) cudaEventDestroy(in);
    if (out) cudaEventDestroy(out);
  }
};

static void rf_key(const scd_scene *s, const RfBuffers &B, int64_t cap, int64_t ccap, int deep,
                   int rounds, int levels, int64_t k[11]) {
  k[0] = cap;
  k[1] = ccap;
  k[2] = deep;
  k[3] = rounds;
  k[4] = levels;
  k[5] = s->n;
  k[6] = s->T;
  k[7] = s->box_mode * 1000000 + (int64_t)(split_of(s->tune) * 10.0f);
  k[8] = (int64_t)reinterpret_cast<uintptr_t>(B.obj[0].p) ^ (int64_t)reinterpret_cast<uintptr_t>(s->d_par.p);
  int64_t tb;
  memcpy(&tb, &s->tick_s, sizeof(tb));
  k[9] = tb;
  k[10] = (int64_t)(rf_start_unit(s) * 1e6);  // baked into the first round's launch
}

// queue the rounds: by the cached graph when its shape matches, else
// eagerly
static int rf_rounds(scd_scene *s, RfBuffers &B, RfCache *gc, int64_t cap, int64_t ccap,
                     int deep, int rounds, int levels, unsigned long long h[RF_WORDS],
                     unsigned long long *round_counts, unsigned int &trav_flags) {
  int64_t k[11];
  rf_key(s, B, cap, ccap, deep, rounds, levels, k);
  if (gc && gc->exec && memcmp(k, gc->key, sizeof(k)) == 0) {
    if (cudaEventRecord(gc->in, B.st) != cudaSuccess ||
        cudaStreamWaitEvent(gc->gst, gc->in, 0) != cudaSuccess ||
        cudaGraphLaunch(gc->exec, gc->gst) != cudaSuccess ||
        cudaEventRecord(gc->out, gc->gst) != cudaSuccess ||
        cudaStreamWaitEvent(B.st, gc->out, 0) != cudaSuccess)
      return SCD_ERR_CUDA;
    note_launch(gc->nlaunch);
  } else {
    int rc = rf_queue(s, B, cap, ccap, deep, rounds, levels);
    if (rc != SCD_OK) return rc;
  }
  return rf_collect(B, h, round_counts, trav_flags);
}

// capture the queue of a shape that has just run eagerly (nothing is
// allocated while capturing: every buffer is sized); without a graph the
// calls stay eager
static void rf_capture(scd_scene *s, RfCache &gc, int64_t cap, int64_t ccap, int deep,
                       int rounds, int levels) {
  if (!gc.gst) {
    if (cudaStreamCreateWithFlags(&gc.gst, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&gc.in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&gc.out, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
  }
  if (gc.exec) {
    cudaGraphExecDestroy(gc.exec);
    gc.exec = nullptr;
  }
  if (cudaStreamSynchronize(gc.B.st) != cudaSuccess) return;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(gc.gst, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const cudaStream_t st = gc.B.st;
  gc.B.st = gc.gst;
  const unsigned long long mark = launch_count();
  const int rc = rf_queue(s, gc.B, cap, ccap, deep, rounds, levels);
  const cudaError_t e = cudaStreamEndCapture(gc.gst, &g);
  gc.B.st = st;
  gc.nlaunch = launch_count() - mark;
  if (rc == SCD_OK && e == cudaSuccess && g &&
      cudaGraphInstantiate(&gc.exec, g, 0) == cudaSuccess) {
    rf_key(s, gc.B, cap, ccap, deep, rounds, levels, gc.key);
  } else {
    gc.exec = nullptr;
    cudaGetLastError();
  }
  if (g) cudaGraphDestroy(g);
}

}  // namespace scd

namespace scd {
// Queue the rounds, and again with more room while a round's intervals, the
// candidates or a traversal stack did not fit.  The capacities that sufficed
// stay on the scene for its next call.
// Discrete rounds (levels < 0) set `rounds` from their first intervals.
static int rf_run(scd_scene *s, RfBuffers &B, RfCache *gc, int &rounds, int levels,
                  unsigned long long h[RF_WORDS], unsigned long long *round_counts) {
  cudaStream_t st = B.st;
  if (!B.state.ensure(RF_WORDS, st) || !B.sort_err.ensure(1, st) ||
      !B.rounds.ensure(kRfMaxRounds, st) || !B.ctr.ensure(1, st))
    return SCD_ERR_OOM;
  B.sc.err = B.sort_err.p;
  B.sc_post.err = B.sort_err.p;
  int64_t cap = std::max<int64_t>(s->rf_cap, std::max<int64_t>(4 * s->n, 1 << 16));
  if (levels < 0) {
    int rc = rf_start(s, B, rounds);
    if (rc != SCD_OK) return rc;
    if (rounds > kRfMaxRounds) return SCD_ERR_INTERNAL;
    cap = std::max<int64_t>(cap, B.start_total);
  }
  int64_t ccap = std::max<int64_t>(s->rf_ccap, 1 << 16);
  int deep = s->rf_deep;
  for (int attempt = 0; attempt < 8; ++attempt) {
    if (!B.size(cap, ccap)) return SCD_ERR_OOM;
    unsigned int tf = 0;
    int rc = rf_rounds(s, B, gc, cap, ccap, deep, rounds, levels, h, round_counts, tf);
    if (rc != SCD_OK) return rc;
    bool again = false;
    if (h[RF_OVER] > (unsigned long long)cap) {
      cap = (int64_t)std::max<unsigned long long>(2ull * (unsigned long long)cap, 2ull * h[RF_OVER]);
      again = true;
    }
    if (h[RF_NCAND] > (unsigned long long)ccap) {
      ccap = (int64_t)(2ull * h[RF_NCAND]);
      again = true;
    }
    if (tf & ERR_STACK) {
      if (deep) return SCD_ERR_INTERNAL;
      deep = 1;
      again = true;
    }
    if (!again) {
      s->rf_cap = cap;
      s->rf_ccap = ccap;
      s->rf_deep = deep;
      if (gc) {
        int64_t k[11];
        rf_key(s, B, cap, ccap, deep, rounds, levels, k);
        if (!gc->exec || memcmp(k, gc->key, sizeof(k)) != 0)
          rf_capture(s, *gc, cap, ccap, deep, rounds, levels);
      }
      return SCD_OK;
    }
  }
  return SCD_ERR_CAPACITY;
}

// the scene's refinement buffers and graph, made on first use
static RfCache &rf_cache(scd_scene *s) {
  if (!s->rf) s->rf = new RfCache(s->stream);
  s->rf->B.st = s->stream;
  return *s->rf;
}

void rf_release(scd_scene *s) {
  delete s->rf;
  s->rf = nullptr;
}

static int rf_check_scene(const scd_scene *s) {
  if (!s->boxes_built) return SCD_ERR_STATE;
  if (s->n_scenes > 0) return SCD_ERR_INVALID_ARG;  // one horizon for all objects
  if (s->n > kRfMaxObjects) return SCD_ERR_CAPACITY;
  return SCD_OK;
}
}  // namespace scd

using namespace scd;

extern "C" SCD_API int scd_refine_witnesses(scd_scene *s, scd_witness *host_out, int64_t cap,
                                            int64_t *n_out, int64_t *round_boxes,
                                            int *rounds) {
  if (!s || !n_out || cap < 0 || (cap > 0 && !host_out)) return SCD_ERR_INVALID_ARG;
  if (int rc = rf_check_scene(s)) return rc;
  const unsigned long long mark = launch_count();
  cudaStream_t st = s->stream;
  RfCache &gc = rf_cache(s);
  RfBuffers &B = gc.B;
  // the halvings of the longest first interval down to single ticks, one
  // round to decide them and one for single ticks that wait for a longer
  // interval
  int nr = 0;
  unsigned long long h[RF_WORDS], rc_[kRfMaxRounds];
  int rc = rf_run(s, B, &gc, nr, -1, h, rc_);
  if (rc != SCD_OK) return rc;
  int r = 0;
  while (r < nr && rc_[r] > 0) {
    if (round_boxes) round_boxes[r] = (int64_t)rc_[r];
    ++r;
  }
  if (rounds) *rounds = r;
  if (h[RF_M] > 0) return SCD_ERR_INTERNAL;  // more rounds than the halvings allow
  if (h[RF_ERR]) return SCD_ERR_KEPLER_NOCONV;
  const int64_t ncand = (int64_t)h[RF_NCAND];
  // distinct tick candidates, then Alg 1's test at each tick
  int64_t nw = 0;
  if (ncand > 0) {
    int rc2 = radix_sort_u64(B.cand.p, nullptr, ncand, 64, B.sc_post, st);
    if (rc2 != SCD_OK) return rc2;
    if (!B.pairs.ensure(ncand, st) || !B.first.ensure(ncand, st)) return SCD_ERR_OOM;
    k_rf_unique<<<grid_of(ncand), kRfThreads, 0, st>>>(B.cand.p, ncand, B.pairs.p, B.state.p);
    note_launch();
    if ((rc2 = rf_read_state(B, h)) != SCD_OK) return rc2;
    const int64_t nu = (int64_t)h[RF_NUNIQ];
    rc2 = scd_narrow_phase(s, B.pairs.p, nu, B.first.p, nullptr, nullptr);
    if (rc2 != SCD_OK) return rc2;
    if (!B.wkey.ensure(nu, st)) return SCD_ERR_OOM;
    k_rf_witness_keys<<<grid_of(nu), kRfThreads, 0, st>>>(B.pairs.p, B.first.p, nu, B.wkey.p,
                                                         B.state.p);
    note_launch();
    if ((rc2 = rf_read_state(B, h)) != SCD_OK) return rc2;
    nw = (int64_t)h[RF_NWIT];
    if (nw > 0) {
      if ((rc2 = radix_sort_u64(B.wkey.p, nullptr, nw, 64, B.sc_post, st)) != SCD_OK) return rc2;
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
  s->last_launches = launch_count() - mark;
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
}  // namespace scd

extern "C" SCD_API int scd_refine_continuous(scd_scene *s, double eps_s, scd_span *host_out,
                                             int64_t cap, int64_t *n_out, int64_t *round_boxes,
                                             int *rounds) {
  if (!s || !n_out || cap < 0 || (cap > 0 && !host_out) || !(eps_s > 0.0))
    return SCD_ERR_INVALID_ARG;
  if (int rc = rf_check_scene(s)) return rc;
  const double T_s = (double)s->T * s->tick_s;
  int L = 0;
  while (L <= kRfMaxLevels && ldexp(T_s, -L) > eps_s) ++L;
  if (L > kRfMaxLevels) return SCD_ERR_CAPACITY;  // eps_s below T / 2^22
  const unsigned long long mark = launch_count();
  cudaStream_t st = s->stream;
  RfCache &gc = rf_cache(s);
  RfBuffers &B = gc.B;
  unsigned long long h[RF_WORDS], rc_[kRfMaxRounds];
  int nr = 0;
  int rc = rf_run(s, B, &gc, nr, L, h, rc_);
  if (rc != SCD_OK) return rc;
  int r = 0;
  while (r <= L && rc_[r] > 0) {
    if (round_boxes) round_boxes[r] = (int64_t)rc_[r];
    ++r;
  }
  if (rounds) *rounds = r;
  if (h[RF_ERR]) return SCD_ERR_KEPLER_NOCONV;
  const int64_t ncand = (int64_t)h[RF_NCAND];
  int64_t nu = 0;
  if (ncand > 0) {  // spans of the finest level: distinct, in (i, j, t0, t1) order
    int rc2 = radix_sort_u64(B.cand.p, nullptr, ncand, 64, B.sc_post, st);
    if (rc2 != SCD_OK) return rc2;
    if (!B.wkey.ensure(ncand, st)) return SCD_ERR_OOM;
    k_rf_distinct<<<grid_of(ncand), kRfThreads, 0, st>>>(B.cand.p, ncand, B.wkey.p, B.state.p);
    note_launch();
    if ((rc2 = rf_read_state(B, h)) != SCD_OK) return rc2;
    nu = (int64_t)h[RF_NUNIQ];
    if ((rc2 = radix_sort_u64(B.wkey.p, nullptr, nu, 64, B.sc_post, st)) != SCD_OK) return rc2;
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
  s->last_launches = launch_count() - mark;
  *n_out = nu;
  if (nu > cap) return SCD_ERR_BUFFER_TOO_SMALL;
  if (nu > 0 &&
      (cudaMemcpyAsync(host_out, B.span.p, sizeof(scd_span) * (size_t)nu, cudaMemcpyDeviceToHost,
                       st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    return SCD_ERR_CUDA;
  return SCD_OK;
}

extern "C" SCD_API int scd_refine_trace(scd_scene *s, double eps_s, float *lo4, float *hi4,
                                        uint32_t *obj, int64_t cap, int64_t *n_out,
                                        int64_t *round_boxes, int *rounds) {
  if (!s || !n_out || cap < 0 || (cap > 0 && (!lo4 || !hi4 || !obj))) return SCD_ERR_INVALID_ARG;
  if (int rc = rf_check_scene(s)) return rc;
  int nr = 0, L = -1;  // discrete rounds: nr from the first intervals
  if (eps_s > 0.0) {
    const double T_s = (double)s->T * s->tick_s;
    L = 0;
    while (L <= kRfMaxLevels && ldexp(T_s, -L) > eps_s) ++L;
    if (L > kRfMaxLevels) return SCD_ERR_CAPACITY;
  }
  cudaStream_t st = s->stream;
  RfBuffers B(st);
  B.tcap = std::max<int64_t>(cap, 1);
  if (!B.tlo.ensure((size_t)B.tcap, st) || !B.thi.ensure((size_t)B.tcap, st) ||
      !B.tobj.ensure((size_t)B.tcap, st))
    return SCD_ERR_OOM;
  unsigned long long h[RF_WORDS], rc_[kRfMaxRounds];
  int rc = rf_run(s, B, nullptr, nr, L, h, rc_);
  if (rc != SCD_OK) return rc;
  const int nrounds = L >= 0 ? L + 1 : nr;
  int r = 0;
  int64_t total = 0;
  while (r < nrounds && rc_[r] > 0) {
    if (round_boxes) round_boxes[r] = (int64_t)rc_[r];
    total += (int64_t)rc_[r];
    ++r;
  }
  if (rounds) *rounds = r;
  if (h[RF_ERR]) return SCD_ERR_KEPLER_NOCONV;
  *n_out = total;
  if (total > cap) return SCD_ERR_BUFFER_TOO_SMALL;
  if (total > 0 &&
      (cudaMemcpyAsync(lo4, B.tlo.p, sizeof(float4) * (size_t)total, cudaMemcpyDeviceToHost, st) !=
           cudaSuccess ||
       cudaMemcpyAsync(hi4, B.thi.p, sizeof(float4) * (size_t)total, cudaMemcpyDeviceToHost, st) !=
           cudaSuccess ||
       cudaMemcpyAsync(obj, B.tobj.p, sizeof(uint32_t) * (size_t)total, cudaMemcpyDeviceToHost,
                       st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    return SCD_ERR_CUDA;
  return SCD_OK;
}
