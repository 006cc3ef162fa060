// traverse.cu -- step A8: every box queries the hierarchy for the boxes it
// meets (the tree query of Sec. 3.2, run for all boxes at once) and the
// candidate records are emitted; step A9: the canonical list.
//
// Each box pair is found once: box p only visits subtrees whose rightmost
// leaf lies after its own leaf, and inside its own leaf only later boxes.
//
// Merged output without sorting the raw set: for one object pair the tick
// intersections of their overlapping box pairs ("cells") are disjoint and
// tile the horizon in order, so a merged interval is a maximal run of
// consecutive overlapping cells.  Every hit looks at the cell just before it
// (one segment back on whichever object's segment begins at the cell's first
// tick) and the cell just after it (one segment forward on whichever ends at
// its last tick).  A run's first cell emits a start record; if that cell is
// also the run's last, the record is "closed" and carries the last tick,
// else it is "open" and the run's last cell emits an end record.  After the
// starts and the ends are sorted by (i, j, tick), the k-th open start pairs
// with the k-th end.  The last tick is packed below the start's key when
// 2 (object bits + tick bits) <= 64 and an all-ones tick field cannot be a
// tick (the open tag), else it travels as a 32-bit sort value.
#include <algorithm>
#include <type_traits>

#include "scd_internal.cuh"

namespace scd {

struct TravArgs {
  const TravNode *nodes;
  const QBox *qbox;           // compact nodes (one box per leaf)
  const uint32_t *qlink;      // their split gamma with the two leaf flags
  const W4Node *w4;           // four-wide nodes (one box per leaf, node width 4)
  const SBox *sbox;           // sorted boxes
  const uint32_t *sobj, *sid; // object and unsorted id of each sorted box
  const int2 *nb;             // sorted positions of the previous / next segment
  const float4 *lo, *hi;      // unsorted boxes (object-major)
  int64_t N;
  int L;
  int64_t M;
  int T;
  int raw;
  int obj_bits, t_bits;
  int packed;                 // run starts carry their last tick in the low t_bits
  uint32_t open_tag;          // last tick of an open run start
  unsigned long long *starts, *ends;
  uint32_t *rawval;           // raw cells' (or unpacked run starts') last tick
  unsigned long long cap;
  DevCounters *ctr;
  // static decomposition (kind SCD_DECOMP_NONE: one tree, root 0)
  int dkind;
  int n_slabs, p_bands;
  const uint32_t *scell;     // cell of each sorted reference
  const int32_t *cellroot;   // root node of each cell's subtree (-1: none)
  const double2 *rr;         // radial ranges (ALT_BANDS)
  const double *edges;       // band edges (ALT_BANDS)
  const int32_t *objT;       // per-object horizon (a batch of scenes), or null
  // refinement rounds (kRefine): the box count on the device (N is the
  // capacity), a flag word per interval (indexed by unsorted id) and the
  // round's candidates (tick candidates, or spans at the finest level of
  // the continuous variant)
  const unsigned long long *d_N;
  uint32_t *rflags;
  unsigned long long *rcand, *rncand;
  unsigned long long rcap;
  int rspans;
};

// Is `cell` the one cell that reports the overlapping pair (q, b)?  The
// lower corner of the boxes' intersection (SLAB_OCT), or the lower end of
// the two objects' common radial range (ALT_BANDS, which also drops pairs
// with no potential-collision edge).
__device__ __forceinline__ bool reports_here(const TravArgs &a, uint32_t cell, float4 ql, float4 bl,
                                             uint32_t qo, uint32_t bo) {
  if (a.dkind == SCD_DECOMP_SLAB_OCT) {
    float cx = fmaxf(ql.x, bl.x), cy = fmaxf(ql.y, bl.y), cz = fmaxf(ql.z, bl.z);
    int64_t ct = (int64_t)fmaxf(ql.w, bl.w);
    uint32_t c = (uint32_t)(slab_of(ct, a.n_slabs, a.T) * 8 + ((cx >= 0.f) << 2) +
                            ((cy >= 0.f) << 1) + (cz >= 0.f));
    return c == cell;
  }
  if (a.dkind == SCD_DECOMP_ALT_BANDS) {
    double2 r1 = a.rr[qo], r2 = a.rr[bo];
    double lo = fmax(r1.x, r2.x), hi = fmin(r1.y, r2.y);
    return lo <= hi && (uint32_t)band_of(lo, a.edges, a.p_bands) == cell;
  }
  return true;
}

// a slot that holds no record: all key bits set, so it sorts after every
// real record (whose object fields can never be all ones)
constexpr unsigned long long kHole = ~0ull;

// One record per predicate-true lane, each with its own atomic slot range
// (used by the one-thread-per-box traversal, whose lanes are not in step).
struct DirectEmit {
  __device__ __forceinline__ void put(unsigned long long *buf, uint32_t *vbuf,
                                      unsigned long long *slots, unsigned long long *valid,
                                      unsigned long long cap, bool pred, unsigned long long key,
                                      uint32_t v) {
    unsigned mask = __activemask();
    unsigned vote = __ballot_sync(mask, pred);
    if (!pred) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(vote) - 1;
    unsigned long long base = 0;
    if (lane == leader) {
      base = atomicAdd(slots, (unsigned long long)__popc(vote));
      atomicAdd(valid, (unsigned long long)__popc(vote));
    }
    base = __shfl_sync(vote, base, leader);
    unsigned long long idx = base + (unsigned long long)__popc(vote & ((1u << lane) - 1u));
    if (idx < cap) {
      buf[idx] = key;
      if (vbuf) vbuf[idx] = v;
    }
  }
};

// Whole-warp emission into a chunk of slots reserved by the warp (one atomic
// per kChunk records).  A chunk's unused tail is filled with holes.  Every
// lane of the warp calls put() together; the chunk state is warp-uniform.
constexpr unsigned kChunk = 512;
struct ChunkCursor {
  unsigned long long next = 0, end = 0, count = 0;
};

__device__ __forceinline__ void chunk_fill_holes(ChunkCursor &c, unsigned long long *buf,
                                                 unsigned long long cap) {
  const int lane = threadIdx.x & 31;
  for (unsigned long long k = c.next + lane; k < c.end; k += 32)
    if (k < cap) buf[k] = kHole;
  c.next = c.end;
}

__device__ __forceinline__ void chunk_put(ChunkCursor &c, unsigned long long *buf, uint32_t *vbuf,
                                          unsigned long long *slots, unsigned long long cap,
                                          bool pred, unsigned long long key, uint32_t v) {
  const int lane = threadIdx.x & 31;
  unsigned vote = __ballot_sync(0xffffffffu, pred);
  unsigned cnt = __popc(vote);
  if (cnt == 0) return;
  if (c.next + cnt > c.end) {
    chunk_fill_holes(c, buf, cap);
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(slots, (unsigned long long)kChunk);
    b = __shfl_sync(0xffffffffu, b, 0);
    c.next = b;
    c.end = b + kChunk;
  }
  if (pred) {
    unsigned long long idx = c.next + __popc(vote & ((1u << lane) - 1u));
    if (idx < cap) {
      buf[idx] = key;
      if (vbuf) vbuf[idx] = v;
    }
  }
  c.next += cnt;
  c.count += cnt;
}

struct Query {
  float4 lo, hi;
  uint32_t obj, uid;
};

// Is (q, b) the first / last cell of its run?  Both need the neighbouring
// cell: one segment back (forward) on whichever box starts (ends) there.
__device__ __forceinline__ void run_ends(const TravArgs &a, const Query &q, float4 bl, float4 bh,
                                         uint32_t bu, int s, int e, int T, bool &start,
                                         bool &end) {
  int qt0 = (int)q.lo.w, qt1 = (int)q.hi.w, bt0 = (int)bl.w, bt1 = (int)bh.w;
  if (start && s > 0) {
    float4 ql = q.lo, qh = q.hi, cl = bl, ch = bh;
    if (qt0 == s) { ql = __ldg(a.lo + q.uid - 1); qh = __ldg(a.hi + q.uid - 1); }
    if (bt0 == s) { cl = __ldg(a.lo + bu - 1); ch = __ldg(a.hi + bu - 1); }
    start = !box_overlap(ql, qh, cl, ch);
  }
  if (end && e < T) {
    float4 ql = q.lo, qh = q.hi, cl = bl, ch = bh;
    if (qt1 == e) { ql = __ldg(a.lo + q.uid + 1); qh = __ldg(a.hi + q.uid + 1); }
    if (bt1 == e) { cl = __ldg(a.lo + bu + 1); ch = __ldg(a.hi + bu + 1); }
    end = !box_overlap(ql, qh, cl, ch);
  }
}

// The same test with the neighbouring segments found by sorted position
// (they lie close to the pair in the Morton order, so the loads hit cache).
__device__ __forceinline__ void run_ends_sorted(const TravArgs &a, float4 ql0, float4 qh0,
                                                int2 qn, float4 bl, float4 bh, int2 bn, int s,
                                                int e, int T, bool &start, bool &end) {
  int qt0 = (int)ql0.w, qt1 = (int)qh0.w, bt0 = (int)bl.w, bt1 = (int)bh.w;
  if (start && s > 0) {
    float4 ql = ql0, qh = qh0, cl = bl, ch = bh;
    if (qt0 == s) ldg_box(a.sbox + qn.x, ql, qh);
    if (bt0 == s) ldg_box(a.sbox + bn.x, cl, ch);
    start = !box_overlap(ql, qh, cl, ch);
  }
  if (end && e < T) {
    float4 ql = ql0, qh = qh0, cl = bl, ch = bh;
    if (qt1 == e) ldg_box(a.sbox + qn.y, ql, qh);
    if (bt1 == e) ldg_box(a.sbox + bn.y, cl, ch);
    end = !box_overlap(ql, qh, cl, ch);
  }
}

__device__ __forceinline__ unsigned long long pair_key(const TravArgs &a, uint32_t oa,
                                                       uint32_t ob) {
  unsigned long long i = min(oa, ob), j = max(oa, ob);
  return (i << (a.obj_bits + a.t_bits)) | (j << a.t_bits);
}

// A start record: (i, j, first tick), with the run's last tick (or the open
// tag) packed below it; `last` is also the sort value when unpacked.
__device__ __forceinline__ unsigned long long start_key(const TravArgs &a, unsigned long long pk,
                                                        int s, uint32_t last) {
  unsigned long long key = pk | (unsigned long long)s;
  return a.packed ? (key << a.t_bits) | (unsigned long long)last : key;
}

// ---------------------------------------------------------------------------
// One thread per box, for leaves of several boxes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void on_candidate(const TravArgs &a, const Query &q, int64_t pb,
                                             unsigned long long &leaf_tests) {
  float4 bl, bh;
  ldg_box(a.sbox + pb, bl, bh);
  ++leaf_tests;
  if (!box_overlap(q.lo, q.hi, bl, bh)) return;
  uint32_t bo = __ldg(a.sobj + pb);
  if (bo == q.obj) return;
  uint32_t bu = __ldg(a.sid + pb);
  int s = max((int)q.lo.w, (int)bl.w), e = min((int)q.hi.w, (int)bh.w);
  unsigned long long pk = pair_key(a, q.obj, bo);
  DirectEmit em;
  if (a.raw) {
    em.put(a.starts, a.rawval, &a.ctr->n_raw, &a.ctr->v_raw, a.cap, true,
           pk | (unsigned long long)s, (uint32_t)e);
    return;
  }
  bool start = true, end = true;
  run_ends(a, q, bl, bh, bu, s, e, a.objT ? __ldg(a.objT + q.obj) : a.T, start, end);
  const uint32_t last = end ? (uint32_t)e : a.open_tag;
  em.put(a.starts, a.packed ? nullptr : a.rawval, &a.ctr->n_starts, &a.ctr->v_starts, a.cap,
         start, start_key(a, pk, s, last), last);
  em.put(a.ends, nullptr, &a.ctr->n_ends, &a.ctr->v_ends, a.cap, end && !start,
         pk | (unsigned long long)e, 0u);
}

__device__ __forceinline__ void visit_leaf(const TravArgs &a, const Query &q, int64_t leaf,
                                           unsigned long long &lt) {
  int64_t b0 = leaf * a.L, b1 = b0 + a.L < a.N ? b0 + a.L : a.N;
  for (int64_t pb = b0; pb < b1; ++pb) on_candidate(a, q, pb, lt);
}

template <int kDepth>
__global__ void __launch_bounds__(256) k_traverse(TravArgs a) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long nt = 0, lt = 0;
  if (p < a.N) {
    Query q;
    ldg_box(a.sbox + p, q.lo, q.hi);
    q.obj = __ldg(a.sobj + p);
    q.uid = __ldg(a.sid + p);
    int64_t c = p / a.L;
    int64_t e1 = (c + 1) * a.L < a.N ? (c + 1) * a.L : a.N;
    for (int64_t pb = p + 1; pb < e1; ++pb) on_candidate(a, q, pb, lt);
    if (a.M > 1) {
      int32_t stack[kDepth];
      int sp = 0;
      int32_t node = 0;
      for (;;) {
        const float4 *np = reinterpret_cast<const float4 *>(a.nodes + node);
        float4 lol = __ldg(np + 0), hil = __ldg(np + 1), lor = __ldg(np + 2), hir = __ldg(np + 3);
        int4 lk = __ldg(reinterpret_cast<const int4 *>(np + 4));
        nt += 2;
        bool gl = lk.z > c && box_overlap(q.lo, q.hi, lol, hil);
        bool gr = lk.w > c && box_overlap(q.lo, q.hi, lor, hir);
        if (gl && (lk.x & kLeafBit)) {
          visit_leaf(a, q, lk.x & ~kLeafBit, lt);
          gl = false;
        }
        if (gr && (lk.y & kLeafBit)) {
          visit_leaf(a, q, lk.y & ~kLeafBit, lt);
          gr = false;
        }
        if (gl && gr) {
          if (sp >= kDepth) {
            atomicOr(&a.ctr->trav_flags, ERR_STACK);
            break;
          }
          stack[sp++] = lk.y;
          node = lk.x;
        } else if (gl) {
          node = lk.x;
        } else if (gr) {
          node = lk.y;
        } else {
          if (sp == 0) break;
          node = stack[--sp];
        }
      }
    }
  }
  // one atomic per warp for the test counters
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nt += __shfl_down_sync(0xffffffffu, nt, o);
    lt += __shfl_down_sync(0xffffffffu, lt, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&a.ctr->node_tests, nt);
    atomicAdd(&a.ctr->leaf_tests, lt);
  }
}

// ---------------------------------------------------------------------------
// Persistent traversal for one box per leaf.  Every loop iteration of every
// lane is the same step (load one compact node, test its two child boxes), so
// lanes stay in lock step; a lane whose query is done takes the next one from
// a pool its warp claims in blocks; overlapping box pairs go to a per-warp
// buffer and their records are worked out by the whole warp together, into
// output chunks the warp reserves kChunk slots at a time.
// ---------------------------------------------------------------------------
// block shape: 64, 128 and 256 threads (with 16, 8 and 4 resident blocks)
// measured the same on the 24 h catalog screen (21.9, 21.9, 22.0 ms)
constexpr int kT2Threads = 128;
constexpr int kT2Warps = kT2Threads / 32;
// candidate pairs buffered per warp, drained when fewer than one step's
// worth (128) of slots remain: fewer, longer drains.  Measured on the 24 h
// catalog screen: 256 18.70 ms, 384 18.39, 448 18.32, 512 18.56 (a larger
// shared-memory carve-out takes L1), 768 34.9 (fewer resident blocks)
constexpr int kHitCap = 448;
// queries claimed per warp atomic; small, so that the queries in flight stay
// a narrow window of the Morton order and their nodes stay in L2
// (64 per claim: +4% traversal time, 128: +17%)
constexpr unsigned kQueryChunk = 32;
// a refill can hand out up to 32 queries at once, from the pool's rest and
// one new chunk: a chunk smaller than a warp would leave lanes without one
static_assert(kQueryChunk >= 32, "a query chunk covers at least one warp's refill");

struct WarpEmit {
  ChunkCursor s, e;  // start and end record chunks (raw cells use s)
};

// A refinement round's hits: both intervals of a pair of meeting boxes of
// different objects are flagged; two single ticks that meet (the same tick)
// are a tick candidate, and at the finest level of the continuous variant
// every meeting pair is a span.
__device__ __forceinline__ void drain_round_hits(const TravArgs &a, const uint2 *buf, int cnt) {
  const int lane = threadIdx.x & 31;
  for (int k = lane; k < cnt; k += 32) {
    const uint2 h = buf[k];
    float4 ql, qh, bl, bh;
    ldg_box(a.sbox + h.x, ql, qh);
    ldg_box(a.sbox + h.y, bl, bh);
    const uint32_t qo = __ldg(a.sobj + h.x), bo = __ldg(a.sobj + h.y);
    if (bo == qo || !box_overlap(ql, qh, bl, bh)) continue;
    const bool longq = qh.w > ql.w, longb = bh.w > bl.w;
    atomicOr(a.rflags + __ldg(a.sid + h.x), kRfHit | (longb ? kRfHitLong : 0u));
    atomicOr(a.rflags + __ldg(a.sid + h.y), kRfHit | (longq ? kRfHitLong : 0u));
    unsigned long long key;
    if (a.rspans) {
      key = rf_span_key(min(qo, bo), max(qo, bo), (int32_t)ql.w, (int32_t)bl.w);
    } else if (!longq && !longb) {
      key = rf_tick_key((uint32_t)ql.w, min(qo, bo), max(qo, bo));
    } else {
      continue;
    }
    const unsigned long long q = atomicAdd(a.rncand, 1ull);
    if (q < a.rcap) a.rcand[q] = key;
  }
}

__device__ __forceinline__ void drain_hits(const TravArgs &a, const uint2 *buf, int cnt,
                                           WarpEmit &we) {
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < cnt; base += 32) {
    int k = base + lane;
    bool valid = k < cnt;
    float4 ql = make_float4(0.f, 0.f, 0.f, 0.f), qh = ql, bl = ql, bh = ql;
    uint32_t qo = 0, bo = 0;
    uint2 h = make_uint2(0u, 0u);
    if (valid) {
      h = buf[k];
      ldg_box(a.sbox + h.x, ql, qh);
      qo = __ldg(a.sobj + h.x);
      ldg_box(a.sbox + h.y, bl, bh);
      bo = __ldg(a.sobj + h.y);
      // the tree test was on quantised boxes: decide on the exact ones
      valid = bo != qo && box_overlap(ql, qh, bl, bh);
      if (valid && a.dkind != SCD_DECOMP_NONE)
        valid = reports_here(a, __ldg(a.scell + h.x), ql, bl, qo, bo);
    }
    int s = max((int)ql.w, (int)bl.w), e = min((int)qh.w, (int)bh.w);
    unsigned long long pk = pair_key(a, qo, bo);
    if (a.raw) {
      chunk_put(we.s, a.starts, a.rawval, &a.ctr->n_raw, a.cap, valid,
                pk | (unsigned long long)s, (uint32_t)e);
      continue;
    }
    bool start = valid, end = valid;
    if (valid)
      run_ends_sorted(a, ql, qh, __ldg(a.nb + h.x), bl, bh, __ldg(a.nb + h.y), s, e,
                      a.objT ? __ldg(a.objT + qo) : a.T, start, end);
    const uint32_t last = end ? (uint32_t)e : a.open_tag;
    chunk_put(we.s, a.starts, a.packed ? nullptr : a.rawval, &a.ctr->n_starts, a.cap, start,
              start_key(a, pk, s, last), last);
    chunk_put(we.e, a.ends, nullptr, &a.ctr->n_ends, a.cap, end && !start,
              pk | (unsigned long long)e, 0u);
  }
}

// One node's two children against the quantised query: the child nodes to
// descend into (gl, gr) and the leaf children that are candidates (hl, hr).
// Only subtrees with a leaf after the query's own leaf p are of interest.
// The left child's rightmost leaf is the split gamma, so it needs the test
// gamma > p.  The right child needs none: every node a query visits either
// holds p or lies wholly after it (the root holds p; a child of a node that
// holds p either holds p or, being right of the split, lies after it, or
// being left of it, is kept only when gamma > p; children of a node wholly
// after p are wholly after p), so the right child always ends after p
// unless it holds p as its last leaf.  That one case costs a descent along
// the subtree's right edge down to p itself, whose pair with itself the
// exact test drops (same object).
__device__ __forceinline__ void test_children(const TravArgs &a, const QBox &q, int64_t p,
                                              int32_t node, bool &gl, bool &gr, bool &hl,
                                              bool &hr, int32_t &cl) {
  uint4 bl, br;
  ldg_qbox_pair(a.qbox + 2 * (int64_t)node, bl, br);
  const uint32_t lk = __ldg(a.qlink + node);
  const uint32_t g = lk & kQIndex;
  cl = (int32_t)g;
  // child lo <= query hi and query lo <= child hi: x, y per 16-bit lane,
  // then the z and tick fields
  const uint32_t ml = __vcmpleu2(bl.x, q.hi_xy) & __vcmpleu2(q.lo_xy, bl.z);
  const uint32_t mr = __vcmpleu2(br.x, q.hi_xy) & __vcmpleu2(q.lo_xy, br.z);
  gl = (int64_t)g > p && ml == 0xffffffffu && zt_le(bl.y, q.hi_zt) && zt_le(q.lo_zt, bl.w);
  gr = mr == 0xffffffffu && zt_le(br.y, q.hi_zt) && zt_le(q.lo_zt, br.w);
  hl = gl && (lk & kQLeftLeaf);
  hr = gr && (lk & kQRightLeaf);
  gl &= !hl;
  gr &= !hr;
}

// one slot of a four-wide node: it meets the quantised query and its
// rightmost leaf lies after the query's own leaf (empty slots: leaf 0)
__device__ __forceinline__ bool w4_slot(const QBox &q, int64_t p, const uint4 &b, uint32_t last) {
  return (int64_t)last > p &&
         (__vcmpleu2(b.x, q.hi_xy) & __vcmpleu2(q.lo_xy, b.z)) == 0xffffffffu &&
         zt_le(b.y, q.hi_zt) && zt_le(q.lo_zt, b.w);
}

// kTwo: two binary nodes per lane and step; kW4: four-wide nodes.  The
// lanes' stacks stay in local memory: a stack in shared memory (entry-major,
// free of bank conflicts) was measured 1.7x slower, because the shared
// memory it takes comes out of the L1 cache that the node loads rely on.
// 8 resident blocks of 128 threads: 64 registers and a few bytes of spills;
// 9 or 10 blocks (56 or 48 registers) spill 112-280 bytes and measured
// 12% and 41% slower
template <int kDepth, bool kTwo, bool kW4, bool kRefine = false>
__global__ void __launch_bounds__(kT2Threads, 8) k_traverse2(TravArgs a) {
  __shared__ uint2 hits[kT2Warps][kHitCap];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  uint2 *buf = hits[w];
  int nhit = 0;  // warp-uniform
  unsigned long long nt = 0, ntests = 0;
  int64_t p = -1;  // current query (sorted position), -1 = none
  bool exhausted = false;
  // the last box has no later partner: queries are 0 .. N-2
  const int64_t nbox = kRefine && a.d_N && *a.d_N < (unsigned long long)a.N ? (int64_t)*a.d_N
                                                                            : a.N;
  const unsigned long long nq = nbox > 1 ? (unsigned long long)(nbox - 1) : 0ull;
  unsigned long long q_next = 0, q_end = 0;  // the warp's query pool
  WarpEmit we;
  const QFrame fr = scene_frame(a.ctr, a.T);
  QBox q = {0u, 0u, 0u, 0u};  // the query box, quantised outward like the nodes
  int32_t stack[kDepth];
  int sp = 0, sb = 0;  // the lane's deferred subtrees are stack[sb .. sp)
  int32_t node = 0;
  int32_t node2 = -1;  // a second node visited in the same step (kTwo)
  for (;;) {
    // lanes without a query take the next ones from the warp's pool
    unsigned need = __ballot_sync(0xffffffffu, p < 0 && !exhausted);
    if (need) {
      unsigned cnt = __popc(need);
      unsigned long long have = q_end - q_next;
      unsigned long long nb = 0;
      if (have < cnt) {
        if (lane == 0) nb = atomicAdd(&a.ctr->work_next, (unsigned long long)kQueryChunk);
        nb = __shfl_sync(0xffffffffu, nb, 0);
      }
      if (need & (1u << lane)) {
        unsigned r = __popc(need & lt);
        unsigned long long mine = r < have ? q_next + r : nb + (r - have);
        if (mine < nq) {
          p = (int64_t)mine;
          float4 plo, phi;
          ldg_box(a.sbox + p, plo, phi);
          q = quantize_box(fr, plo, phi);
          // the query starts at the root of its own cell's subtree
          node = a.dkind == SCD_DECOMP_NONE ? 0 : __ldg(a.cellroot + __ldg(a.scell + p));
          node2 = -1;
          sp = sb = 0;
          if (node < 0) p = -1;  // alone in its cell: nothing to find
        } else {
          exhausted = true;
        }
      }
      if (have < cnt) {
        q_next = nb + (cnt - have);
        q_end = nb + kQueryChunk;
      } else {
        q_next += cnt;
      }
    }
    // Once the queue is empty, a lane without a query takes the oldest
    // deferred subtree (the largest) of a lane that has one, with its query:
    // one long query then spreads over the warp instead of holding it.
    if (__ballot_sync(0xffffffffu, exhausted)) {
      const unsigned idle = __ballot_sync(0xffffffffu, p < 0);
      const unsigned donors = __ballot_sync(0xffffffffu, p >= 0 && sp > sb);
      const int moves = min(__popc(idle), __popc(donors));
      if (moves > 0) {
        const bool is_idle = (idle >> lane) & 1u, is_donor = (donors >> lane) & 1u;
        const int ri = __popc(idle & lt), rd = __popc(donors & lt);
        const int32_t give = is_donor ? stack[sb] : 0;
        // the receiver of rank k takes from the donor of rank k
        int src = lane;
        if (is_idle && ri < moves) {
          unsigned m = donors;
          for (int k = 0; k < ri; ++k) m &= m - 1u;
          src = __ffs(m) - 1;
        }
        const int32_t gnode = __shfl_sync(0xffffffffu, give, src);
        const uint32_t gp = __shfl_sync(0xffffffffu, (uint32_t)p, src);
        QBox gq;
        gq.lo_xy = __shfl_sync(0xffffffffu, q.lo_xy, src);
        gq.lo_zt = __shfl_sync(0xffffffffu, q.lo_zt, src);
        gq.hi_xy = __shfl_sync(0xffffffffu, q.hi_xy, src);
        gq.hi_zt = __shfl_sync(0xffffffffu, q.hi_zt, src);
        if (is_idle && ri < moves) {
          p = (int64_t)gp;
          q = gq;
          node = gnode;
          node2 = -1;
          sp = sb = 0;
        }
        if (is_donor && rd < moves) ++sb;
      }
    }
    bool active = p >= 0;
    if (__ballot_sync(0xffffffffu, active) == 0) break;
    const uint32_t pq = (uint32_t)p;  // this step's query, before p may end
    bool hl = false, hr = false, hl2 = false, hr2 = false;
    int32_t cl = 0, cl2 = 0;
    // the subtrees to visit next: the first one (two) are this lane's next
    // node(s), the rest go on the stack
    int32_t first = -1, second = -1;
    bool overflow = false;
    auto take = [&](bool go, int32_t c) {
      if (!go) return;
      if (first < 0) {
        first = c;
      } else if (kTwo && second < 0) {
        second = c;
      } else if (sp < kDepth) {
        stack[sp++] = c;
      } else {
        overflow = true;
      }
    };
    // four-wide: the leaf slots that pass, with their leaf indices
    bool h4[4] = {false, false, false, false};
    uint32_t c4[4] = {0u, 0u, 0u, 0u};
    if (active) {
      if constexpr (kW4) {
        const W4Node *nd = a.w4 + node;
        uint4 b0, b1, b2, b3, la, lb;
        ldg_qbox_pair(nd->box, b0, b1);
        ldg_qbox_pair(nd->box + 2, b2, b3);
        ldg_w4_links(nd->link, la, lb);
        nt += 4;
        const uint32_t lx[4] = {la.x, la.z, lb.x, lb.z};
        const bool ok[4] = {w4_slot(q, p, b0, la.y), w4_slot(q, p, b1, la.w),
                            w4_slot(q, p, b2, lb.y), w4_slot(q, p, b3, lb.w)};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const bool leaf = (lx[k] & kW4Leaf) != 0u;
          h4[k] = ok[k] && leaf;
          c4[k] = lx[k] & kW4Index;
          take(ok[k] && !leaf, (int32_t)c4[k]);
        }
      } else {
        if (kTwo && node2 < 0 && sp > sb) node2 = stack[--sp];
        bool gl, gr, gl2 = false, gr2 = false;
        test_children(a, q, p, node, gl, gr, hl, hr, cl);
        if (kTwo && node2 >= 0) {
          test_children(a, q, p, node2, gl2, gr2, hl2, hr2, cl2);
          nt += 2;
        }
        nt += 2;
        take(gl, cl);
        take(gr, cl + 1);
        if (kTwo) {
          take(gl2, cl2);
          take(gr2, cl2 + 1);
        }
      }
      if (overflow) {
        atomicOr(&a.ctr->trav_flags, ERR_STACK);
        p = -1;
      } else if (first >= 0) {
        node = first;
        node2 = second;
      } else if (sp > sb) {
        node = stack[--sp];
        node2 = -1;
      } else {
        p = -1;  // query (or the subtree taken from another lane) done
      }
    }
    // append this step's hits to the warp buffer
    auto append = [&](bool h, int32_t c) {
      unsigned v = __ballot_sync(0xffffffffu, h);
      if (h) buf[nhit + __popc(v & lt)] = make_uint2(pq, (uint32_t)c);
      nhit += __popc(v);
    };
    if constexpr (kW4) {
#pragma unroll
      for (int k = 0; k < 4; ++k) append(h4[k], (int32_t)c4[k]);
    } else {
      append(hl, cl);
      append(hr, cl + 1);
      if (kTwo) {
        append(hl2, cl2);
        append(hr2, cl2 + 1);
      }
    }
    __syncwarp();
    if (nhit > kHitCap - (kTwo || kW4 ? 128 : 64)) {
      if constexpr (kRefine) drain_round_hits(a, buf, nhit);
      else drain_hits(a, buf, nhit, we);
      __syncwarp();
      ntests += nhit;  // exact box tests, counted once per warp
      nhit = 0;
    }
  }
  __syncwarp();
  if constexpr (kRefine) {
    if (nhit > 0) drain_round_hits(a, buf, nhit);
  } else {
    if (nhit > 0) drain_hits(a, buf, nhit, we);
    chunk_fill_holes(we.s, a.starts, a.cap);
    if (!a.raw) chunk_fill_holes(we.e, a.ends, a.cap);
  }
  ntests += nhit;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nt += __shfl_down_sync(0xffffffffu, nt, o);
  if (lane == 0) {
    atomicAdd(&a.ctr->node_tests, nt);
    atomicAdd(&a.ctr->leaf_tests, ntests);
    if (kRefine) {
    } else if (a.raw) {
      atomicAdd(&a.ctr->v_raw, we.s.count);
    } else {
      atomicAdd(&a.ctr->v_starts, we.s.count);
      atomicAdd(&a.ctr->v_ends, we.e.count);
    }
  }
}

// persistent: as many blocks as fit on the GPU at once
template <int kDepth, bool kTwo, bool kW4>
static void launch_t2(const TravArgs &a, int sms, cudaStream_t st) {
  static int per_sm = 0;
  if (!per_sm)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traverse2<kDepth, kTwo, kW4>,
                                                  kT2Threads, 0);
  k_traverse2<kDepth, kTwo, kW4><<<(unsigned)(sms * std::max(per_sm, 1)), kT2Threads, 0, st>>>(
      a);
}

// One refinement round's traversal over up to cap sorted boxes (their count
// on the device): one box per leaf, binary nodes, two nodes per step.
int traverse_round(const QBox *qbox, const uint32_t *qlink, const SBox *sbox,
                   const uint32_t *sobj, const uint32_t *sid, int64_t cap,
                   const unsigned long long *d_N, int64_t T, DevCounters *ctr, uint32_t *rflags,
                   unsigned long long *rcand, unsigned long long *rncand, unsigned long long rcap,
                   int spans, int deep, cudaStream_t st) {
  if (cap < 2) return SCD_OK;
  if ((reinterpret_cast<uintptr_t>(sbox) | reinterpret_cast<uintptr_t>(qbox)) & 31)
    return SCD_ERR_INTERNAL;
  TravArgs a{};
  a.qbox = qbox;
  a.qlink = qlink;
  a.sbox = sbox;
  a.sobj = sobj;
  a.sid = sid;
  a.N = cap;
  a.L = 1;
  a.T = (int)T;
  a.ctr = ctr;
  a.dkind = SCD_DECOMP_NONE;
  a.d_N = d_N;
  a.rflags = rflags;
  a.rcand = rcand;
  a.rncand = rncand;
  a.rcap = rcap;
  a.rspans = spans;
  static int sms = 0, per64 = 0, per128 = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per64, k_traverse2<64, true, false, true>,
                                                  kT2Threads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per128, k_traverse2<128, true, false, true>,
                                                  kT2Threads, 0);
  }
  if (deep)
    k_traverse2<128, true, false, true>
        <<<(unsigned)(sms * std::max(per128, 1)), kT2Threads, 0, st>>>(a);
  else
    k_traverse2<64, true, false, true>
        <<<(unsigned)(sms * std::max(per64, 1)), kT2Threads, 0, st>>>(a);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

int traverse(scd_scene *s, int64_t n_leaves, int raw_mode, int obj_bits, int t_bits) {
  TravArgs a{};
  a.nodes = s->d_nodes.p;
  a.qbox = s->d_qbox.p;
  a.qlink = s->d_qlink.p;
  a.w4 = s->d_w4.p;
  a.sbox = s->s_box.p;
  a.sobj = s->s_obj.p;
  a.nb = s->s_nb.p;
  a.sid = s->d_id.p;
  a.lo = s->d_lo.p;
  a.hi = s->d_hi.p;
  a.N = s->N;
  a.L = s->tune.leaf_size;
  a.M = n_leaves;
  a.T = (int)s->T;
  a.raw = raw_mode;
  a.obj_bits = obj_bits;
  a.t_bits = t_bits;
  a.packed = !raw_mode && runs_packed(obj_bits, t_bits, s->T);
  a.open_tag = open_tag(a.packed, t_bits);
  a.starts = s->d_starts.p;
  a.ends = s->d_ends.p;
  a.rawval = s->d_rawval.p;
  a.cap = (unsigned long long)s->pair_cap;
  a.ctr = s->d_ctr.p;
  a.dkind = s->dkind;
  a.n_slabs = s->n_slabs;
  a.p_bands = s->p_bands;
  a.scell = s->s_cell.p;
  a.cellroot = s->d_cellroot.p;
  a.rr = s->d_rr.p;
  a.edges = s->d_edges.p;
  a.objT = s->n_scenes > 0 ? s->d_objT.p : nullptr;
  if (a.dkind != SCD_DECOMP_NONE) a.N = s->n_refs;  // one query per reference
  // sorted boxes (and node pairs) are read with 32-byte loads
  if (reinterpret_cast<uintptr_t>(a.sbox) & 31) return SCD_ERR_INTERNAL;
  if (a.L == 1) {
    if (reinterpret_cast<uintptr_t>(a.qbox) & 31) return SCD_ERR_INTERNAL;
    // persistent: as many blocks as fit on the GPU at once
    static int sms = 0;
    if (!sms) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    const bool two = s->tune.nodes_per_step == 2, w4 = s->tune.node_width == 4;
    if (w4 && (reinterpret_cast<uintptr_t>(a.w4) & 127)) return SCD_ERR_INTERNAL;
    auto go = [&](auto depth) {
      constexpr int D = decltype(depth)::value;
      if (w4) launch_t2<D, false, true>(a, sms, s->stream);
      else if (two) launch_t2<D, true, false>(a, sms, s->stream);
      else launch_t2<D, false, false>(a, sms, s->stream);
    };
    switch (s->tune.stack_depth) {
      case 32: go(std::integral_constant<int, 32>()); break;
      case 128: go(std::integral_constant<int, 128>()); break;
      default: go(std::integral_constant<int, 64>()); break;
    }
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
  }
  int bs = s->tune.block_threads;
  if (bs < 32 || bs > 256 || bs % 32) bs = 128;
  int64_t g = (s->N + bs - 1) / bs;
  if (g == 0) return SCD_OK;
  switch (s->tune.stack_depth) {
    case 32: k_traverse<32><<<(unsigned)g, bs, 0, s->stream>>>(a); break;
    case 128: k_traverse<128><<<(unsigned)g, bs, 0, s->stream>>>(a); break;
    default: k_traverse<64><<<(unsigned)g, bs, 0, s->stream>>>(a); break;
  }
  note_launch();
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Step A9: sort the run starts (or the raw cells) and the run ends by
// (i, j, tick), then unpack the starts; the k-th open start takes the k-th
// end.  Holes sort last, so the first n sorted slots are the n records.
// ---------------------------------------------------------------------------
constexpr int kUpThreads = 256, kUpItems = 8, kUpTile = kUpThreads * kUpItems;

struct UnpackArgs {
  const unsigned long long *starts;  // sorted starts (or raw cells)
  const uint32_t *lastv;             // their last ticks when not packed
  const unsigned long long *ends;    // sorted ends of the open runs
  int64_t n;                         // starts to unpack (a capacity when d_n is set)
  const unsigned long long *d_n;     // the count, when known on the device only
  unsigned long long n_ends;         // ends (a capacity when d_ne is set)
  const unsigned long long *d_ne;
  int ob, tb;
  int packed, raw;
  uint32_t open_tag;
  uint32_t *bcnt;                    // per tile: open starts, then their exclusive prefix
  const uint32_t *open_total;
  scd_pair *out;
  DevCounters *ctr;
};

__device__ __forceinline__ int64_t unpack_count(const UnpackArgs &a) {
  return a.d_n && *a.d_n < (unsigned long long)a.n ? (int64_t)*a.d_n : a.n;
}

__device__ __forceinline__ uint32_t last_of(const UnpackArgs &a, unsigned long long key,
                                            int64_t r) {
  return a.packed ? (uint32_t)(key & ((1ull << a.tb) - 1ull)) : __ldg(a.lastv + r);
}

// Tile items are warp-striped: item k of thread t is tile item k * 256 + t,
// so every load and store of a warp is contiguous.

// open starts per tile
__global__ void __launch_bounds__(kUpThreads) k_open_count(UnpackArgs a) {
  const int64_t n = unpack_count(a);
  const int64_t base = (int64_t)blockIdx.x * kUpTile + threadIdx.x;
  uint32_t c = 0;
#pragma unroll
  for (int k = 0; k < kUpItems; ++k) {
    int64_t r = base + (int64_t)k * kUpThreads;
    if (r < n) c += last_of(a, __ldg(a.starts + r), r) == a.open_tag;
  }
  __shared__ uint32_t ws[kUpThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int q = 0; q < kUpThreads / 32; ++q) t += ws[q];
    a.bcnt[blockIdx.x] = t;
  }
}

static_assert(kUpItems * (kUpThreads / 32) == 64, "the tile prefix takes two counts per lane");

__global__ void __launch_bounds__(kUpThreads) k_unpack(UnpackArgs a) {
  constexpr int kWarps = kUpThreads / 32;
  const int64_t n = unpack_count(a);
  const int64_t base = (int64_t)blockIdx.x * kUpTile + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const unsigned long long tmask = (1ull << a.tb) - 1ull, omask = (1ull << a.ob) - 1ull;
  unsigned long long key[kUpItems];
  uint32_t last[kUpItems];
  unsigned open[kUpItems];  // the warp's open-start mask per item
  // opens per (item, warp), then their exclusive prefix in tile order
  __shared__ uint32_t pre[kUpItems][kWarps];
#pragma unroll
  for (int k = 0; k < kUpItems; ++k) {
    int64_t r = base + (int64_t)k * kUpThreads;
    key[k] = r < n ? __ldg(a.starts + r) : 0ull;
    last[k] = r < n ? (a.raw ? __ldg(a.lastv + r) : last_of(a, key[k], r)) : 0u;
    open[k] = __ballot_sync(0xffffffffu, !a.raw && r < n && last[k] == a.open_tag);
    if (lane == 0) pre[k][w] = __popc(open[k]);
  }
  __syncthreads();
  if (w == 0) {
    // kUpItems * kWarps = 64 counts, two per lane, scanned in (item, warp) order
    uint32_t c0 = (&pre[0][0])[2 * lane], c1 = (&pre[0][0])[2 * lane + 1];
    uint32_t x = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    uint32_t b = (a.raw ? 0u : a.bcnt[blockIdx.x]) + x - c0 - c1;
    (&pre[0][0])[2 * lane] = b;
    (&pre[0][0])[2 * lane + 1] = b + c0;
  }
  __syncthreads();
  const unsigned long long n_ends = a.d_ne && *a.d_ne < a.n_ends ? *a.d_ne : a.n_ends;
  if (!a.raw && blockIdx.x == 0 && threadIdx.x == 0 && *a.open_total != n_ends)
    atomicOr(&a.ctr->trav_flags, ERR_ZIP);
  bool bad = false;
#pragma unroll
  for (int k = 0; k < kUpItems; ++k) {
    int64_t r = base + (int64_t)k * kUpThreads;
    if (r < n) {
      unsigned long long kk = a.packed ? key[k] >> a.tb : key[k];
      scd_pair p;
      p.i = (uint32_t)(kk >> (a.ob + a.tb));
      p.j = (uint32_t)((kk >> a.tb) & omask);
      p.tlo = (int32_t)(kk & tmask);
      p.thi = (int32_t)last[k];
      if (open[k] & (1u << lane)) {
        unsigned long long rank = pre[k][w] + __popc(open[k] & lt);
        if (rank < n_ends) {
          unsigned long long ek = __ldg(a.ends + rank);
          p.thi = (int32_t)(ek & tmask);
          bad |= (ek >> a.tb) != (kk >> a.tb) || p.thi <= p.tlo;
        } else {
          bad = true;
        }
      }
      a.out[r] = p;
    }
  }
  if (bad) atomicOr(&a.ctr->trav_flags, ERR_ZIP);
}

static UnpackArgs unpack_args(scd_scene *s, int raw_mode, int obj_bits, int t_bits) {
  UnpackArgs a;
  a.starts = s->d_starts.p;
  a.lastv = s->d_rawval.p;
  a.ends = s->d_ends.p;
  a.d_n = nullptr;
  a.d_ne = nullptr;
  a.ob = obj_bits;
  a.tb = t_bits;
  a.raw = raw_mode;
  a.packed = !raw_mode && runs_packed(obj_bits, t_bits, s->T);
  a.open_tag = open_tag(a.packed, t_bits);
  a.out = s->d_out.p;
  a.ctr = s->d_ctr.p;
  return a;
}

static PairEmit pair_emit(scd_scene *s, int obj_bits, int t_bits, const unsigned long long *ends,
                          unsigned long long n_ends, const unsigned long long *d_ne,
                          scd_pair *out, int64_t n, const unsigned long long *d_n) {
  PairEmit pe;
  pe.ob = obj_bits;
  pe.tb = t_bits;
  pe.ends = ends;
  pe.n_ends = n_ends;
  pe.d_ne = d_ne;
  pe.out = out;
  pe.n = n;
  pe.d_n = d_n;
  pe.flags = &s->d_ctr.p->trav_flags;
  return pe;
}

// k_open_count, the prefix over the tiles, k_unpack
static int unpack(scd_scene *s, UnpackArgs a, cudaStream_t st) {
  int64_t tiles = (a.n + kUpTile - 1) / kUpTile;
  if (tiles == 0) return SCD_OK;
  if (!a.raw) {
    if (!s->d_tilecnt.ensure((size_t)tiles + 1, st)) return SCD_ERR_OOM;
    a.bcnt = s->d_tilecnt.p;
    a.open_total = s->d_tilecnt.p + tiles;
    k_open_count<<<(unsigned)tiles, kUpThreads, 0, st>>>(a);
    scan_u32_exclusive(a.bcnt, tiles, s->d_tilecnt.p + tiles, st);
    note_launch(2);
  }
  k_unpack<<<(unsigned)tiles, kUpThreads, 0, st>>>(a);
  note_launch();
  return SCD_OK;
}

// The record sorts skip the lowest w bits of the tick field when that
// saves a whole 8-bit pass (w = the bits of the last, partial digit).  The
// sort is stable, so the records then stand in the order of (i, j, tick >>
// w), each group of equal prefixes in emission order; k_window_fix sorts
// each group by the whole key.  Records are unique (a pair's runs do not
// overlap) and holes are all ones, so the result is the full sort's order.
static int window_bits(int bits, int t_bits) {
  const int passes = (bits + 7) / 8;
  const int w = bits - 8 * (passes - 1);
  return passes >= 2 && w <= t_bits ? w : 0;
}

// Each group of equal key >> shift (in slots [0, n), n a device count when
// d_n is set) sorted by its first slot's thread: insertion sort, the groups
// hold the runs of one pair within 2^w ticks.  Threads of the group's other
// slots see the same prefixes whatever the order, so only first slots sort.
__global__ void __launch_bounds__(256) k_window_fix(unsigned long long *keys, int64_t n,
                                                    const unsigned long long *d_n, int shift) {
  if (d_n && *d_n < (unsigned long long)n) n = (int64_t)*d_n;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const unsigned long long k = keys[p];
  if (k == kHole) return;
  const unsigned long long g = k >> shift;
  if (p > 0 && (keys[p - 1] >> shift) == g) return;
  int64_t q = p + 1;
  while (q < n && (keys[q] >> shift) == g) ++q;
  for (int64_t x = p + 1; x < q; ++x) {
    const unsigned long long v = keys[x];
    int64_t y = x - 1;
    while (y >= p && keys[y] > v) {
      keys[y + 1] = keys[y];
      --y;
    }
    keys[y + 1] = v;
  }
}

static int window_fix(unsigned long long *keys, int64_t n, const unsigned long long *d_n,
                      int shift, cudaStream_t st) {
  if (n < 2) return SCD_OK;
  k_window_fix<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(keys, n, d_n, shift);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

int canonicalize(scd_scene *s, int raw_mode, int obj_bits, int t_bits) {
  cudaStream_t st = s->stream;
  // slots to sort (records plus holes) and records to keep
  int64_t ns = raw_mode ? (int64_t)s->h_ctr.n_raw : (int64_t)s->h_ctr.n_starts;
  int64_t n = raw_mode ? (int64_t)s->h_ctr.v_raw : (int64_t)s->h_ctr.v_starts;
  UnpackArgs a = unpack_args(s, raw_mode, obj_bits, t_bits);
  const int lo = a.packed ? t_bits : 0, bits = 2 * obj_bits + t_bits;
  if (!s->d_out.ensure(n > 0 ? n : 1, st)) return SCD_ERR_OOM;
  a.out = s->d_out.p;
  // packed starts and the ends: one pass fewer, then the window fix-up
  const int w = a.packed && !raw_mode ? window_bits(bits, t_bits) : 0;
  int rc = radix_sort_u64(s->d_starts.p, a.packed ? nullptr : s->d_rawval.p, ns, lo + w,
                          bits + lo, s->sort_sc, st);
  if (rc) return rc;
  if (w && (rc = window_fix(s->d_starts.p, ns, nullptr, lo + w, st))) return rc;
  if (!raw_mode && s->h_ctr.v_ends > 0) {
    rc = radix_sort_u64(s->d_ends.p, nullptr, (int64_t)s->h_ctr.n_ends, w, bits, s->sort_sc, st);
    if (rc) return rc;
    if (w && (rc = window_fix(s->d_ends.p, (int64_t)s->h_ctr.n_ends, nullptr, w, st))) return rc;
  }
  a.n = n;
  a.n_ends = raw_mode ? 0 : s->h_ctr.v_ends;
  if (int rc2 = unpack(s, a, st)) return rc2;
  s->n_out = n;
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

// The canonical list for a host destination, in buckets of the pair's
// first object that go to the host while the next ones are sorted: one
// stable pass over the top digit of the starts' and the ends' keys (the top
// bits of i) splits both into digit ranges (starting 16-byte aligned); runs
// of whole digits with about equal numbers of starts form the buckets, and
// each bucket is sorted by the whole key, unpacked into its place in the
// output and copied out on a second stream (the bucket's last sort pass
// writes the pairs themselves: no unpack pass per bucket; for the whole
// list on the device the separate unpack measured faster).  A pair's starts and ends share
// their i, so each bucket zips its own open starts with its own ends.  The
// output equals canonicalize's; one more pass over the records, hidden
// under the copies.
#define TRY_(x)                   \
  do {                            \
    int rc_ = (x);                \
    if (rc_ != SCD_OK) return rc_; \
  } while (0)

int canonicalize_streamed(scd_scene *s, int obj_bits, int t_bits, scd_pair *host) {
  cudaStream_t st = s->stream;
  UnpackArgs a = unpack_args(s, 0, obj_bits, t_bits);
  const int lo = t_bits, bits = 2 * obj_bits + t_bits;
  // the top digit must lie inside the (i, j) fields, so that a pair's open
  // start and its end (different ticks) fall into the same bucket
  if (!a.packed || 2 * obj_bits < 8) return SCD_ERR_STATE;
  const int64_t ns = (int64_t)s->h_ctr.n_starts, n = (int64_t)s->h_ctr.v_starts;
  const int64_t nes = (int64_t)s->h_ctr.n_ends, ne = (int64_t)s->h_ctr.v_ends;
  if (!s->d_out.ensure(n > 0 ? n : 1, st) || !s->d_part.ensure(ns + 256, st) ||
      !s->d_parte.ensure(nes + 256, st))
    return SCD_ERR_OOM;
  if (!s->cstream) {
    if (cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking) != cudaSuccess)
      return SCD_ERR_CUDA;
    for (int b = 0; b < kStreamBuckets; ++b)
      if (cudaEventCreateWithFlags(&s->cev[b], cudaEventDisableTiming) != cudaSuccess)
        return SCD_ERR_CUDA;
  }
  uint32_t ts[256], te[256];
  TRY_(radix_partition_u64(s->d_starts.p, s->d_part.p, ns, lo + bits - 8, s->sort_sc, ts, st));
  TRY_(radix_partition_u64(s->d_ends.p, s->d_parte.p, nes, bits - 8, s->sort_sc, te, st));
  // digit d's range starts at ps[d] (pe[d]); its records: the keys of the
  // digit, except that the all-ones digit also holds the holes
  int64_t ps[257], pe[257], vs[256], ve[256], sum_s = 0, sum_e = 0;
  ps[0] = pe[0] = 0;
  for (int d = 0; d < 256; ++d) {
    ps[d + 1] = ps[d] + ((ts[d] + 1) & ~1u);
    pe[d + 1] = pe[d] + ((te[d] + 1) & ~1u);
    vs[d] = d < 255 ? ts[d] : n - sum_s;
    ve[d] = d < 255 ? te[d] : ne - sum_e;
    sum_s += vs[d];
    sum_e += ve[d];
  }
  if (vs[255] < 0 || ve[255] < 0 || sum_s != n || sum_e != ne) return SCD_ERR_INTERNAL;
  int64_t out_at = 0;
  int d0 = 0;
  for (int b = 0; b < kStreamBuckets && d0 < 256; ++b) {
    // whole digits up to about an equal share of the starts still left; the
    // first bucket small, so that the copies (the slower stream) start early
    const int64_t share = b == 0 ? (n + 63) / 64
                                 : (n - out_at + (kStreamBuckets - b) - 1) / (kStreamBuckets - b);
    int d1 = d0;
    int64_t m = 0, me = 0;
    while (d1 < 256 && (m < share || b == kStreamBuckets - 1)) {
      m += vs[d1];
      me += ve[d1];
      ++d1;
    }
    const int64_t slots = ps[d1] - ps[d0], eslots = pe[d1] - pe[d0];
    unsigned long long *ks = s->d_part.p + ps[d0], *ke = s->d_parte.p + pe[d0];
    if (m > 0) {
      if (me > 0) TRY_(radix_sort_u64(ke, nullptr, eslots, bits, s->sort_sc, st));
      TRY_(radix_sort_u64_pairs(ks, slots, nullptr, lo, bits + lo, s->sort_sc,
                                pair_emit(s, obj_bits, t_bits, ke, (unsigned long long)me,
                                          nullptr, s->d_out.p + out_at, m, nullptr),
                                st));
    } else if (me > 0) {
      return SCD_ERR_INTERNAL;  // ends without starts
    }
    if (m > 0) {
      if (cudaEventRecord(s->cev[b], st) != cudaSuccess ||
          cudaStreamWaitEvent(s->cstream, s->cev[b], 0) != cudaSuccess ||
          cudaMemcpyAsync(host + out_at, s->d_out.p + out_at, sizeof(scd_pair) * (size_t)m,
                          cudaMemcpyDeviceToHost, s->cstream) != cudaSuccess)
        return SCD_ERR_CUDA;
    }
    out_at += m;
    d0 = d1;
  }
  if (out_at != n) return SCD_ERR_INTERNAL;
  s->n_out = n;
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}
#undef TRY_

int canonicalize_dev(scd_scene *s, int obj_bits, int t_bits) {
  cudaStream_t st = s->stream;
  const int64_t cap = s->pair_cap;
  if (!s->d_out.ensure(cap, st)) return SCD_ERR_OOM;
  UnpackArgs a = unpack_args(s, 0, obj_bits, t_bits);
  const int lo = a.packed ? t_bits : 0, bits = 2 * obj_bits + t_bits;
  DevCounters *c = s->d_ctr.p;
  const int w = a.packed ? window_bits(bits, t_bits) : 0;
  int rc = radix_sort_u64_dev(s->d_starts.p, a.packed ? nullptr : s->d_rawval.p, cap,
                              &c->n_starts, lo + w, bits + lo, s->sort_sc, st);
  if (rc) return rc;
  if (w && (rc = window_fix(s->d_starts.p, cap, &c->n_starts, lo + w, st))) return rc;
  rc = radix_sort_u64_dev(s->d_ends.p, nullptr, cap, &c->n_ends, w, bits, s->sort_sc, st);
  if (rc) return rc;
  if (w && (rc = window_fix(s->d_ends.p, cap, &c->n_ends, w, st))) return rc;
  a.n = cap;
  a.d_n = &c->v_starts;
  a.n_ends = (unsigned long long)cap;
  a.d_ne = &c->v_ends;
  if (int rc2 = unpack(s, a, st)) return rc2;
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

}  // namespace scd
