// scd_internal.cuh -- types and helpers shared by the CUDA translation units
// of libscd (sm_103a).  Not part of the public ABI (include/scd.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/scd.h"

namespace scd {

// geocentric gravitational parameter [km^3/s^2] and equatorial Earth radius
// [km] (WGS-84); the paper's Eq. 1 names mu without giving a value
constexpr double kMu = 398600.4418;
constexpr double kRe = 6378.137;
constexpr double kTwoPi = 6.283185307179586;
constexpr double kPi = 3.141592653589793;
// margin added to every box half-width before outward FP32 rounding [km]
constexpr double kEpsKm = 1e-6;

// device error word bits
enum : uint32_t {
  ERR_KEPLER = 1u << 0,     // Kepler iteration hit its limit
  ERR_STACK = 1u << 1,      // traversal stack overflow
  ERR_INVALID = 1u << 2,    // invalid element seen on the device
  ERR_ZIP = 1u << 3,        // open run starts and run ends did not pair up
  ERR_SORT = 1u << 4,       // a sort's tile copy did not arrive in time
};

// Per-object propagation constants, derived once per scene from the
// elements (112 bytes, read through the read-only path by every box).
struct __align__(16) ObjParams {
  double A[3];   // a * P  (P: perifocal x axis in ECI)
  double B[3];   // a sqrt(1-e^2) * Q  (Q: perifocal y axis in ECI)
  double n;      // mean motion [rad/s]
  double M0;     // mean anomaly at t = 0 [rad]
  double e;      // eccentricity
  double vmax;   // perigee speed [km/s]
  double r;      // radius [km]
  double P;      // period [s]
  double tolE;   // eccentric-anomaly accuracy of the Kepler solve [rad]: 1e-7 km / a
  // the largest squared last Newton correction d that leaves the solve within
  // tolE / 4 for any E: Newton's error after the step, e |sin E| d^2 /
  // (2 (1 - e cos E)), is at most e d^2 / (2 (1 - e)); so tolE (1 - e) / (2 e)
  // (infinite for e = 0)
  float dmax2;
  float ef;      // e in FP32 (the Kepler solve's FP32 steps)
};

// Device-side counters of one scene, read back with one copy.  The first
// block is zeroed before every traversal; the second is written by the box
// build.
struct DevCounters {
  unsigned long long n_starts;  // record slots handed out (holes included)
  unsigned long long n_ends;
  unsigned long long n_raw;
  unsigned long long v_starts;  // records actually written
  unsigned long long v_ends;
  unsigned long long v_raw;
  unsigned long long node_tests;
  unsigned long long leaf_tests;
  unsigned long long work_next;  // next query claimed by the persistent traversal
  unsigned int trav_flags;   // ERR_STACK, ERR_ZIP
  unsigned int pad0;
  unsigned long long extent_bits;  // max object extent [km] as double bits
  unsigned int build_flags;        // ERR_KEPLER, ERR_INVALID
  unsigned int kepler_max_iter;
  unsigned long long n_boxes;      // seg_off[n]
  unsigned long long refs_total;   // references of the last decomposed build
  unsigned int sort_flags;         // ERR_SORT (set by any sort since the box build)
  unsigned int pad1;
};

// Traversal node: both children's boxes inline, child links and the
// rightmost leaf of each child (80 bytes).
struct __align__(16) TravNode {
  float4 lo_l, hi_l, lo_r, hi_r;
  int32_t left, right;  // child index; bit 31 set = leaf
  int32_t last_l, last_r;  // rightmost leaf index under each child
};

static_assert(sizeof(TravNode) == 80 && offsetof(TravNode, left) == 64,
              "the links are the node's fifth 16-byte word");

constexpr int32_t kLeafBit = (int32_t)0x80000000u;

// Compact node of the one-box-per-leaf traversal (36 bytes): both child
// boxes quantised in the scene frame (lower faces rounded down, upper faces
// up, so a quantised test never rejects a pair that overlaps in FP32) and
// the split gamma (left child gamma, right child gamma + 1) with two leaf
// flags; gamma is also the left child's rightmost leaf.  x and y take 16 bits, z 15 and the tick 17: one
// quantum per tick up to 131071 ticks, so boxes of consecutive segments
// (which touch, tick hi + 1 = tick lo, but do not overlap) stay apart.
struct __align__(16) QBox {
  uint32_t lo_xy, lo_zt, hi_xy, hi_zt;  // x | y << 16 and z | t << 15
};
constexpr uint32_t kQLeftLeaf = 0x80000000u, kQRightLeaf = 0x40000000u;
constexpr uint32_t kQIndex = 0x3fffffffu;

// Four-wide node (one box per leaf, node width 4): the grandchildren of a
// binary node in one 128-byte line.  Slots 0 and 1 hold the two children of
// the left child (or the left child itself when it is a leaf, and an empty
// slot), slots 2 and 3 those of the right child.  link.x = binary node or
// leaf index with flags, link.y = the slot's rightmost leaf (0 when empty).
// One traversal step reads the line with three 256-bit loads and descends
// two binary levels.
struct __align__(128) W4Node {
  QBox box[4];
  uint2 link[4];
  uint32_t pad[8];
};
static_assert(sizeof(W4Node) == 128, "one cache line per four-wide node");
constexpr uint32_t kW4Leaf = 0x80000000u, kW4Empty = 0x40000000u, kW4Index = 0x3fffffffu;
// the right-child bit of a parent link (the Karras build marks which side
// of its parent each internal node is)
constexpr int32_t kRightChildBit = 0x40000000;

// A sorted box: both corners in one 32-byte record (x, y, z in km, the tick
// in w), read with one 256-bit load.
struct __align__(32) SBox {
  float4 lo, hi;
};
__device__ __forceinline__ void ldg_box(const SBox *p, float4 &lo, float4 &hi) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z),
        "=f"(hi.w)
      : "l"(p));
}

// Both child boxes of a compact node (32 bytes, 32-byte aligned) in one
// 256-bit read-only load.
__device__ __forceinline__ void ldg_qbox_pair(const QBox *p, uint4 &l, uint4 &r) {
  asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(l.x), "=r"(l.y), "=r"(l.z), "=r"(l.w), "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p));
}
// the four links of a four-wide node
__device__ __forceinline__ void ldg_w4_links(const uint2 *p, uint4 &a, uint4 &b) {
  asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
      : "l"(p));
}

// the scene frame of the quantisation: x, y, z in [-R, R] km, t in [0, T]
struct QFrame {
  float R, sx, sz, st;  // sx = 65535 / 2R, sz = 32767 / 2R, st = min(1, 131071 / T)
};

// the frame of a scene, from the extent found by the box build; every kernel
// that quantises derives it with this same code, so the values agree
__device__ inline QFrame scene_frame(const DevCounters *ctr, int64_t T) {
  QFrame f;
  f.R = (float)__longlong_as_double((long long)ctr->extent_bits);
  f.sx = 65535.0f / (2.0f * f.R);
  f.sz = 32767.0f / (2.0f * f.R);
  f.st = fminf(1.0f, 131071.0f / (float)(T > 0 ? T : 1));
  return f;
}

// outward quantisation to [0, top]
__host__ __device__ inline uint32_t q_lo(float v, float top) {
  float f = floorf(v);
  f = f < 0.f ? 0.f : (f > top ? top : f);
  return (uint32_t)f;
}
__host__ __device__ inline uint32_t q_hi(float v, float top) {
  float f = ceilf(v);
  f = f < 0.f ? 0.f : (f > top ? top : f);
  return (uint32_t)f;
}
// quantise a box outward; the map x -> (x + R) * sx is monotone in FP32, so
// box order relations survive it
__host__ __device__ inline QBox quantize_box(const QFrame &f, float4 lo, float4 hi) {
  QBox q;
  q.lo_xy = q_lo((lo.x + f.R) * f.sx, 65535.f) | (q_lo((lo.y + f.R) * f.sx, 65535.f) << 16);
  q.lo_zt = q_lo((lo.z + f.R) * f.sz, 32767.f) | (q_lo(lo.w * f.st, 131071.f) << 15);
  q.hi_xy = q_hi((hi.x + f.R) * f.sx, 65535.f) | (q_hi((hi.y + f.R) * f.sx, 65535.f) << 16);
  q.hi_zt = q_hi((hi.z + f.R) * f.sz, 32767.f) | (q_hi(hi.w * f.st, 131071.f) << 15);
  return q;
}

// a <= b in both fields of a z | t << 15 word
__device__ __forceinline__ bool zt_le(uint32_t a, uint32_t b) {
  return (a & 0x7fffu) <= (b & 0x7fffu) && (a >> 15) <= (b >> 15);
}

__device__ inline uint32_t quantize(float u, int bits) {
  float s = (float)(1u << bits);
  float q = floorf(u * s);
  q = fminf(fmaxf(q, 0.0f), s - 1.0f);
  return (uint32_t)q;
}

__device__ inline unsigned long long morton4(uint32_t x, uint32_t y, uint32_t z, uint32_t t,
                                             int bits) {
  unsigned long long key = 0;
  for (int b = 0; b < bits; ++b) {
    key |= (unsigned long long)((t >> b) & 1u) << (4 * b + 0);
    key |= (unsigned long long)((z >> b) & 1u) << (4 * b + 1);
    key |= (unsigned long long)((y >> b) & 1u) << (4 * b + 2);
    key |= (unsigned long long)((x >> b) & 1u) << (4 * b + 3);
  }
  return key;
}

// 4D Morton key (bits per axis) of a box centre in the scene cube [-R, R]^3
// x [0, T]; optionally log-compressed in space (a monotone map, so any key
// order is a valid tree order).  time_scale weighs time against space: below
// 1 the horizon takes that share of the time axis's cells, above 1 the
// scene cube takes 1 / time_scale of the space axes' cells (around the
// centre), so time counts that many times more in the curve's order.
// R is the cube's half-side, T1 the horizon plus one tick; all in FP32.
__device__ inline unsigned long long box_morton(float4 L, float4 H, float R, float T1, int bits,
                                                float time_scale, int space_warp) {
  const float sw = time_scale > 1.0f ? 1.0f / time_scale : 1.0f;
  const float tw = time_scale > 1.0f ? 1.0f : time_scale;
  float ux, uy, uz;
  if (space_warp) {
    const float s_km = 1000.0f;
    float inv = sw * 0.5f / log1pf(R / s_km);
    float cx = 0.5f * (L.x + H.x), cy = 0.5f * (L.y + H.y), cz = 0.5f * (L.z + H.z);
    ux = copysignf(log1pf(fabsf(cx) / s_km), cx) * inv + 0.5f;
    uy = copysignf(log1pf(fabsf(cy) / s_km), cy) * inv + 0.5f;
    uz = copysignf(log1pf(fabsf(cz) / s_km), cz) * inv + 0.5f;
  } else {
    float inv = sw * (0.5f / R);
    ux = (0.5f * (L.x + H.x)) * inv + 0.5f;
    uy = (0.5f * (L.y + H.y)) * inv + 0.5f;
    uz = (0.5f * (L.z + H.z)) * inv + 0.5f;
  }
  float ut = (0.5f * (L.w + H.w)) / T1 * tw;  // ticks below 2^24: the sum is exact
  return morton4(quantize(ux, bits), quantize(uy, bits), quantize(uz, bits), quantize(ut, bits),
                 bits);
}

// The size group of a box (tuning split_km): boxes whose largest spatial
// side exceeds |split_km| km form one group and the others another; the
// group bit goes above the Morton key, so each group is sorted apart and
// gets its own subtree.  1 = the group sorted last: the large boxes when
// split_km > 0, the small ones when split_km < 0.
__device__ __forceinline__ uint32_t split_bit(float4 L, float4 H, float split_km) {
  if (split_km == 0.0f) return 0u;
  const float ext = fmaxf(fmaxf(H.x - L.x, H.y - L.y), H.z - L.z);
  return (split_km > 0.0f) == (ext > fabsf(split_km)) ? 1u : 0u;
}
// the split applies to Morton keys with room above them: 10 or 12 bits per axis
inline float split_of(const scd_tuning &t) {
  return t.morton_bits == 10 || t.morton_bits == 12 ? t.split_km : 0.0f;
}
// The sort key of a box: its Morton key with the size group's bit above it.
// With 12-bit axes the group bit takes the place of the key's lowest bit
// (the finest time bit), so that the key stays 48 bits (6 sort passes, not
// 7; measured: node tests +0.25%, the screen 0.15 ms shorter); with 10-bit
// axes that bit is worth more than the pass (traversal +12%).
__host__ __device__ inline unsigned long long sort_key(unsigned long long morton, uint32_t group,
                                                       int bits, bool split) {
  if (!split) return morton;
  if (bits >= 12) return (morton >> 1) | (unsigned long long)group << (4 * bits - 1);
  return morton | (unsigned long long)group << (4 * bits);
}
inline int sort_key_bits(const scd_tuning &t) {
  const bool split = split_of(t) != 0.0f;
  return 4 * t.morton_bits + (split && t.morton_bits < 12 ? 1 : 0);
}

// Refinement rounds: flags of an interval (it met a box of another object;
// that box was longer than one tick), a tick candidate t (24 bits) | i (20)
// | j (20), which sorts in Alg 1's order, and a span of two meeting
// intervals [ka, ka + 1], [kb, kb + 1] of one level of the continuous
// variant, i (20) | j (20) | the later start (22) | whether the starts agree
// (1), which sorts by (i, j, t0, t1) of the intersection.
constexpr uint32_t kRfHit = 1u, kRfHitLong = 2u;
__host__ __device__ inline unsigned long long rf_tick_key(uint32_t t, uint32_t i, uint32_t j) {
  return ((unsigned long long)t << 40) | ((unsigned long long)i << 20) | (unsigned long long)j;
}
__host__ __device__ inline unsigned long long rf_span_key(uint32_t i, uint32_t j, int32_t ka,
                                                          int32_t kb) {
  const uint32_t km = (uint32_t)(ka > kb ? ka : kb), same = ka == kb ? 1u : 0u;
  return ((unsigned long long)i << 44) | ((unsigned long long)j << 24) |
         ((unsigned long long)km << 1) | same;
}

// decomposition cells: the tick slab of t, and the altitude band of radius x
// (the number of band edges <= x)
__device__ inline int slab_of(int64_t t, int n_slabs, int64_t T) {
  return (int)((t * (int64_t)n_slabs) / (T + 1));
}
__device__ inline int band_of(double x, const double *edges, int p) {
  int lo = 0, hi = p - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (edges[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__host__ __device__ inline bool box_overlap(const float4 &la, const float4 &ha,
                                            const float4 &lb, const float4 &hb) {
  // closed boxes: overlap iff every axis overlaps
  return la.x <= hb.x && lb.x <= ha.x && la.y <= hb.y && lb.y <= ha.y &&
         la.z <= hb.z && lb.z <= ha.z && la.w <= hb.w && lb.w <= ha.w;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

void *dev_alloc(size_t bytes, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);

template <class T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
  bool ensure(size_t count, cudaStream_t st) {
    if (count <= n && p) return true;
    if (p) dev_free(p, st);
    p = nullptr;
    n = 0;
    size_t c = count < 1 ? 1 : count;
    p = (T *)dev_alloc(c * sizeof(T), st);
    if (!p) return false;
    n = c;
    return true;
  }
  // grow to at least `count` elements keeping the first `used`
  bool grow_keep(size_t count, size_t used, cudaStream_t st) {
    if (count <= n && p) return true;
    T *q = (T *)dev_alloc((count < 1 ? 1 : count) * sizeof(T), st);
    if (!q) return false;
    if (p && used > 0 &&
        cudaMemcpyAsync(q, p, used * sizeof(T), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      dev_free(q, st);
      return false;
    }
    if (p) dev_free(p, st);
    p = q;
    n = count < 1 ? 1 : count;
    return true;
  }
  void release(cudaStream_t st) {
    if (p) dev_free(p, st);
    p = nullptr;
    n = 0;
  }
};

// radix sort scratch: ping-pong key/value buffers and block counts
struct SortScratch {
  DevBuf<unsigned char> keys_alt;
  DevBuf<uint32_t> vals_alt;
  DevBuf<uint32_t> counts;
  DevBuf<uint32_t> ocounts;  // open run starts per digit and tile (last pass into pairs)
  unsigned int *err = nullptr;  // device word that receives ERR_SORT (may be null)
  void release(cudaStream_t st) {
    keys_alt.release(st);
    vals_alt.release(st);
    counts.release(st);
    ocounts.release(st);
  }
};

// The last pass of the run starts' sort written straight out as pairs: the
// start keys (i, j, first tick) carry the run's last tick in their low tb
// bits, all ones for an open run, whose last tick is that of the k-th
// sorted end for the k-th open start (k counted in the final order).
struct PairEmit {
  int ob, tb;
  const unsigned long long *ends;     // the sorted ends of the open runs
  unsigned long long n_ends;          // their count (a capacity when d_ne is set)
  const unsigned long long *d_ne;
  scd_pair *out;
  int64_t n;                          // starts that are records (the rest are holes)
  const unsigned long long *d_n;
  unsigned int *flags;                // receives ERR_ZIP
};

// Sort (key, value) pairs by the low `bits` bits of the key, LSD, 8-bit
// digits, stable.  keys/vals are sorted in place (via the scratch ping-pong).
// vals may be null (keys only).  Returns cudaSuccess or the launch error.
int radix_sort_u32(uint32_t *keys, uint32_t *vals, int64_t n, int bits, SortScratch &sc,
                   cudaStream_t st);
int radix_sort_u64(unsigned long long *keys, uint32_t *vals, int64_t n, int bits,
                   SortScratch &sc, cudaStream_t st);
// the same by key bits [lo, bits) only (the bits below lo are payload)
int radix_sort_u64(unsigned long long *keys, uint32_t *vals, int64_t n, int lo, int bits,
                   SortScratch &sc, cudaStream_t st);
// size the scratch for sorts of up to n elements (nothing allocated later)
int sort_reserve(SortScratch &sc, int64_t n, size_t key_bytes, bool vals, cudaStream_t st);
// the same with the element count read on the device (min(*d_n, n_cap)), for
// sorts inside a captured graph; grids are sized for n_cap
// Sort the packed run starts keys[0, n) (a capacity with d_n) by bits
// [lo, bits) and write the sorted records as pairs into pe.out: the passes
// before the last as radix_sort_u64, the last one scattering decoded pairs
// (each open start zipped with its end) instead of keys.  The keys are left
// in an unspecified order.
int radix_sort_u64_pairs(unsigned long long *keys, int64_t n, const unsigned long long *d_n,
                         int lo, int bits, SortScratch &sc, const PairEmit &pe, cudaStream_t st);
int radix_sort_u64_dev(unsigned long long *keys, uint32_t *vals, int64_t n_cap,
                       const unsigned long long *d_n, int lo, int bits, SortScratch &sc,
                       cudaStream_t st);

// Run starts carry their last tick below the (i, j, first tick) key when
// both fit in 64 bits and the all-ones tick field is free to tag open runs
// (T < 2^t_bits - 1); otherwise the last tick travels as a 32-bit sort value
// and open runs carry 0xffffffff.
inline bool runs_packed(int obj_bits, int t_bits, int64_t T) {
  return 2 * (obj_bits + t_bits) <= 64 && T < (1ll << t_bits) - 1;
}
inline uint32_t open_tag(bool packed, int t_bits) {
  return packed ? (uint32_t)((1ull << t_bits) - 1ull) : 0xffffffffu;
}

// exclusive prefix sum of a[0..n) in place; *total = the sum (one block)
void scan_u32_exclusive(uint32_t *a, int64_t n, uint32_t *total, cudaStream_t st);
// One stable scatter pass of the keys kin[0, n) by their 8-bit digit at
// `shift` into kout, every digit's range starting at an even position (an
// odd range is followed by one hole key, all ones), so that every run of
// whole digits starts 16-byte aligned; kout holds n + 256 keys.  h_totals
// (host, 256 entries) receives each digit's key count (the call waits for
// the stream).
int radix_partition_u64(const unsigned long long *kin, unsigned long long *kout, int64_t n,
                        int shift, SortScratch &sc, uint32_t *h_totals, cudaStream_t st);

// process-wide count of kernel launches issued by this library
void note_launch(int k = 1);
unsigned long long launch_count();

// exclusive scan of n int64 values; out has n+1 entries (out[n] = total)
int scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, DevBuf<int64_t> &tmp,
                       cudaStream_t st);

}  // namespace scd

// the scene (opaque in the ABI)
namespace scd {
constexpr int kStreamBuckets = 16;  // buckets of a canonical list streamed to the host
struct RfCache;  // the refinement's buffers and captured rounds (refine.cu)
}

struct scd_scene {
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t n = 0;
  double horizon_s = 0, tick_s = 0;
  int64_t T = 0;  // horizon in ticks
  int step_kind = 0;
  uint32_t fixed_ticks = 1;
  double period_fraction = 100.0;
  std::vector<double> band_edges, band_fracs;
  const void *stepnet = nullptr;
  int box_mode = 0;
  scd_tuning tune{};

  // per-object
  scd::DevBuf<scd_element> d_el;
  scd::DevBuf<scd::ObjParams> d_par;
  scd::DevBuf<int32_t> d_k;
  scd::DevBuf<int64_t> d_segcnt, d_segoff, d_scan_tmp;
  scd::DevBuf<double> d_band;  // edges then fractions
  scd::DevBuf<scd::DevCounters> d_ctr;
  scd::DevCounters h_ctr{};  // pinned copy target lives in h_ctr_pinned
  scd::DevCounters *h_ctr_pinned = nullptr;

  // boxes (object-major)
  int64_t N = 0;
  bool boxes_built = false;
  scd::DevBuf<float4> d_lo, d_hi;
  scd::DevBuf<uint32_t> d_obj;
  scd::DevBuf<unsigned long long> d_key64;
  scd::DevBuf<uint32_t> d_key32;
  scd::DevBuf<uint32_t> d_id;  // box ids, sorted along with the keys

  // sorted leaves and hierarchy
  scd::DevBuf<scd::SBox> s_box;
  scd::DevBuf<uint32_t> s_obj;
  scd::DevBuf<uint32_t> d_posof;  // sorted position of each box id
  scd::DevBuf<int2> s_nb;         // sorted positions of the previous / next segment (-1: none)
  scd::DevBuf<uint32_t> s_cell;   // decomposition cell of each sorted reference
  scd::DevBuf<int32_t> d_first;   // first leaf under each internal node

  // static decomposition: references (cell, box) and per-cell subtrees
  int64_t n_refs = 0;
  int n_cells = 0;
  int dkind = 0, n_slabs = 0, p_bands = 0;  // decomposition of the last find_pairs
  scd::DevBuf<int64_t> d_refcnt, d_refoff;
  scd::DevBuf<unsigned long long> d_refkey;
  scd::DevBuf<uint32_t> d_refid;
  scd::DevBuf<double2> d_rr;       // padded radial range of each object
  scd::DevBuf<double> d_edges;     // altitude band edges (p - 1)
  scd::DevBuf<unsigned long long> d_abits;  // semi-major axes as sortable bits
  scd::DevBuf<int32_t> d_cellroot; // root node of each cell (-1: fewer than 2 refs)

  // learned steps: features, network outputs, steps [s]
  scd::DevBuf<float> d_feat, d_ny, d_learned;

  // a batch of independent scenes in one scene: per-object scene and
  // horizon, scene object offsets (host), one cell per scene
  int n_scenes = 0;
  std::vector<int64_t> scene_off;
  scd::DevBuf<int32_t> d_objT, d_objscene;
  scd::DevBuf<int64_t> d_sceneoff, d_pairoff;

  // graph mode: the captured find sequence and the sizes it was captured for
  cudaGraphExec_t graph_exec = nullptr;
  bool graph_ok = false;
  int last_graph = 0;  // last find: 0 eager, 1 eager + capture, 2 replay
  // capture and replay run on the scene's own stream, ordered after and
  // before the caller's stream by events (the legacy default stream cannot
  // be captured)
  cudaStream_t gstream = nullptr;
  cudaEvent_t g_in = nullptr, g_out = nullptr;
  // a find into host memory: the destination, its room, and whether the
  // canonical list was streamed into it (buckets copied on cstream)
  scd_pair *host_dst = nullptr;
  int64_t host_cap = 0;
  bool host_done = false;
  scd::RfCache *rf = nullptr;  // the adaptive refinement's buffers and graph
  cudaStream_t cstream = nullptr;
  cudaEvent_t cev[scd::kStreamBuckets] = {};
  scd::DevBuf<unsigned long long> d_part, d_parte;  // the records split by their top digit
  int64_t graph_key[8] = {};
  int64_t graph_M = 0;
  scd::DevBuf<uint32_t> s_leafkey32;
  scd::DevBuf<unsigned long long> s_leafkey64;
  scd::DevBuf<scd::TravNode> d_nodes;
  scd::DevBuf<scd::QBox> d_qbox;     // 2 per internal node (one box per leaf)
  scd::DevBuf<scd::W4Node> d_w4;     // four-wide nodes (node width 4)
  scd::DevBuf<uint32_t> d_qlink;     // per internal node: gamma | leaf flags
  scd::DevBuf<float4> d_nlo, d_nhi;     // internal node boxes (refit)
  scd::DevBuf<float4> d_leaflo, d_leafhi;
  scd::DevBuf<int32_t> d_parent_int, d_parent_leaf;
  scd::DevBuf<uint32_t> d_flags;
  scd::DevBuf<int32_t> d_first_last;   // per internal node: first, last

  // pair emission and canonical list
  int64_t pair_cap = 0;
  scd::DevBuf<unsigned long long> d_starts, d_ends;
  scd::DevBuf<uint32_t> d_tilecnt;  // open run starts per unpack tile
  scd::DevBuf<uint32_t> d_rawval;
  scd::DevBuf<scd_pair> d_out;
  int64_t n_out = 0;
  scd::SortScratch sort_sc;

  // narrow phase: device state words, tick evaluations of the last call
  scd::DevBuf<unsigned long long> d_narrow;
  scd::DevBuf<unsigned char> d_npobj;  // per-object FP32 constants (64 B each)
  unsigned long long last_np_evals = 0, last_np_evals64 = 0;

  // refinement: the capacities (intervals a round, candidates) and the
  // traversal stack that sufficed last time
  int64_t rf_cap = 0, rf_ccap = 0;
  int rf_deep = 0;

  // metrics of the last find_pairs
  double ms_sort = 0, ms_build = 0, ms_traverse = 0, ms_canon = 0, ms_boxes = 0;
  unsigned long long last_node_tests = 0, last_leaf_tests = 0, last_runs = 0, last_open = 0;
  unsigned long long launch_mark = 0, last_launches = 0;  // kernels of build + find
  cudaEvent_t ev[8] = {};
  bool events_ready = false;
};

namespace scd {
// launchers defined in the .cu files
int launch_prepare_objects(scd_scene *s);
int launch_build_boxes(scd_scene *s);
int launch_propagate(const scd_element *d_el, int64_t n, const uint32_t *obj, const double *t,
                     int64_t m, double *out, cudaStream_t st);
int build_hierarchy(scd_scene *s, int64_t &n_leaves);
int build_round_tree(const unsigned long long *keys, const SBox *sbox, int64_t cap,
                     const unsigned long long *d_M, TravNode *nodes, int32_t *parent_int,
                     int32_t *parent_leaf, uint32_t *arrive, QBox *nq, QBox *qbox,
                     uint32_t *qlink, const DevCounters *ctr, int64_t T, cudaStream_t st);
template <class K>
int build_tree(scd_scene *s, const K *keys_sorted, const uint32_t *ids_sorted, int64_t Nq,
               K *leafkey, int cell_shift, int64_t &M);
// decomposed screen: references, their sort, the tree and each cell's root
int build_decomposed(scd_scene *s, const scd_decomp *d, int64_t &n_leaves,
                     bool capturing = false);
// learned per-object steps [s] into s->d_learned (SCD_STEP_LEARNED)
int learned_steps(scd_scene *s);
// internal decomposition kind of a batch of scenes: one cell per scene
constexpr int kDecompScenes = 100;
int traverse(scd_scene *s, int64_t n_leaves, int raw_mode, int obj_bits, int t_bits);
int traverse_round(const QBox *qbox, const uint32_t *qlink, const SBox *sbox,
                   const uint32_t *sobj, const uint32_t *sid, int64_t cap,
                   const unsigned long long *d_N, int64_t T, DevCounters *ctr, uint32_t *rflags,
                   unsigned long long *rcand, unsigned long long *rncand, unsigned long long rcap,
                   int spans, int deep, cudaStream_t st);
int canonicalize(scd_scene *s, int raw_mode, int obj_bits, int t_bits);
// canonical list with every count read on the device (graph capture)
int canonicalize_dev(scd_scene *s, int obj_bits, int t_bits);
// the refinement's buffers and graph kept by the scene, freed with it
void rf_release(scd_scene *s);
// canonical list streamed into host memory bucket by bucket (run starts
// packed with their last tick); SCD_ERR_STATE when the records do not allow
// it; the copies are left running on the scene's copy stream
int canonicalize_streamed(scd_scene *s, int obj_bits, int t_bits, scd_pair *host);
}  // namespace scd
