// radix_sort.cu -- LSD radix sort of 32- or 64-bit keys with optional 32-bit
// values (step A5: ordering boxes along the 4D Morton curve; step A9:
// ordering candidate records by (i, j, tick)).
//
// Reduce-then-scan per 8-bit digit: (1) every block counts the digits of its
// tile, (2) one block per digit scans that digit's counts over the blocks,
// (3) every block ranks its tile stably in shared memory (warp match + per
// warp counters) and writes each digit's run to its global offset.  No block
// ever waits on another block.
#include <algorithm>

#include "scd_internal.cuh"

namespace scd {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;

template <class K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift) {
  return (uint32_t)(key >> shift) & 0xffu;
}

// The element count: a host value, or (inside a captured graph) a device
// count clamped to the capacity the grid was sized for.  Blocks past the
// count see no items: they count zeros and write nothing.
__device__ __forceinline__ int64_t sort_count(int64_t n, const unsigned long long *d_n) {
  if (!d_n) return n;
  unsigned long long v = *d_n;
  return v < (unsigned long long)n ? (int64_t)v : n;
}

// kOpen: also count, per digit, the keys whose low tmask bits are all ones
// (open run starts; holes too, which sort last) into ocounts
template <class K, bool kOpen = false>
__global__ void __launch_bounds__(kRsThreads) k_rs_upsweep(const K *__restrict__ keys, int64_t n,
                                                           const unsigned long long *__restrict__ d_n,
                                                           int shift, uint32_t *__restrict__ counts,
                                                           int64_t nblk,
                                                           uint32_t *__restrict__ ocounts = nullptr,
                                                           unsigned long long tmask = 0) {
  n = sort_count(n, d_n);
  // past a device count: no counts (the scan and the scatter stop there)
  if (d_n && (int64_t)blockIdx.x * kRsTile >= n) return;
  __shared__ uint32_t wh[kRsWarps][256];
  __shared__ uint32_t wo[kOpen ? kRsWarps : 1][256];
  int w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&wh[0][0])[i] = 0;
  if (kOpen)
    for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&wo[0][0])[i] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kRsTile;
  // all loads first, so that every item's load is in flight together
  uint32_t dig[kRsItems];
  bool op[kRsItems];
#pragma unroll
  for (int k = 0; k < kRsItems; ++k) {
    int64_t idx = base + (int64_t)k * kRsThreads + threadIdx.x;
    const K key = idx < n ? keys[idx] : (K)0;
    dig[k] = idx < n ? digit_of(key, shift) : 256u;
    op[k] = kOpen && ((unsigned long long)key & tmask) == tmask;
  }
#pragma unroll
  for (int k = 0; k < kRsItems; ++k)
    if (dig[k] < 256u) {
      atomicAdd(&wh[w][dig[k]], 1u);
      if (kOpen && op[k]) atomicAdd(&wo[w][dig[k]], 1u);
    }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += kRsThreads) {
    uint32_t s = 0, o = 0;
#pragma unroll
    for (int q = 0; q < kRsWarps; ++q) {
      s += wh[q][d];
      if (kOpen) o += wo[q][d];
    }
    counts[(int64_t)d * nblk + blockIdx.x] = s;
    if (kOpen) ocounts[(int64_t)d * nblk + blockIdx.x] = o;
  }
}

// exclusive scan over one digit's block counts; totals[d] = the digit's count.
// A chunk is 1024 x kScanItems counts: warp w holds a segment of 32 x
// kScanItems, item k of lane l at k * 32 + l (coalesced), scanned within
// the warp in registers; one block-wide scan of the warp totals per chunk.
constexpr int kScanItems = 8;
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t *__restrict__ counts, int64_t nblk,
                                                  uint32_t *__restrict__ totals,
                                                  const unsigned long long *__restrict__ d_n =
                                                      nullptr,
                                                  int64_t n = 0) {
  __shared__ uint32_t ws[32];
  uint32_t *c = counts + (int64_t)blockIdx.x * nblk;  // rows of nblk
  // with a device count, only the blocks that hold items counted
  if (d_n) nblk = std::min<int64_t>(nblk, (sort_count(n, d_n) + kRsTile - 1) / kRsTile);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t carry = 0;
  for (int64_t b0 = 0; b0 < nblk; b0 += 1024 * kScanItems) {
    const int64_t seg = b0 + (int64_t)w * 32 * kScanItems + lane;
    uint32_t v[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) v[k] = seg + k * 32 < nblk ? c[seg + k * 32] : 0u;
    uint32_t wrun = 0;  // the warp segment's items before item k
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      uint32_t x = v[k];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      const uint32_t item = v[k];
      v[k] = wrun + x - item;  // exclusive, within the warp's segment
      wrun += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) ws[w] = wrun;
    __syncthreads();
    if (w == 0) {
      uint32_t s = ws[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      ws[lane] = s;
    }
    __syncthreads();
    const uint32_t before = (w > 0 ? ws[w - 1] : 0u) + carry;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
      if (seg + k * 32 < nblk) c[seg + k * 32] = before + v[k];
    carry += ws[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

static_assert(kRsThreads == 256, "one thread per digit in the digit scans");

// exclusive scan of one value per thread over the 256 threads of the block
__device__ __forceinline__ uint32_t digit_scan_excl(uint32_t v, uint32_t *buf) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  buf[threadIdx.x] = x;
  __syncthreads();
  uint32_t add = 0;
  for (int q = 0; q < w; ++q) add += buf[q * 32 + 31];
  __syncthreads();
  return x + add - v;
}

// --- bulk copies (TMA) of whole tiles into shared memory ------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// one contiguous global -> shared copy completing on `bar`; both addresses
// 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Wait for the phase with the given parity to complete; gives up after a
// bounded number of polls (about a second) and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  for (int it = 0; it < (1 << 23); ++it) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

// Scatter pass, persistent: block b handles tiles b, b + G, b + 2G, ... .
// Every full tile's keys (and values) arrive by bulk copy into one of two
// shared buffers while the tile before is ranked and written, so a copy is
// in flight during every block's compute; the buffer of the tile at hand
// then serves as the staging area of its scatter.  A last partial tile is
// read with plain loads.  Items of a tile are warp-striped: warp w holds
// tile items [w*32*I, (w+1)*32*I), item k of lane l at w*32*I + k*32 + l,
// so (k, lane) order is input order and ranks are stable.
// kPairs (the last pass of the packed run starts' sort): instead of the
// keys, the decoded pairs of the records go to their sorted positions, each
// open start with the last tick of the end whose rank among the ends equals
// its own rank among the open starts (from the open counts per digit and
// tile, ocounts / ototals, and an in-tile prefix).
template <class K, bool kVals, bool kPairs = false>
__global__ void __launch_bounds__(kRsThreads, 4) k_rs_downsweep(
    const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout,
    uint32_t *__restrict__ vout, int64_t n, const unsigned long long *__restrict__ d_n, int shift,
    const uint32_t *__restrict__ counts, const uint32_t *__restrict__ totals, int64_t nblk,
    unsigned int *err, int even = 0, const uint32_t *__restrict__ ocounts = nullptr,
    const uint32_t *__restrict__ ototals = nullptr, PairEmit pe = PairEmit{}) {
  n = sort_count(n, d_n);
  const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
  extern __shared__ __align__(128) unsigned char smem[];
  K *kbuf0 = (K *)smem;
  K *kbuf1 = kbuf0 + kRsTile;
  uint32_t *vbuf0 = (uint32_t *)(smem + 2 * sizeof(K) * kRsTile);
  uint32_t *vbuf1 = vbuf0 + kRsTile;
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t wcnt[kRsWarps][256];  // per warp, per digit
  __shared__ uint32_t scanbuf[256];
  __shared__ uint32_t gdig[256];   // first global position of each digit
  __shared__ uint32_t gbase[256];  // global position of the tile's first item of each digit,
                                   // less the digit's first tile position (mod 2^32)
  // kPairs: open starts before the digit's first open start (ordered), and
  // the open starts of the tile's staged items before each digit's run
  __shared__ uint32_t odig[kPairs ? 256 : 1], obase[kPairs ? 256 : 1];
  __shared__ uint16_t opre[kPairs ? kRsTile : 1];  // open starts before each staged item

  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int d = threadIdx.x;  // one thread per digit in the digit phases
  const uint32_t tile_bytes = (uint32_t)(sizeof(K) * kRsTile);
  auto full_tile = [&](int64_t t) { return t < ntiles && (t + 1) * kRsTile <= n; };
  auto issue = [&](int64_t t, int b) {  // thread 0 only
    if (!full_tile(t)) return;
    mbar_expect_tx(&bar[b], tile_bytes + (kVals ? 4u * kRsTile : 0u));
    bulk_load(b ? kbuf1 : kbuf0, kin + t * kRsTile, tile_bytes, &bar[b]);
    if (kVals) bulk_load(b ? vbuf1 : vbuf0, vin + t * kRsTile, 4u * kRsTile, &bar[b]);
  };

  // (even: every digit's range rounded up to an even length)
  gdig[d] = digit_scan_excl(even ? (totals[d] + 1u) & ~1u : totals[d], scanbuf);
  if constexpr (kPairs) odig[d] = digit_scan_excl(ototals[d], scanbuf);
  const unsigned long long tmask = kPairs ? (1ull << pe.tb) - 1ull : 0ull;
  const int64_t nvalid = kPairs ? sort_count(pe.n, pe.d_n) : 0;
  const unsigned long long n_ends =
      kPairs ? (pe.d_ne && *pe.d_ne < pe.n_ends ? *pe.d_ne : pe.n_ends) : 0ull;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    issue(blockIdx.x, 0);
    issue((int64_t)blockIdx.x + gridDim.x, 1);
  }
  uint32_t parity0 = 0, parity1 = 0;
  int b = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, b ^= 1) {
    const int64_t base = tile * kRsTile;
    const bool full = full_tile(tile);
    K *kb = b ? kbuf1 : kbuf0;
    uint32_t *vb = b ? vbuf1 : vbuf0;
    for (int i = lane; i < 256; i += 32) wcnt[w][i] = 0;
    gbase[d] = gdig[d] + counts[(int64_t)d * nblk + tile];
    if constexpr (kPairs) obase[d] = odig[d] + ocounts[(int64_t)d * nblk + tile];
    bool ok = true;
    if (full) {
      ok = mbar_wait(&bar[b], b ? parity1 : parity0);
      if (b) parity1 ^= 1u; else parity0 ^= 1u;
    }
    // the whole block decides together (a barrier; the counters above are
    // zeroed and gbase written before it)
    if (!__syncthreads_and(ok)) {
      // give up: report, then leave only once the copies into both buffers
      // have landed or their (bounded) waits have run out again, so that no
      // copy is still writing into the block's shared memory when it exits
      if (threadIdx.x == 0 && err) atomicOr(err, (unsigned)ERR_SORT);
      if (full) mbar_wait(&bar[b], (b ? parity1 : parity0) ^ 1u);
      if (full_tile(tile + gridDim.x)) mbar_wait(&bar[b ^ 1], b ? parity0 : parity1);
      return;
    }

    // (b) rank every item inside its warp
    const int seg = w * 32 * kRsItems;
    K key[kRsItems];
    uint32_t val[kRsItems];
    uint32_t rnk[kRsItems];
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
      const int i = seg + k * 32 + lane;
      if (full) {
        key[k] = kb[i];
        if (kVals) val[k] = vb[i];
      } else {
        const bool valid = base + i < n;
        key[k] = valid ? kin[base + i] : (K)0;
        if (kVals) val[k] = valid ? vin[base + i] : 0u;
      }
    }
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
      const bool valid = base + seg + k * 32 + lane < n;
      uint32_t dg = valid ? digit_of(key[k], shift) : 256u;
      unsigned peers = __match_any_sync(0xffffffffu, dg);
      uint32_t before = valid ? wcnt[w][dg] : 0u;
      rnk[k] = before + __popc(peers & lt);
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) wcnt[w][dg] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();  // every warp's counts are in; the tile buffer is free

    // (c) per digit: the digit's first tile position (a scan over the
    // digits), then each warp's first position within it; afterwards
    // wcnt[w][dg] is warp w's first tile position for digit dg
    {
      uint32_t run = 0;
#pragma unroll
      for (int q = 0; q < kRsWarps; ++q) run += wcnt[q][d];
      uint32_t at = digit_scan_excl(run, scanbuf);
      gbase[d] -= at;
#pragma unroll
      for (int q = 0; q < kRsWarps; ++q) {
        const uint32_t c = wcnt[q][d];
        wcnt[q][d] = at;
        at += c;
      }
    }
    __syncthreads();

    // (d) scatter into the tile buffer at the tile-local rank
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
      if (base + seg + k * 32 + lane < n) {
        uint32_t dg = digit_of(key[k], shift);
        uint32_t r = wcnt[w][dg] + rnk[k];
        kb[r] = key[k];
        if (kVals) vb[r] = val[k];
      }
    }
    __syncthreads();

    // (e) each digit's run goes to consecutive global positions
    const int cnt = n - base < kRsTile ? (int)(n - base) : kRsTile;
    if constexpr (kPairs) {
      // the open starts before every staged item: per thread over kRsItems
      // consecutive items, then across the threads
      const int r0 = threadIdx.x * kRsItems;
      uint32_t mine = 0;
#pragma unroll
      for (int k = 0; k < kRsItems; ++k)
        if (r0 + k < cnt) mine += ((unsigned long long)kb[r0 + k] & tmask) == tmask;
      uint32_t run = digit_scan_excl(mine, scanbuf);
#pragma unroll
      for (int k = 0; k < kRsItems; ++k)
        if (r0 + k < cnt) {
          opre[r0 + k] = (uint16_t)run;
          run += ((unsigned long long)kb[r0 + k] & tmask) == tmask;
        }
      __syncthreads();
      // then the pairs, warp-contiguous as the keys would be
      bool bad = false;
      const unsigned long long omask = (1ull << pe.ob) - 1ull;
      for (int r = threadIdx.x; r < cnt; r += kRsThreads) {
        const unsigned long long kk = (unsigned long long)kb[r];
        const uint32_t dg = digit_of((K)kk, shift);
        const int64_t pos = (int64_t)(uint32_t)(gbase[dg] + (uint32_t)r);
        if (pos >= nvalid) continue;
        const bool open = (kk & tmask) == tmask;
        // open starts before this one in the final order
        const unsigned long long rank =
            (unsigned long long)obase[dg] + (uint32_t)(opre[r] - opre[wcnt[0][dg]]);
        const unsigned long long key = kk >> pe.tb;  // (i, j, first tick)
        scd_pair q;
        q.i = (uint32_t)(key >> (pe.ob + pe.tb));
        q.j = (uint32_t)((key >> pe.tb) & omask);
        q.tlo = (int32_t)(key & tmask);
        q.thi = (int32_t)(kk & tmask);
        if (open) {
          if (rank < n_ends) {
            const unsigned long long ek = __ldg(pe.ends + rank);
            q.thi = (int32_t)(ek & tmask);
            bad |= (ek >> pe.tb) != (key >> pe.tb) || q.thi <= q.tlo;
          } else {
            bad = true;
          }
        }
        pe.out[pos] = q;
        // the last record: every end taken by exactly one open start
        if (pos == nvalid - 1 && rank + (open ? 1u : 0u) != n_ends) bad = true;
      }
      if (bad) atomicOr(pe.flags, (unsigned)ERR_ZIP);
    } else {
      for (int r = threadIdx.x; r < cnt; r += kRsThreads) {
        K kk = kb[r];
        uint32_t dg = digit_of(kk, shift);
        uint32_t pos = gbase[dg] + (uint32_t)r;
        kout[pos] = kk;
        if (kVals) vout[pos] = vb[r];
      }
    }
    __syncthreads();  // the buffer is read out: the copy of the tile after next may land
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(tile + 2 * (int64_t)gridDim.x, b);
    }
  }
}

template <class K>
static int rs_impl(K *keys, uint32_t *vals, int64_t n, const unsigned long long *d_n, int lo,
                   int bits, SortScratch &sc, cudaStream_t st, const PairEmit *pe = nullptr) {
  if (!pe && (n <= 1 || bits <= lo)) return SCD_OK;
  if (pe && (n < 1 || bits <= lo || vals || sizeof(K) != 8)) return SCD_ERR_INTERNAL;
  if (n >= (1ll << 32) - 1) return SCD_ERR_CAPACITY;  // positions are 32-bit
  // tiles are copied whole into shared memory: 16-byte aligned arrays
  if ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(vals)) & 15)
    return SCD_ERR_INTERNAL;
  int64_t nblk = (n + kRsTile - 1) / kRsTile;
  if (!sc.keys_alt.ensure(sizeof(K) * (size_t)n, st)) return SCD_ERR_OOM;
  if (vals && !sc.vals_alt.ensure((size_t)n, st)) return SCD_ERR_OOM;
  if (!sc.counts.ensure((size_t)(256 * nblk + 256), st)) return SCD_ERR_OOM;
  uint32_t *counts = sc.counts.p;
  uint32_t *totals = sc.counts.p + 256 * nblk;
  K *ka = keys, *kb = (K *)sc.keys_alt.p;
  uint32_t *va = vals, *vb = sc.vals_alt.p;
  // two tile buffers of keys (and values); persistent grid of the blocks
  // that fit at once
  size_t smem = 2 * (sizeof(K) * kRsTile + (vals ? sizeof(uint32_t) * kRsTile : 0));
  static int grid_of[2][2] = {{0, 0}, {0, 0}};
  int ki = sizeof(K) == 8 ? 1 : 0, vi = vals ? 1 : 0;
  if (!grid_of[ki][vi]) {
    int sms = 0, per_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (vals) {
      cudaFuncSetAttribute(k_rs_downsweep<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rs_downsweep<K, true>, kRsThreads,
                                                    smem);
    } else {
      cudaFuncSetAttribute(k_rs_downsweep<K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rs_downsweep<K, false>,
                                                    kRsThreads, smem);
    }
    grid_of[ki][vi] = std::max(1, sms) * std::max(1, per_sm);
  }
  const unsigned grid = (unsigned)std::min<int64_t>(nblk, grid_of[ki][vi]);
  uint32_t *ocounts = nullptr, *ototals = nullptr;
  if (pe) {
    if (!sc.ocounts.ensure((size_t)(256 * nblk + 256), st)) return SCD_ERR_OOM;
    ocounts = sc.ocounts.p;
    ototals = sc.ocounts.p + 256 * nblk;
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_rs_downsweep<unsigned long long, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr = true;
    }
  }
  int passes = 0;
  for (int shift = lo; shift < bits; shift += 8, ++passes) {
    if (pe && shift + 8 >= bits) {
      // the last pass: decoded pairs to their sorted positions
      const unsigned long long tmask = (1ull << pe->tb) - 1ull;
      k_rs_upsweep<unsigned long long, true><<<(unsigned)nblk, kRsThreads, 0, st>>>(
          (const unsigned long long *)ka, n, d_n, shift, counts, nblk, ocounts, tmask);
      k_rs_scan<<<256, 1024, 0, st>>>(counts, nblk, totals, d_n, n);
      k_rs_scan<<<256, 1024, 0, st>>>(ocounts, nblk, ototals, d_n, n);
      k_rs_downsweep<unsigned long long, false, true><<<grid, kRsThreads, smem, st>>>(
          (const unsigned long long *)ka, nullptr, nullptr, nullptr, n, d_n, shift, counts,
          totals, nblk, sc.err, 0, ocounts, ototals, *pe);
      note_launch(4);
      return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
    }
    k_rs_upsweep<K><<<(unsigned)nblk, kRsThreads, 0, st>>>(ka, n, d_n, shift, counts, nblk);
    k_rs_scan<<<256, 1024, 0, st>>>(counts, nblk, totals, d_n, n);
    if (vals)
      k_rs_downsweep<K, true><<<grid, kRsThreads, smem, st>>>(ka, va, kb, vb, n, d_n, shift,
                                                               counts, totals, nblk, sc.err);
    else
      k_rs_downsweep<K, false><<<grid, kRsThreads, smem, st>>>(
          ka, nullptr, kb, nullptr, n, d_n, shift, counts, totals, nblk, sc.err);
    note_launch(3);
    K *t = ka; ka = kb; kb = t;
    uint32_t *tv = va; va = vb; vb = tv;
  }
  if (passes & 1) {
    cudaMemcpyAsync(keys, ka, sizeof(K) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    if (vals) cudaMemcpyAsync(vals, va, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
  }
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

// the one slot that ends an odd digit's range of the even partition: a hole
__global__ void k_partition_gaps(const uint32_t *__restrict__ totals,
                                 unsigned long long *__restrict__ out) {
  __shared__ uint32_t scanbuf[256];
  const uint32_t c = totals[threadIdx.x];
  const uint32_t at = digit_scan_excl((c + 1u) & ~1u, scanbuf);
  if (c & 1u) out[at + c] = ~0ull;
}

int radix_partition_u64(const unsigned long long *kin, unsigned long long *kout, int64_t n,
                        int shift, SortScratch &sc, uint32_t *h_totals, cudaStream_t st) {
  for (int d = 0; d < 256; ++d) h_totals[d] = 0;
  if (n <= 0) return SCD_OK;
  if (n >= (1ll << 32) - 512) return SCD_ERR_CAPACITY;
  if ((reinterpret_cast<uintptr_t>(kin) | reinterpret_cast<uintptr_t>(kout)) & 15)
    return SCD_ERR_INTERNAL;
  const int64_t nblk = (n + kRsTile - 1) / kRsTile;
  if (!sc.counts.ensure((size_t)(256 * nblk + 256), st)) return SCD_ERR_OOM;
  uint32_t *counts = sc.counts.p, *totals = sc.counts.p + 256 * nblk;
  const size_t smem = 2 * sizeof(unsigned long long) * kRsTile;
  static int grid = 0;
  if (!grid) {
    int sms = 0, per_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_rs_downsweep<unsigned long long, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rs_downsweep<unsigned long long, false>,
                                                  kRsThreads, smem);
    grid = std::max(1, sms) * std::max(1, per_sm);
  }
  k_rs_upsweep<unsigned long long><<<(unsigned)nblk, kRsThreads, 0, st>>>(kin, n, nullptr, shift,
                                                                          counts, nblk);
  k_rs_scan<<<256, 1024, 0, st>>>(counts, nblk, totals);
  k_rs_downsweep<unsigned long long, false>
      <<<(unsigned)std::min<int64_t>(nblk, grid), kRsThreads, smem, st>>>(
          kin, nullptr, kout, nullptr, n, nullptr, shift, counts, totals, nblk, sc.err, 1);
  k_partition_gaps<<<1, 256, 0, st>>>(totals, kout);
  note_launch(4);
  if (cudaMemcpyAsync(h_totals, totals, 256 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SCD_ERR_CUDA;
  return SCD_OK;
}

int radix_sort_u32(uint32_t *keys, uint32_t *vals, int64_t n, int bits, SortScratch &sc,
                   cudaStream_t st) {
  return rs_impl<uint32_t>(keys, vals, n, nullptr, 0, bits, sc, st);
}

int radix_sort_u64(unsigned long long *keys, uint32_t *vals, int64_t n, int bits,
                   SortScratch &sc, cudaStream_t st) {
  return rs_impl<unsigned long long>(keys, vals, n, nullptr, 0, bits, sc, st);
}

int radix_sort_u64(unsigned long long *keys, uint32_t *vals, int64_t n, int lo, int bits,
                   SortScratch &sc, cudaStream_t st) {
  return rs_impl<unsigned long long>(keys, vals, n, nullptr, lo, bits, sc, st);
}

void scan_u32_exclusive(uint32_t *a, int64_t n, uint32_t *total, cudaStream_t st) {
  k_rs_scan<<<1, 1024, 0, st>>>(a, n, total);
}

int sort_reserve(SortScratch &sc, int64_t n, size_t key_bytes, bool vals, cudaStream_t st) {
  int64_t nblk = (n + kRsTile - 1) / kRsTile;
  if (!sc.keys_alt.ensure(key_bytes * (size_t)n, st)) return SCD_ERR_OOM;
  if (vals && !sc.vals_alt.ensure((size_t)n, st)) return SCD_ERR_OOM;
  if (!sc.counts.ensure((size_t)(256 * nblk + 256), st)) return SCD_ERR_OOM;
  return SCD_OK;
}

int radix_sort_u64_pairs(unsigned long long *keys, int64_t n, const unsigned long long *d_n,
                         int lo, int bits, SortScratch &sc, const PairEmit &pe, cudaStream_t st) {
  return rs_impl<unsigned long long>(keys, nullptr, n, d_n, lo, bits, sc, st, &pe);
}

int radix_sort_u64_dev(unsigned long long *keys, uint32_t *vals, int64_t n_cap,
                       const unsigned long long *d_n, int lo, int bits, SortScratch &sc,
                       cudaStream_t st) {
  return rs_impl<unsigned long long>(keys, vals, n_cap, d_n, lo, bits, sc, st);
}

}  // namespace scd
