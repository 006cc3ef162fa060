// lbvh.cu -- steps A6-A7: the 4D box hierarchy.  The paper's AABB tree
// (Sec. 3.2) is built there by incremental insertion; here the whole tree
// is built at once from the Morton-sorted boxes as a binary radix tree
// (Karras 2012: node ranges and split points from the longest common key
// prefix, ties broken by index), then boxes are unioned bottom-up.
#include "scd_internal.cuh"

namespace scd {

// ---------------------------------------------------------------------------
// Gather the sorted boxes and the key of every leaf (the key of its first
// box; a leaf holds L consecutive sorted boxes).
// ---------------------------------------------------------------------------
template <class K>
__global__ void k_gather_sorted(const uint32_t *__restrict__ id, const float4 *__restrict__ lo,
                                const float4 *__restrict__ hi, const uint32_t *__restrict__ obj,
                                const K *__restrict__ keys, int64_t N, int L,
                                SBox *__restrict__ sbox,
                                uint32_t *__restrict__ sobj, K *__restrict__ leafkey,
                                uint32_t *__restrict__ posof, int cell_shift,
                                uint32_t *__restrict__ scell) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  uint32_t b = id[p];
  sbox[p].lo = lo[b];
  sbox[p].hi = hi[b];
  sobj[p] = obj[b];
  // a box referenced from several cells: any copy will do, their data agree
  if (posof) posof[b] = (uint32_t)p;
  if (scell) scell[p] = (uint32_t)((unsigned long long)keys[p] >> cell_shift);
  if (p % L == 0) leafkey[p / L] = keys[p];
}

// Sorted positions of each box's previous and next segment of the same
// object (-1 at the ends of the horizon).  Adjacent segments lie close in
// space and time, so these positions stay near p in the Morton order.
__global__ void k_neighbors(const uint32_t *__restrict__ id, const uint32_t *__restrict__ obj,
                            const uint32_t *__restrict__ posof, int64_t Nq, int64_t nbox,
                            int2 *__restrict__ nb) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Nq) return;
  uint32_t u = id[p];
  uint32_t o = obj[u];
  int prev = (u > 0 && obj[u - 1] == o) ? (int)posof[u - 1] : -1;
  int next = ((int64_t)u + 1 < nbox && obj[u + 1] == o) ? (int)posof[u + 1] : -1;
  nb[p] = make_int2(prev, next);
}

template <class K>
__device__ __forceinline__ int clz_key(K x);
template <>
__device__ __forceinline__ int clz_key<uint32_t>(uint32_t x) { return __clz(x); }
template <>
__device__ __forceinline__ int clz_key<unsigned long long>(unsigned long long x) {
  return __clzll(x);
}

// longest common prefix of leaves i and j; -1 outside [0, M)
template <class K>
__device__ __forceinline__ int delta(const K *__restrict__ keys, int64_t M, int64_t i, int64_t j) {
  if (j < 0 || j >= M) return -1;
  K a = keys[i], b = keys[j];
  if (a != b) return clz_key<K>(a ^ b);
  return (int)(8 * sizeof(K)) + __clz((uint32_t)(i ^ j));
}

// the leaf count: the host's, or (refinement rounds) the smaller of a
// device count and the capacity the grid was sized for
__device__ __forceinline__ int64_t leaf_count(int64_t M, const unsigned long long *d_M) {
  if (!d_M) return M;
  const unsigned long long v = *d_M;
  return v < (unsigned long long)M ? (int64_t)v : M;
}

template <class K>
__global__ void k_karras(const K *__restrict__ keys, int64_t M, TravNode *__restrict__ nodes,
                         int32_t *__restrict__ parent_int, int32_t *__restrict__ parent_leaf,
                         uint32_t *__restrict__ flags, int32_t *__restrict__ first_out,
                         const unsigned long long *__restrict__ d_M = nullptr) {
  M = leaf_count(M, d_M);
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M - 1) return;
  // direction of the node's range
  int dn = delta(keys, M, i, i + 1), dp = delta(keys, M, i, i - 1);
  int64_t d = dn > dp ? 1 : -1;
  int dmin = d > 0 ? dp : dn;
  // upper bound of the range length, then binary search for the other end
  int64_t lmax = 2;
  while (delta(keys, M, i, i + lmax * d) > dmin) lmax <<= 1;
  int64_t l = 0;
  for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(keys, M, i, i + (l + t) * d) > dmin) l += t;
  int64_t j = i + l * d;
  int dnode = delta(keys, M, i, j);
  // split: the last position that shares more than dnode bits with i
  int64_t s = 0;
  int64_t t = l;
  do {
    t = (t + 1) >> 1;
    if (delta(keys, M, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
  int64_t first = i < j ? i : j, last = i < j ? j : i;
  // the links only: the child boxes are written by the refit
  int4 lk;
  lk.x = first == gamma ? (int32_t)gamma | kLeafBit : (int32_t)gamma;
  lk.y = last == gamma + 1 ? (int32_t)(gamma + 1) | kLeafBit : (int32_t)(gamma + 1);
  lk.z = (int32_t)gamma;
  lk.w = (int32_t)last;
  reinterpret_cast<int4 *>(nodes + i)[4] = lk;
  if (first == gamma) parent_leaf[gamma] = (int32_t)i; else parent_int[gamma] = (int32_t)i;
  if (last == gamma + 1) parent_leaf[gamma + 1] = (int32_t)i;
  else parent_int[gamma + 1] = (int32_t)i | kRightChildBit;
  if (i == 0) parent_int[0] = -1;
  flags[i] = 0;
  if (first_out) first_out[i] = (int32_t)first;
}

__device__ __forceinline__ float4 f4min(float4 a, float4 b) {
  return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), fminf(a.w, b.w));
}
__device__ __forceinline__ float4 f4max(float4 a, float4 b) {
  return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z), fmaxf(a.w, b.w));
}

// Bottom-up union.  The second thread to reach a node (atomic arrival count)
// reads both children and goes on; the first one stops.  Nobody waits.
// With one box per leaf the sorted boxes are the leaf boxes.  This pass
// serves the float nodes (several boxes per leaf) and the four-wide ones;
// binary compact nodes take k_refit_q below.
template <bool kWide>
__global__ void k_refit(const SBox *__restrict__ sbox, int64_t N, int L, int64_t M,
                        float4 *__restrict__ leaflo, float4 *__restrict__ leafhi,
                        TravNode *__restrict__ nodes, float4 *__restrict__ nlo,
                        float4 *__restrict__ nhi, const int32_t *__restrict__ parent_int,
                        const int32_t *__restrict__ parent_leaf, uint32_t *__restrict__ flags,
                        W4Node *__restrict__ w4, const DevCounters *__restrict__ ctr,
                        int64_t T) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= M) return;
  const QFrame fr = scene_frame(ctr, T);
  if (L > 1) {
    int64_t b0 = c * L, b1 = b0 + L < N ? b0 + L : N;
    float4 lo = sbox[b0].lo, hi = sbox[b0].hi;
    for (int64_t b = b0 + 1; b < b1; ++b) {
      lo = f4min(lo, sbox[b].lo);
      hi = f4max(hi, sbox[b].hi);
    }
    leaflo[c] = lo;
    leafhi[c] = hi;
  }
  auto leaf_box = [&](int32_t q, float4 &lo, float4 &hi) {
    if (L == 1) {
      lo = __ldcg(&sbox[q].lo);
      hi = __ldcg(&sbox[q].hi);
    } else {
      lo = __ldcg(leaflo + q);
      hi = __ldcg(leafhi + q);
    }
  };
  if (M == 1) return;
  int32_t p = parent_leaf[c];
  while (p >= 0) {
    // release this thread's node box, acquire the sibling's (the second
    // thread to arrive reads both)
    uint32_t arrived;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                 : "=r"(arrived)
                 : "l"(flags + p)
                 : "memory");
    if (arrived == 0u) return;
    // the links only (the boxes are what this pass writes)
    const int4 lk = __ldcg(reinterpret_cast<const int4 *>(nodes + p) + 4);
    float4 llo, lhi, rlo, rhi;
    if (lk.x & kLeafBit) {
      leaf_box(lk.x & ~kLeafBit, llo, lhi);
    } else {
      llo = __ldcg(nlo + lk.x);
      lhi = __ldcg(nhi + lk.x);
    }
    if (lk.y & kLeafBit) {
      leaf_box(lk.y & ~kLeafBit, rlo, rhi);
    } else {
      rlo = __ldcg(nlo + lk.y);
      rhi = __ldcg(nhi + lk.y);
    }
    const int32_t up = parent_int[p];  // -1 at the root; bit 30: p is a right child
    if constexpr (kWide) {
      // four-wide nodes: p's children go into its parent's node (slots 0-1
      // or 2-3 by p's side), p's leaf children into p's own node
      const QBox ql = quantize_box(fr, llo, lhi), qr = quantize_box(fr, rlo, rhi);
      const uint32_t g = (uint32_t)lk.z;
      const uint2 linkl = make_uint2(g | ((lk.x & kLeafBit) ? kW4Leaf : 0u), g);
      const uint2 linkr = make_uint2((g + 1) | ((lk.y & kLeafBit) ? kW4Leaf : 0u), (uint32_t)lk.w);
      if (up >= 0) {
        W4Node &pn = w4[up & ~kRightChildBit];
        const int s = (up & kRightChildBit) ? 2 : 0;
        pn.box[s] = ql;
        pn.box[s + 1] = qr;
        pn.link[s] = linkl;
        pn.link[s + 1] = linkr;
      }
      const QBox empty = {0xffffffffu, 0xffffffffu, 0u, 0u};
      const uint2 none = make_uint2(kW4Empty, 0u);
      if (lk.x & kLeafBit) {
        w4[p].box[0] = ql;
        w4[p].link[0] = linkl;
        w4[p].box[1] = empty;
        w4[p].link[1] = none;
      }
      if (lk.y & kLeafBit) {
        w4[p].box[2] = qr;
        w4[p].link[2] = make_uint2((g + 1) | kW4Leaf, g + 1);
        w4[p].box[3] = empty;
        w4[p].link[3] = none;
      }
    } else {
      float4 *np = reinterpret_cast<float4 *>(nodes + p);
      np[0] = llo;
      np[1] = lhi;
      np[2] = rlo;
      np[3] = rhi;
    }
    __stcg(nlo + p, f4min(llo, rlo));
    __stcg(nhi + p, f4max(lhi, rhi));
    p = up >= 0 ? (up & ~kRightChildBit) : -1;
  }
}

// the union of two quantised boxes: per field, the lower corner's minimum
// and the upper corner's maximum (x, y in 16-bit lanes, then z | t << 15)
__device__ __forceinline__ QBox qbox_union(const QBox &a, const QBox &b) {
  QBox u;
  u.lo_xy = __vminu2(a.lo_xy, b.lo_xy);
  u.hi_xy = __vmaxu2(a.hi_xy, b.hi_xy);
  u.lo_zt = min(a.lo_zt & 0x7fffu, b.lo_zt & 0x7fffu) | (min(a.lo_zt >> 15, b.lo_zt >> 15) << 15);
  u.hi_zt = max(a.hi_zt & 0x7fffu, b.hi_zt & 0x7fffu) | (max(a.hi_zt >> 15, b.hi_zt >> 15) << 15);
  return u;
}

// The refit of binary compact nodes (one box per leaf) in the quantised
// frame: a node's quantised box is the union of its children's.  Outward
// quantisation is monotone per coordinate, so that union equals the
// quantised union of the exact boxes, bit for bit, at half the bytes per
// node (16 instead of 32).
// One compact node's work in the refit: both children's quantised boxes
// into the node's pair, the split with the leaf flags, and the union as the
// node's own box for its parent.
__device__ __forceinline__ void refit_q_node(const SBox *__restrict__ sbox, const QFrame &fr,
                                             int32_t p, const int4 &lk, QBox *__restrict__ nq,
                                             QBox *__restrict__ qbox,
                                             uint32_t *__restrict__ qlink) {
  auto child = [&](int32_t link) {
    if (link & kLeafBit) {
      const int32_t q = link & ~kLeafBit;
      return quantize_box(fr, __ldcg(&sbox[q].lo), __ldcg(&sbox[q].hi));
    }
    const uint4 v = __ldcg(reinterpret_cast<const uint4 *>(nq + link));
    return QBox{v.x, v.y, v.z, v.w};
  };
  const QBox ql = child(lk.x), qr = child(lk.y);
  qbox[2 * p] = ql;
  qbox[2 * p + 1] = qr;
  const uint32_t g = (uint32_t)lk.z;  // the split: left child gamma, right gamma + 1
  const uint32_t fl =
      ((lk.x & kLeafBit) ? kQLeftLeaf : 0u) | ((lk.y & kLeafBit) ? kQRightLeaf : 0u);
  qlink[p] = g | fl;
  const QBox u = qbox_union(ql, qr);
  __stcg(reinterpret_cast<uint4 *>(nq + p), make_uint4(u.lo_xy, u.lo_zt, u.hi_xy, u.hi_zt));
}

// the arrival at node p: true for the second thread to arrive, which then
// sees its sibling's writes (acquire) after releasing its own
__device__ __forceinline__ bool arrive_gpu(uint32_t *flags, int32_t p) {
  uint32_t arrived;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
               : "=r"(arrived)
               : "l"(flags + p)
               : "memory");
  return arrived != 0u;
}

__global__ void k_refit_q(const SBox *__restrict__ sbox, int64_t M,
                          const TravNode *__restrict__ nodes, QBox *__restrict__ nq,
                          const int32_t *__restrict__ parent_int,
                          const int32_t *__restrict__ parent_leaf, uint32_t *__restrict__ flags,
                          QBox *__restrict__ qbox, uint32_t *__restrict__ qlink,
                          const DevCounters *__restrict__ ctr, int64_t T,
                          const unsigned long long *__restrict__ d_M = nullptr) {
  M = leaf_count(M, d_M);
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= M || M == 1) return;
  const QFrame fr = scene_frame(ctr, T);
  int32_t p = parent_leaf[c];
  while (p >= 0) {
    if (!arrive_gpu(flags, p)) return;
    const int4 lk = __ldcg(reinterpret_cast<const int4 *>(nodes + p) + 4);
    refit_q_node(sbox, fr, p, lk, nq, qbox, qlink);
    const int32_t up = parent_int[p];
    p = up >= 0 ? (up & ~kRightChildBit) : -1;
  }
}

// The same refit with the lower levels kept inside a block: block b takes
// the kRqChunk leaves [c0, c1) and, for the nodes whose leaf range lies
// inside them (the node's index lies there too: it is one end of its
// range), counts arrivals in shared memory and orders the two threads'
// writes with block-scope fences.  Only the nodes whose range crosses a
// chunk boundary (a few per cent) take the device-scope atomics.  The
// block-scope message passing and the device-scope one compose (fences are
// cumulative), so a node's union reaches whichever block completes its
// parent.
constexpr int kRqThreads = 256, kRqChunk = 8 * kRqThreads;
__global__ void __launch_bounds__(kRqThreads) k_refit_q_local(
    const SBox *__restrict__ sbox, int64_t M, const TravNode *__restrict__ nodes,
    const int32_t *__restrict__ nfirst, QBox *__restrict__ nq,
    const int32_t *__restrict__ parent_int, const int32_t *__restrict__ parent_leaf,
    uint32_t *__restrict__ flags, QBox *__restrict__ qbox, uint32_t *__restrict__ qlink,
    const DevCounters *__restrict__ ctr, int64_t T) {
  __shared__ uint32_t arr[kRqChunk];  // arrivals at the block's own nodes, by index - c0
  for (int i = threadIdx.x; i < kRqChunk; i += kRqThreads) arr[i] = 0u;
  __syncthreads();
  if (M == 1) return;
  const int64_t c0 = (int64_t)blockIdx.x * kRqChunk;
  const int64_t c1 = c0 + kRqChunk < M ? c0 + kRqChunk : M;
  const QFrame fr = scene_frame(ctr, T);
  for (int k = 0; k < kRqChunk / kRqThreads; ++k) {
    const int64_t c = c0 + (int64_t)k * kRqThreads + threadIdx.x;
    if (c >= c1) break;
    int32_t p = parent_leaf[c];
    while (p >= 0) {
      const int4 lk = __ldcg(reinterpret_cast<const int4 *>(nodes + p) + 4);
      const bool local = nfirst[p] >= c0 && (int64_t)lk.w < c1;
      if (local) {
        __threadfence_block();
        const bool second = atomicAdd(&arr[p - c0], 1u) != 0u;
        if (!second) break;
        __threadfence_block();
      } else if (!arrive_gpu(flags, p)) {
        break;
      }
      refit_q_node(sbox, fr, p, lk, nq, qbox, qlink);
      const int32_t up = parent_int[p];
      p = up >= 0 ? (up & ~kRightChildBit) : -1;
    }
  }
}

template <class K>
int build_tree(scd_scene *s, const K *keys_sorted, const uint32_t *ids_sorted, int64_t Nq,
               K *leafkey, int cell_shift, int64_t &M) {
  cudaStream_t st = s->stream;
  int L = s->tune.leaf_size;
  M = (Nq + L - 1) / L;
  if (!s->s_box.ensure(Nq, st) || !s->s_obj.ensure(Nq, st) ||
      (L > 1 && (!s->d_leaflo.ensure(M, st) || !s->d_leafhi.ensure(M, st))) ||
      !s->d_nodes.ensure(M > 1 ? M - 1 : 1, st) || !s->d_nlo.ensure(M > 1 ? M - 1 : 1, st) ||
      !s->d_nhi.ensure(M > 1 ? M - 1 : 1, st) || !s->d_parent_int.ensure(M, st) ||
      !s->d_parent_leaf.ensure(M, st) || !s->d_flags.ensure(M, st))
    return SCD_ERR_OOM;
  const bool compact = L == 1;
  const bool cells = cell_shift >= 0;
  const bool wide = compact && s->tune.node_width == 4;
  if (compact && !wide && (!s->d_qbox.ensure(2 * (M > 1 ? M - 1 : 1), st) ||
                           !s->d_qlink.ensure(M > 1 ? M - 1 : 1, st)))
    return SCD_ERR_OOM;
  if (wide && !s->d_w4.ensure(M > 1 ? M - 1 : 1, st)) return SCD_ERR_OOM;
  if (compact && (!s->d_posof.ensure(s->N, st) || !s->s_nb.ensure(Nq, st))) return SCD_ERR_OOM;
  if (cells && (!s->s_cell.ensure(Nq, st) || !s->d_first.ensure(M > 1 ? M - 1 : 1, st)))
    return SCD_ERR_OOM;
  int bs = 256;
  k_gather_sorted<K><<<(unsigned)((Nq + bs - 1) / bs), bs, 0, st>>>(
      ids_sorted, s->d_lo.p, s->d_hi.p, s->d_obj.p, keys_sorted, Nq, L, s->s_box.p,
      s->s_obj.p, leafkey, compact ? s->d_posof.p : nullptr, cell_shift,
      cells ? s->s_cell.p : nullptr);
  note_launch(2);
  if (compact) {
    k_neighbors<<<(unsigned)((Nq + bs - 1) / bs), bs, 0, st>>>(ids_sorted, s->d_obj.p,
                                                               s->d_posof.p, Nq, s->N, s->s_nb.p);
    note_launch();
  }
  // the nodes' first leaves: the cells' roots, and the block-local refit
  const bool want_first = cells || (compact && !wide);
  if (want_first && !s->d_first.ensure(M > 1 ? M - 1 : 1, st)) return SCD_ERR_OOM;
  if (M > 1) {
    k_karras<K><<<(unsigned)((M - 1 + bs - 1) / bs), bs, 0, st>>>(
        leafkey, M, s->d_nodes.p, s->d_parent_int.p, s->d_parent_leaf.p, s->d_flags.p,
        want_first ? s->d_first.p : nullptr);
    note_launch();
  }
  static_assert(sizeof(QBox) == sizeof(float4), "the quantised node boxes use the float ones' buffer");
  if (compact && !wide) {
    k_refit_q_local<<<(unsigned)((M + kRqChunk - 1) / kRqChunk), kRqThreads, 0, st>>>(
        s->s_box.p, M, s->d_nodes.p, s->d_first.p, reinterpret_cast<QBox *>(s->d_nlo.p),
        s->d_parent_int.p, s->d_parent_leaf.p, s->d_flags.p, s->d_qbox.p, s->d_qlink.p,
        s->d_ctr.p, s->T);
  } else {
    (wide ? k_refit<true> : k_refit<false>)<<<(unsigned)((M + bs - 1) / bs), bs, 0, st>>>(
        s->s_box.p, Nq, L, M, s->d_leaflo.p, s->d_leafhi.p, s->d_nodes.p, s->d_nlo.p,
        s->d_nhi.p, s->d_parent_int.p, s->d_parent_leaf.p, s->d_flags.p,
        wide ? s->d_w4.p : nullptr, s->d_ctr.p, s->T);
  }
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

template int build_tree<uint32_t>(scd_scene *, const uint32_t *, const uint32_t *, int64_t,
                                  uint32_t *, int, int64_t &);
template int build_tree<unsigned long long>(scd_scene *, const unsigned long long *,
                                            const uint32_t *, int64_t, unsigned long long *, int,
                                            int64_t &);

// The hierarchy of one refinement round: up to cap boxes already sorted
// along the Morton curve (keys and boxes in sorted order), their count on
// the device.  Karras links, then compact quantised nodes (one box per
// leaf) in the frame of the scene's extent and a horizon of T ticks.
int build_round_tree(const unsigned long long *keys, const SBox *sbox, int64_t cap,
                     const unsigned long long *d_M, TravNode *nodes, int32_t *parent_int,
                     int32_t *parent_leaf, uint32_t *arrive, QBox *nq, QBox *qbox,
                     uint32_t *qlink, const DevCounters *ctr, int64_t T, cudaStream_t st) {
  const int bs = 256;
  if (cap < 2) return SCD_OK;
  k_karras<unsigned long long><<<(unsigned)((cap - 1 + bs - 1) / bs), bs, 0, st>>>(
      keys, cap, nodes, parent_int, parent_leaf, arrive, nullptr, d_M);
  k_refit_q<<<(unsigned)((cap + bs - 1) / bs), bs, 0, st>>>(sbox, cap, nodes, nq, parent_int,
                                                           parent_leaf, arrive, qbox, qlink,
                                                           ctr, T, d_M);
  note_launch(2);
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

int build_hierarchy(scd_scene *s, int64_t &n_leaves) {
  int64_t Mx = (s->N + s->tune.leaf_size - 1) / s->tune.leaf_size;
  if (s->tune.morton_bits > 8) {
    if (!s->s_leafkey64.ensure(Mx, s->stream)) return SCD_ERR_OOM;
    return build_tree<unsigned long long>(s, s->d_key64.p, s->d_id.p, s->N, s->s_leafkey64.p, -1,
                                          n_leaves);
  }
  if (!s->s_leafkey32.ensure(Mx, s->stream)) return SCD_ERR_OOM;
  return build_tree<uint32_t>(s, s->d_key32.p, s->d_id.p, s->N, s->s_leafkey32.p, -1, n_leaves);
}

}  // namespace scd
