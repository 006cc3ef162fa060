// decomp.cu -- step A10: the paper's static decomposition of the search
// (Sec. 5: independent sub-problems from an edge partition of the
// potential-collision graph; Sec. 6.1: altitude bands), run on one GPU as
// independent subtrees of one sorted reference array, traversed in one
// persistent launch.
//
// A box is referenced from every cell it touches.  Keys are (cell, Morton):
// one sort groups each cell's references, and in the radix tree over them
// every cell is a subtree, whose root the traversal starts from.  A pair of
// boxes is reported only in the cell that holds a reference point common to
// both, so it is reported once:
//   SLAB_OCT   cells = n_slabs equal tick slabs x 8 ECI sign octants; the
//              point is the lower corner of the two boxes' intersection
//              (half-open cells: a coordinate 0 belongs to the upper half).
//              The output equals the undecomposed one exactly.
//   ALT_BANDS  cells = p altitude bands with edges at every floor(n/p)-th
//              sorted semi-major axis (Sec. 6.1); an object is in every band
//              that its radial range [a(1-e) - sqrt3 r, a(1+e) + sqrt3 r]
//              meets; two objects are joined in the potential-collision
//              graph (Def 9) iff their ranges intersect, and the point is the
//              lower end of that intersection.
#include <algorithm>

#include "scd_internal.cuh"

namespace scd {

struct DecompArgs {
  int kind;
  int n_slabs;
  int p;              // bands
  int64_t T;
  const double2 *rr;  // radial ranges (ALT_BANDS)
  const double *edges;
  const int32_t *objscene;  // scene of each object (a batch of scenes)
  const int32_t *objT;      // horizon of each object's scene [ticks] (a batch)
};

__global__ void k_radial(const scd_element *__restrict__ el, int64_t n, double2 *__restrict__ rr,
                         unsigned long long *__restrict__ abits) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  scd_element x = el[i];
  // the same operations, in the same order, as the oracle's radial range
  double pad = __dmul_rn(1.7320508075688772, x.radius_km);
  double lo = __dsub_rn(__dmul_rn(x.a_km, __dsub_rn(1.0, x.e)), pad);
  double hi = __dadd_rn(__dmul_rn(x.a_km, __dadd_rn(1.0, x.e)), pad);
  rr[i] = make_double2(lo, hi);
  abits[i] = (unsigned long long)__double_as_longlong(x.a_km);  // a > 0: bit order = value order
}

__global__ void k_band_edges(const unsigned long long *__restrict__ asorted, int64_t n, int p,
                             double *__restrict__ edges) {
  int k = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (k >= p) return;
  int64_t d = n / p;
  edges[k - 1] = __longlong_as_double((long long)asorted[(int64_t)k * d]);
}

// the cells a box touches: slabs s0..s1 x the octant halves on each axis
struct CellSpan {
  int s0, s1, x0, x1, y0, y1, z0, z1;  // SLAB_OCT
  int b0, b1;                          // ALT_BANDS
};

__device__ __forceinline__ CellSpan cell_span(const DecompArgs &d, float4 lo, float4 hi,
                                              uint32_t obj) {
  CellSpan c;
  if (d.kind == SCD_DECOMP_SLAB_OCT) {
    c.s0 = slab_of((int64_t)lo.w, d.n_slabs, d.T);
    c.s1 = slab_of((int64_t)hi.w, d.n_slabs, d.T);
    c.x0 = lo.x >= 0.f ? 1 : 0;
    c.x1 = hi.x >= 0.f ? 1 : 0;
    c.y0 = lo.y >= 0.f ? 1 : 0;
    c.y1 = hi.y >= 0.f ? 1 : 0;
    c.z0 = lo.z >= 0.f ? 1 : 0;
    c.z1 = hi.z >= 0.f ? 1 : 0;
    c.b0 = c.b1 = 0;
  } else if (d.kind == kDecompScenes) {
    c.b0 = c.b1 = d.objscene[obj];  // a scene is one cell
    c.s0 = c.s1 = c.x0 = c.x1 = c.y0 = c.y1 = c.z0 = c.z1 = 0;
  } else {
    double2 r = d.rr[obj];
    c.b0 = band_of(r.x, d.edges, d.p);
    c.b1 = band_of(r.y, d.edges, d.p);
    c.s0 = c.s1 = c.x0 = c.x1 = c.y0 = c.y1 = c.z0 = c.z1 = 0;
  }
  return c;
}

__global__ void k_ref_count(const float4 *__restrict__ lo, const float4 *__restrict__ hi,
                            const uint32_t *__restrict__ obj, int64_t N, DecompArgs d,
                            int64_t *__restrict__ cnt) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= N) return;
  CellSpan c = cell_span(d, lo[b], hi[b], obj[b]);
  if (d.kind == SCD_DECOMP_SLAB_OCT)
    cnt[b] = (int64_t)(c.s1 - c.s0 + 1) * (c.x1 - c.x0 + 1) * (c.y1 - c.y0 + 1) *
             (c.z1 - c.z0 + 1);
  else
    cnt[b] = c.b1 - c.b0 + 1;
}

// A reference's key: its cell above the size bit (if any) above the top
// mbits bits of the box's Morton key.  The key's time frame is the cell's
// own: a tick slab's ticks, a batch scene's horizon, else the scene's.
struct RefKeyArgs {
  int bits;          // Morton bits per axis
  int mbits;         // Morton bits kept (the top ones)
  float time_scale;
  int space_warp;
  float split_km;    // 0: no size bit
};

__device__ __forceinline__ unsigned long long ref_morton(const RefKeyArgs &k, float4 L, float4 H,
                                                         float R, float t0, float T1) {
  L.w -= t0;
  H.w -= t0;
  unsigned long long m = box_morton(L, H, R, T1, k.bits, k.time_scale, k.space_warp);
  m >>= (4 * k.bits - k.mbits);
  if (k.split_km != 0.0f)
    m |= (unsigned long long)split_bit(L, H, k.split_km) << k.mbits;
  return m;
}

__global__ void k_ref_scatter(const float4 *__restrict__ lo, const float4 *__restrict__ hi,
                              const uint32_t *__restrict__ obj, int64_t N, DecompArgs d,
                              const int64_t *__restrict__ off, const DevCounters *__restrict__ ctr,
                              RefKeyArgs ka, int64_t cap,
                              unsigned long long *__restrict__ key, uint32_t *__restrict__ id) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= N) return;
  float4 L = lo[b], H = hi[b];
  const uint32_t ob = obj[b];
  CellSpan c = cell_span(d, L, H, ob);
  const float R = (float)__longlong_as_double((long long)ctr->extent_bits);
  const int cshift = ka.mbits + (ka.split_km != 0.0f ? 1 : 0);
  int64_t o = off[b];
  if (d.kind == SCD_DECOMP_SLAB_OCT) {
    const float slab = (float)(d.T + 1) / (float)d.n_slabs;
    for (int s = c.s0; s <= c.s1; ++s) {
      const unsigned long long m = ref_morton(ka, L, H, R, (float)s * slab, slab);
      for (int x = c.x0; x <= c.x1; ++x)
        for (int y = c.y0; y <= c.y1; ++y)
          for (int z = c.z0; z <= c.z1; ++z) {
            unsigned long long cell = (unsigned long long)(s * 8 + (x << 2) + (y << 1) + z);
            if (o < cap) {
              key[o] = (cell << cshift) | m;
              id[o] = (uint32_t)b;
            }
            ++o;
          }
    }
  } else {
    const float T1 = (float)((d.objT ? (int64_t)d.objT[ob] : d.T) + 1);
    const unsigned long long m = ref_morton(ka, L, H, R, 0.0f, T1);
    for (int k = c.b0; k <= c.b1; ++k) {
      if (o < cap) {
        key[o] = ((unsigned long long)k << cshift) | m;
        id[o] = (uint32_t)b;
      }
      ++o;
    }
  }
}

// First and last reference of every cell, then the root of its subtree: the
// internal node whose leaf range is exactly [first, last] (in a radix tree
// its index is one of the two ends).
__global__ void k_cell_bounds(const uint32_t *__restrict__ scell, int64_t R,
                              int32_t *__restrict__ cfirst, int32_t *__restrict__ clast) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= R) return;
  uint32_t c = scell[p];
  if (p == 0 || scell[p - 1] != c) cfirst[c] = (int32_t)p;
  if (p == R - 1 || scell[p + 1] != c) clast[c] = (int32_t)p;
}

__global__ void k_cell_roots(const int32_t *__restrict__ cfirst, const int32_t *__restrict__ clast,
                             int n_cells, const int32_t *__restrict__ first,
                             const TravNode *__restrict__ nodes, int32_t *__restrict__ root) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  int32_t f = cfirst[c], l = clast[c];
  if (f < 0 || l <= f) {
    root[c] = -1;  // empty or a single reference: no pair inside
    return;
  }
  root[c] = (first[f] == f && nodes[f].last_r == l) ? f : l;
}

int build_decomposed(scd_scene *s, const scd_decomp *dc, int64_t &M, bool capturing) {
  cudaStream_t st = s->stream;
  const int64_t N = s->N;
  DecompArgs d;
  d.kind = dc->kind;
  d.n_slabs = dc->n_slabs;
  d.p = dc->p_bands;
  d.T = s->T;
  d.rr = nullptr;
  d.edges = nullptr;
  d.objscene = s->d_objscene.p;
  d.objT = s->n_scenes > 0 ? s->d_objT.p : nullptr;
  int n_cells = d.kind == SCD_DECOMP_SLAB_OCT ? d.n_slabs * 8
                : d.kind == kDecompScenes     ? s->n_scenes
                                              : d.p;
  s->n_cells = n_cells;
  const int bs = 256;
  if (d.kind == SCD_DECOMP_ALT_BANDS) {
    if (!s->d_rr.ensure(s->n, st) || !s->d_abits.ensure(s->n, st) ||
        !s->d_edges.ensure(d.p > 1 ? d.p - 1 : 1, st))
      return SCD_ERR_OOM;
    k_radial<<<(unsigned)((s->n + bs - 1) / bs), bs, 0, st>>>(s->d_el.p, s->n, s->d_rr.p,
                                                             s->d_abits.p);
    note_launch();
    int rc = radix_sort_u64(s->d_abits.p, nullptr, s->n, 64, s->sort_sc, st);
    if (rc) return rc;
    if (d.p > 1) {
      k_band_edges<<<(unsigned)((d.p + bs - 1) / bs), bs, 0, st>>>(s->d_abits.p, s->n, d.p,
                                                                  s->d_edges.p);
      note_launch();
    }
    d.rr = s->d_rr.p;
    d.edges = s->d_edges.p;
  }
  // references: count, offsets, scatter, sort
  if (!s->d_refcnt.ensure(N, st) || !s->d_refoff.ensure(N + 1, st)) return SCD_ERR_OOM;
  k_ref_count<<<(unsigned)((N + bs - 1) / bs), bs, 0, st>>>(s->d_lo.p, s->d_hi.p, s->d_obj.p, N,
                                                            d, s->d_refcnt.p);
  note_launch();
  int rc = scan_exclusive_i64(s->d_refcnt.p, s->d_refoff.p, N, s->d_scan_tmp, st);
  if (rc) return rc;
  // the reference total goes to the counters (checked after a graph replay)
  if (cudaMemcpyAsync(&s->d_ctr.p->refs_total, s->d_refoff.p + N, sizeof(int64_t),
                      cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SCD_ERR_CUDA;
  int64_t R = s->n_refs;  // inside a capture: the size the graph is built for
  if (!capturing) {
    if (cudaMemcpyAsync(&s->h_ctr_pinned->refs_total, s->d_refoff.p + N, sizeof(int64_t),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return SCD_ERR_CUDA;
    R = (int64_t)s->h_ctr_pinned->refs_total;
    if (R <= 0 || R >= (1ll << 30)) return SCD_ERR_CAPACITY;
    s->n_refs = R;
  }
  if (!s->d_refkey.ensure(R, st) || !s->d_refid.ensure(R, st) ||
      !s->s_leafkey64.ensure(R, st) || !s->d_cellroot.ensure(n_cells, st) ||
      !s->d_refcnt.ensure(2 * (size_t)n_cells > (size_t)N ? 2 * n_cells : N, st))
    return SCD_ERR_OOM;
  // the cell's bits above the size bit and as many of the Morton key's top
  // bits as the rest of 64 holds
  int cbits = 1;
  while ((1 << cbits) < n_cells) ++cbits;
  RefKeyArgs ka;
  ka.bits = s->tune.morton_bits;
  ka.time_scale = s->tune.time_scale;
  ka.space_warp = s->tune.space_warp;
  ka.split_km = s->tune.split_km;
  const int sb = ka.split_km != 0.0f ? 1 : 0;
  ka.mbits = std::min(4 * ka.bits, 64 - cbits - sb);
  k_ref_scatter<<<(unsigned)((N + bs - 1) / bs), bs, 0, st>>>(
      s->d_lo.p, s->d_hi.p, s->d_obj.p, N, d, s->d_refoff.p, s->d_ctr.p, ka, R, s->d_refkey.p,
      s->d_refid.p);
  note_launch();
  const int cshift = ka.mbits + sb;
  rc = radix_sort_u64(s->d_refkey.p, s->d_refid.p, R, cshift + cbits, s->sort_sc, st);
  if (rc) return rc;
  rc = build_tree<unsigned long long>(s, s->d_refkey.p, s->d_refid.p, R, s->s_leafkey64.p, cshift,
                                      M);
  if (rc) return rc;
  // cell bounds (reusing the count buffer as two int32 arrays) and roots
  int32_t *cfirst = (int32_t *)s->d_refcnt.p, *clast = cfirst + n_cells;
  cudaMemsetAsync(cfirst, 0xff, sizeof(int32_t) * 2 * (size_t)n_cells, st);
  k_cell_bounds<<<(unsigned)((R + bs - 1) / bs), bs, 0, st>>>(s->s_cell.p, R, cfirst, clast);
  k_cell_roots<<<(unsigned)((n_cells + bs - 1) / bs), bs, 0, st>>>(
      cfirst, clast, n_cells, s->d_first.p, s->d_nodes.p, s->d_cellroot.p);
  note_launch(2);
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

}  // namespace scd
