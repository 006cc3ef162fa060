// propagate.cu -- steps A1-A4 of the screen: per-object step policy, FP64
// two-body propagation (Sec. 6.1, Eq. 1 solved through Kepler's equation),
// interval occupancy boxes (Def 7, Def 8, Sec. 4.5) rounded outward to FP32,
// and the 4D Morton key of every box.
#include <math.h>

#include <mutex>

#include "kepler.cuh"
#include "scd_internal.cuh"

namespace scd {

// ---------------------------------------------------------------------------
// A1: per-object constants and step length.  The period and the step are
// evaluated with explicitly rounded operations in a fixed order, so that the
// integer step floor(P / (f dt)) is a reproducible decision.
// ---------------------------------------------------------------------------
struct StepArgs {
  int kind;
  uint32_t fixed;
  double frac;
  double tick_s;
  int64_t T;
  const double *band;  // n_bands-1 edges, then n_bands fractions
  int n_bands;
  const float *learned_k;  // per-object learned step [s] (LEARNED), or null
  const int32_t *objT;     // per-object horizon [ticks] (batches of scenes), or null
};

__global__ void k_prepare_objects(const scd_element *__restrict__ el, int64_t n, StepArgs sa,
                                  ObjParams *__restrict__ par, int32_t *__restrict__ kout,
                                  int64_t *__restrict__ segcnt, DevCounters *ctr) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (sa.objT) sa.T = sa.objT[i];  // this object's own scene horizon
  scd_element x = el[i];
  bool ok = x.a_km > 0.0 && x.e >= 0.0 && x.e < 1.0 && x.radius_km >= 0.0 &&
            isfinite(x.a_km) && isfinite(x.e) && isfinite(x.inc_rad) && isfinite(x.raan_rad) &&
            isfinite(x.argp_rad) && isfinite(x.M0_rad) && isfinite(x.radius_km);
  if (!ok) {
    atomicOr(&ctr->build_flags, ERR_INVALID);
    kout[i] = 1;
    segcnt[i] = sa.T + 1;
    return;
  }
  double a = x.a_km, e = x.e;
  double a3 = __dmul_rn(__dmul_rn(a, a), a);
  double P = __dmul_rn(kTwoPi, __dsqrt_rn(__ddiv_rn(a3, kMu)));
  double nmot = sqrt(kMu / a3);
  double vmax = __dsqrt_rn(__ddiv_rn(__dmul_rn(__ddiv_rn(kMu, a), __dadd_rn(1.0, e)),
                                     __dsub_rn(1.0, e)));

  int64_t k = 1;
  if (sa.kind == SCD_STEP_FIXED) {
    k = sa.fixed < 1 ? 1 : (int64_t)sa.fixed;
  } else {
    double f = sa.frac;
    if (sa.kind == SCD_STEP_BAND_TABLE) {
      double hp = __dsub_rn(__dmul_rn(a, __dsub_rn(1.0, e)), kRe);
      int b = 0;
      while (b < sa.n_bands - 1 && hp >= sa.band[b]) ++b;
      f = sa.band[sa.n_bands - 1 + b];
    }
    double q;
    if (sa.kind == SCD_STEP_LEARNED && sa.learned_k) {
      q = floor((double)sa.learned_k[i] / sa.tick_s);
    } else {
      q = floor(__ddiv_rn(P, __dmul_rn(f, sa.tick_s)));
    }
    k = q < 1.0 ? 1 : (q > (double)(sa.T + 1) ? sa.T + 1 : (int64_t)q);
  }

  // perifocal axes in ECI: rotate by argp about z, inc about x, RAAN about z
  double sO, cO, sw, cw, si, ci;
  sincos(x.raan_rad, &sO, &cO);
  sincos(x.argp_rad, &sw, &cw);
  sincos(x.inc_rad, &si, &ci);
  double Px = cO * cw - sO * sw * ci, Py = sO * cw + cO * sw * ci, Pz = sw * si;
  double Qx = -cO * sw - sO * cw * ci, Qy = -sO * sw + cO * cw * ci, Qz = cw * si;
  double b = a * sqrt(1.0 - e * e);
  ObjParams p;
  p.A[0] = a * Px; p.A[1] = a * Py; p.A[2] = a * Pz;
  p.B[0] = b * Qx; p.B[1] = b * Qy; p.B[2] = b * Qz;
  p.n = nmot;
  p.M0 = x.M0_rad;
  p.e = e;
  p.vmax = vmax;
  p.r = x.radius_km;
  p.P = P;
  p.tolE = 1e-7 / a;
  p.dmax2 = e > 0.0 ? (float)(p.tolE * (1.0 - e) / (2.0 * e)) : INFINITY;
  p.ef = (float)e;
  par[i] = p;
  kout[i] = (int32_t)k;
  segcnt[i] = (sa.T + k) / k;  // ceil((T+1)/k)

  // extent of everything this object's boxes can reach, for key scaling
  double ext = a * (1.0 + e) * 1.4142135623730951 + x.radius_km +
               vmax * (double)k * sa.tick_s * 0.5 + 1.0;
  atomicMax(&ctr->extent_bits, (unsigned long long)__double_as_longlong(ext));
}

int launch_prepare_objects(scd_scene *s) {
  StepArgs sa;
  sa.kind = s->step_kind;
  sa.fixed = s->fixed_ticks;
  sa.frac = s->period_fraction;
  sa.tick_s = s->tick_s;
  sa.T = s->T;
  sa.band = s->d_band.p;
  sa.n_bands = (int)s->band_fracs.size();
  sa.learned_k = s->step_kind == SCD_STEP_LEARNED ? s->d_learned.p : nullptr;
  sa.objT = s->n_scenes > 0 ? s->d_objT.p : nullptr;
  int bs = 256;
  int64_t g = (s->n + bs - 1) / bs;
  k_prepare_objects<<<(unsigned)g, bs, 0, s->stream>>>(s->d_el.p, s->n, sa, s->d_par.p,
                                                        s->d_k.p, s->d_segcnt.p, s->d_ctr.p);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// A2-A4: one thread per box.
// ---------------------------------------------------------------------------
struct BoxArgs {
  const ObjParams *par;
  const int32_t *k;
  const int64_t *segoff;
  int64_t n;
  int64_t N;
  int64_t T;
  float T1f;         // T + 1 (the key frame's time extent)
  double tick_s;
  int mode;
  int bits;          // Morton bits per axis
  float time_scale;  // weight of the time axis in the key
  int space_warp;    // log-compress space coordinates before quantising
  float split_km;    // large boxes sorted apart (one key bit above the Morton key)
  DevCounters *ctr;
  float4 *lo, *hi;
  uint32_t *obj;
  uint32_t *key32;
  unsigned long long *key64;
  uint32_t *id;
  const int32_t *objT;  // per-object horizon [ticks], or null
};

__device__ __forceinline__ int64_t find_object(const int64_t *segoff, int64_t n, int64_t b) {
  // largest i with segoff[i] <= b
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (__ldg(segoff + mid) <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) k_build_boxes(BoxArgs a) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.N) return;
  int64_t i = find_object(a.segoff, a.n, b);
  int64_t m = b - __ldg(a.segoff + i);
  int64_t k = __ldg(a.k + i);
  int64_t tlo = m * k;
  int64_t thi = tlo + k - 1;
  const int64_t Ti = a.objT ? (int64_t)__ldg(a.objT + i) : a.T;
  if (thi > Ti) thi = Ti;
  const ObjParams &p = a.par[i];
  double lo[3], hi[3];
  int iters = 0;
  segment_box(p, a.mode, tlo, thi, a.tick_s, lo, hi, iters);
  if (iters >= kKeplerMaxIter) atomicOr(&a.ctr->build_flags, ERR_KEPLER);
  float4 L, H;
  L.x = __double2float_rd(lo[0]);
  L.y = __double2float_rd(lo[1]);
  L.z = __double2float_rd(lo[2]);
  L.w = (float)tlo;
  H.x = __double2float_ru(hi[0]);
  H.y = __double2float_ru(hi[1]);
  H.z = __double2float_ru(hi[2]);
  H.w = (float)thi;
  a.lo[b] = L;
  a.hi[b] = H;
  a.obj[b] = (uint32_t)i;
  a.id[b] = (uint32_t)b;

  // 4D Morton key of the box centre in the scene's bounding cube
  const float R = (float)__longlong_as_double((long long)a.ctr->extent_bits);
  unsigned long long key = box_morton(L, H, R, a.T1f, a.bits, a.time_scale, a.space_warp);
  key = sort_key(key, split_bit(L, H, a.split_km), a.bits, a.split_km != 0.0f);
  if (a.key64) a.key64[b] = key;
  else a.key32[b] = (uint32_t)key;
}

int launch_build_boxes(scd_scene *s) {
  BoxArgs a;
  a.par = s->d_par.p;
  a.k = s->d_k.p;
  a.segoff = s->d_segoff.p;
  a.n = s->n;
  a.N = s->N;
  a.T = s->T;
  a.T1f = (float)(s->T + 1);
  a.tick_s = s->tick_s;
  a.mode = s->box_mode;
  a.bits = s->tune.morton_bits;
  a.time_scale = s->tune.time_scale;
  a.space_warp = s->tune.space_warp;
  a.split_km = split_of(s->tune);
  a.ctr = s->d_ctr.p;
  a.lo = s->d_lo.p;
  a.hi = s->d_hi.p;
  a.obj = s->d_obj.p;
  a.key32 = s->d_key32.p;
  a.key64 = s->tune.morton_bits > 8 ? s->d_key64.p : nullptr;
  a.id = s->d_id.p;
  a.objT = s->n_scenes > 0 ? s->d_objT.p : nullptr;
  int bs = 256;
  int64_t g = (s->N + bs - 1) / bs;
  if (g > 0) {
    k_build_boxes<<<(unsigned)g, bs, 0, s->stream>>>(a);
    note_launch();
  }
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Stand-alone propagation (for position parity checks): same code path.
// ---------------------------------------------------------------------------
__global__ void k_prepare_params_only(const scd_element *__restrict__ el, int64_t n,
                                      ObjParams *__restrict__ par) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  scd_element x = el[i];
  double a = x.a_km, e = x.e;
  double a3 = __dmul_rn(__dmul_rn(a, a), a);
  double sO, cO, sw, cw, si, ci;
  sincos(x.raan_rad, &sO, &cO);
  sincos(x.argp_rad, &sw, &cw);
  sincos(x.inc_rad, &si, &ci);
  double Px = cO * cw - sO * sw * ci, Py = sO * cw + cO * sw * ci, Pz = sw * si;
  double Qx = -cO * sw - sO * cw * ci, Qy = -sO * sw + cO * cw * ci, Qz = cw * si;
  double b = a * sqrt(1.0 - e * e);
  ObjParams p;
  p.A[0] = a * Px; p.A[1] = a * Py; p.A[2] = a * Pz;
  p.B[0] = b * Qx; p.B[1] = b * Qy; p.B[2] = b * Qz;
  p.n = sqrt(kMu / a3);
  p.M0 = x.M0_rad;
  p.e = e;
  p.vmax = 0;
  p.r = x.radius_km;
  p.P = 0;
  p.tolE = 1e-7 / a;
  p.dmax2 = e > 0.0 ? (float)(p.tolE * (1.0 - e) / (2.0 * e)) : INFINITY;
  p.ef = (float)e;
  par[i] = p;
}

__global__ void k_propagate(const ObjParams *__restrict__ par, const uint32_t *__restrict__ obj,
                            const double *__restrict__ t, int64_t m, double *__restrict__ out) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  double pos[3];
  int it;
  position_at(par[obj[q]], t[q], pos, it);
  out[3 * q + 0] = pos[0];
  out[3 * q + 1] = pos[1];
  out[3 * q + 2] = pos[2];
}

int launch_propagate(const scd_element *d_el, int64_t n, const uint32_t *obj, const double *t,
                     int64_t m, double *out, cudaStream_t st) {
  ObjParams *par = (ObjParams *)dev_alloc(sizeof(ObjParams) * (size_t)n, st);
  if (!par) return SCD_ERR_OOM;
  int bs = 256;
  k_prepare_params_only<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(d_el, n, par);
  if (m > 0) k_propagate<<<(unsigned)((m + bs - 1) / bs), bs, 0, st>>>(par, obj, t, m, out);
  cudaError_t e = cudaGetLastError();
  cudaStreamSynchronize(st);
  dev_free(par, st);
  return e == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Exclusive scan of int64 counts (reduce, scan of block sums, down-sweep).
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_scan_excl(int64_t v, int64_t &total) {
  __shared__ int64_t warp_sums[kScanThreads / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  int64_t before = w > 0 ? warp_sums[w - 1] : 0;
  total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int64_t *in, int64_t n,
                                                              int64_t *bsum) {
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t idx = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  int64_t tot;
  block_scan_excl(s, tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(int64_t *bsum, int64_t nb) {
  // one block scans all block sums, kScanThreads at a time
  int64_t carry = 0;
  for (int64_t base = 0; base < nb; base += kScanThreads) {
    int64_t idx = base + threadIdx.x;
    int64_t v = idx < nb ? bsum[idx] : 0;
    int64_t tot;
    int64_t ex = block_scan_excl(v, tot);
    if (idx < nb) bsum[idx] = carry + ex;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const int64_t *in, int64_t n,
                                                            const int64_t *bsum, int64_t *out) {
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  // blocked arrangement: thread t owns items [t*I, t*I+I) of the tile
  int64_t v[kScanItems];
  int64_t s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t idx = base + (int64_t)threadIdx.x * kScanItems + k;
    v[k] = idx < n ? in[idx] : 0;
    s += v[k];
  }
  int64_t tot;
  int64_t ex = block_scan_excl(s, tot) + bsum[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k) {
    int64_t idx = base + (int64_t)threadIdx.x * kScanItems + k;
    if (idx < n) out[idx] = ex;
    ex += v[k];
    if (idx == n - 1) out[n] = ex;
  }
}

int scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, DevBuf<int64_t> &tmp,
                       cudaStream_t st) {
  if (n <= 0) {
    cudaMemsetAsync(out, 0, sizeof(int64_t), st);
    return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
  }
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (!tmp.ensure((size_t)nb, st)) return SCD_ERR_OOM;
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, tmp.p);
  k_scan_blocks<<<1, kScanThreads, 0, st>>>(tmp.p, nb);
  k_scan_down<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, tmp.p, out);
  note_launch(3);
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}

}  // namespace scd

// ---------------------------------------------------------------------------
// scd_propagate_noalloc: scd_propagate without any device allocation.
//
// scd_propagate needs one ObjParams per object as scratch and gets it from
// the allocator.  Some callers cannot allocate device memory at call time:
// flight or embedded software that must not allocate after start-up, hosts
// whose allocator is not reachable from this library, and latency-bound
// loops that cannot afford the device-wide synchronisation of cudaMalloc and
// cudaFree.  This variant keeps the scratch in a fixed array in device
// memory instead; every GPU that loads the library holds that array
// (kNoAllocMaxObjects * 112 bytes = 3.5 MiB) until the process exits.
// ---------------------------------------------------------------------------
namespace scd {
constexpr int64_t kNoAllocMaxObjects = SCD_NOALLOC_MAX_OBJECTS;
static_assert(sizeof(ObjParams) == 112,
              "the fixed scratch array is documented as 112 bytes per object");
static __device__ __align__(256) ObjParams g_noalloc_params[kNoAllocMaxObjects];

constexpr int kNoAllocMaxDevices = 64;
// per device: the array's device address, looked up exactly once
static std::once_flag g_noalloc_once[kNoAllocMaxDevices];
static ObjParams *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device.  Host code
// only holds a stand-in for the symbol, so the address is looked up once per
// device (std::call_once: first calls from several host threads do not
// race), with that device current.  A failed lookup leaves the slot empty
// and every later call on that device fails the same way.  The address is
// not looked up again after a device reset.
static int noalloc_scratch(ObjParams **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SCD_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return SCD_ERR_CUDA;
  std::call_once(g_noalloc_once[dev], [dev] {
    ObjParams *p = nullptr;
    if (cudaGetSymbolAddress((void **)&p, g_noalloc_params) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    g_noalloc_ptr[dev] = p;
  });
  if (!g_noalloc_ptr[dev]) return SCD_ERR_CUDA;
  *out = g_noalloc_ptr[dev];
  return SCD_OK;
}
}  // namespace scd

extern "C" SCD_API int scd_propagate_noalloc(const scd_element *d_elems, int64_t n,
                                             const uint32_t *d_obj, const double *d_t_s,
                                             int64_t m, double *d_out, void *cuda_stream) {
  if (!d_elems || n <= 0 || m < 0 || (m > 0 && (!d_obj || !d_t_s || !d_out)))
    return SCD_ERR_INVALID_ARG;
  if (n > scd::kNoAllocMaxObjects) return SCD_ERR_CAPACITY;
  scd::ObjParams *par = nullptr;
  int rc = scd::noalloc_scratch(&par);
  if (rc != SCD_OK) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int bs = 256;
  // every entry the second kernel reads is written by the first, so the
  // array needs no clearing between calls
  scd::k_prepare_params_only<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(d_elems, n, par);
  if (m > 0) scd::k_propagate<<<(unsigned)((m + bs - 1) / bs), bs, 0, st>>>(par, d_obj, d_t_s, m, d_out);
  return cudaGetLastError() == cudaSuccess ? SCD_OK : SCD_ERR_CUDA;
}
