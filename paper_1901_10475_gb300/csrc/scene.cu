// scene.cu -- the C ABI of libscd (include/scd.h): argument checks, device
// memory, and the order of the kernel launches of one screen.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "scd_internal.cuh"

using namespace scd;

// ---------------------------------------------------------------------------
// allocator hooks
// ---------------------------------------------------------------------------
static void *(*g_alloc)(size_t, void *, void *) = nullptr;
static void (*g_free)(void *, void *, void *) = nullptr;
static void *g_alloc_ctx = nullptr;

#include <atomic>
static std::atomic<unsigned long long> g_launches{0};

namespace scd {
void note_launch(int k) { g_launches.fetch_add((unsigned long long)k); }
unsigned long long launch_count() { return g_launches.load(); }

void *dev_alloc(size_t bytes, cudaStream_t st) {
  if (g_alloc) return g_alloc(bytes, (void *)st, g_alloc_ctx);
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void dev_free(void *p, cudaStream_t st) {
  if (!p) return;
  if (g_free) {
    g_free(p, (void *)st, g_alloc_ctx);
    return;
  }
  cudaFree(p);
}
}  // namespace scd

extern "C" SCD_API int scd_set_allocator(void *(*alloc_fn)(size_t, void *, void *),
                                         void (*free_fn)(void *, void *, void *), void *ctx) {
  if ((alloc_fn == nullptr) != (free_fn == nullptr)) return SCD_ERR_INVALID_ARG;
  g_alloc = alloc_fn;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return SCD_OK;
}

extern "C" SCD_API const char *scd_status_string(int status) {
  switch (status) {
    case SCD_OK: return "ok";
    case SCD_ERR_INVALID_ARG: return "invalid argument";
    case SCD_ERR_OOM: return "device allocation failed";
    case SCD_ERR_BUFFER_TOO_SMALL: return "output buffer too small";
    case SCD_ERR_CUDA: return "CUDA error";
    case SCD_ERR_KEPLER_NOCONV: return "Kepler iteration did not converge";
    case SCD_ERR_TIMEOUT: return "bounded device wait timed out";
    case SCD_ERR_INTERNAL: return "device consistency check failed";
    case SCD_ERR_STATE: return "call out of order";
    case SCD_ERR_CAPACITY: return "size exceeds the fixed built-in capacity";
    default: return "unknown status";
  }
}

extern "C" SCD_API int scd_default_tuning(scd_tuning *t) {
  if (!t) return SCD_ERR_INVALID_ARG;
  t->leaf_size = 1;  // one box per leaf: the persistent lock-step traversal
  t->stack_depth = 64;
  t->block_threads = 128;
  t->morton_bits = 12;
  t->time_scale = 8.0f;  // time weighed 8x against space in the Morton curve
  t->use_graph = 0;
  t->space_warp = 0;
  t->nodes_per_step = 2;
  t->node_width = 2;
  t->split_km = -1000.0f;  // boxes wider than 1000 km in their own subtree, first
  // the refinement's first intervals: at most a 256th of a period (24 h
  // catalog solve with SPEED boxes 157 -> 119 ms against a 64th, measured;
  // a 512th 137 ms)
  t->refine_start = 256.0f;
  return SCD_OK;
}

static bool tuning_ok(const scd_tuning *t) {
  bool leaf = t->leaf_size == 1 || t->leaf_size == 2 || t->leaf_size == 4 || t->leaf_size == 8;
  bool st = t->stack_depth == 32 || t->stack_depth == 64 || t->stack_depth == 128;
  bool bs = t->block_threads >= 32 && t->block_threads <= 256 && t->block_threads % 32 == 0;
  bool mb = t->morton_bits == 8 || t->morton_bits == 10 || t->morton_bits == 12 ||
            t->morton_bits == 16;
  bool ts = t->time_scale > 0.0f && t->time_scale <= 16.0f;
  bool sw = t->space_warp == 0 || t->space_warp == 1;
  bool ns = t->nodes_per_step == 1 || t->nodes_per_step == 2;
  bool nw = t->node_width == 2 || t->node_width == 4;
  bool sp = isfinite(t->split_km);
  bool rs = isfinite(t->refine_start) && t->refine_start >= 0.0f;
  return leaf && st && bs && mb && ts && sw && ns && nw && sp && rs;
}

static bool element_ok(const scd_element &x) {
  return isfinite(x.a_km) && isfinite(x.e) && isfinite(x.inc_rad) && isfinite(x.raan_rad) &&
         isfinite(x.argp_rad) && isfinite(x.M0_rad) && isfinite(x.radius_km) && x.a_km > 0.0 &&
         x.e >= 0.0 && x.e < 1.0 && x.radius_km >= 0.0;
}

static int cuda_rc(cudaError_t e) { return e == cudaSuccess ? SCD_OK : SCD_ERR_CUDA; }

#define TRY(x)                \
  do {                        \
    int rc_ = (x);            \
    if (rc_ != SCD_OK) return rc_; \
  } while (0)

static int read_counters(scd_scene *s) {
  cudaError_t e = cudaMemcpyAsync(s->h_ctr_pinned, s->d_ctr.p, sizeof(DevCounters),
                                  cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return SCD_ERR_CUDA;
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return SCD_ERR_CUDA;
  s->h_ctr = *s->h_ctr_pinned;
  return SCD_OK;
}

extern "C" SCD_API int scd_scene_create(const scd_element *elems, int64_t n, double horizon_s,
                                        double tick_s, const scd_step_policy *step,
                                        scd_box_mode mode, void *cuda_stream, scd_scene **out) {
  if (!out) return SCD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!elems || n <= 0 || n >= (1ll << 24) || !step) return SCD_ERR_INVALID_ARG;
  if (!(horizon_s > 0.0) || !(tick_s > 0.0) || !isfinite(horizon_s) || !isfinite(tick_s))
    return SCD_ERR_INVALID_ARG;
  double Tq = horizon_s / tick_s;
  double Tr = nearbyint(Tq);
  if (fabs(Tq - Tr) > 1e-9 * std::max(1.0, Tr) || Tr < 1.0 || Tr >= (double)(1 << 24))
    return SCD_ERR_INVALID_ARG;
  if (mode != SCD_BOX_SPEED && mode != SCD_BOX_INTERVAL) return SCD_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (!element_ok(elems[i])) return SCD_ERR_INVALID_ARG;
  switch (step->kind) {
    case SCD_STEP_FIXED: break;
    case SCD_STEP_PERIOD_FRACTION:
      if (!(step->period_fraction > 0.0) || !isfinite(step->period_fraction))
        return SCD_ERR_INVALID_ARG;
      break;
    case SCD_STEP_BAND_TABLE:
      if (step->n_bands < 1 || !step->band_fractions || (step->n_bands > 1 && !step->band_edges_km))
        return SCD_ERR_INVALID_ARG;
      for (int b = 0; b < step->n_bands; ++b)
        if (!(step->band_fractions[b] > 0.0)) return SCD_ERR_INVALID_ARG;
      for (int b = 1; b + 1 < step->n_bands; ++b)
        if (!(step->band_edges_km[b] > step->band_edges_km[b - 1])) return SCD_ERR_INVALID_ARG;
      break;
    case SCD_STEP_LEARNED:
      if (!step->stepnet) return SCD_ERR_INVALID_ARG;
      break;
    default: return SCD_ERR_INVALID_ARG;
  }
  scd_scene *s = new scd_scene();
  cudaGetDevice(&s->device);
  s->stream = (cudaStream_t)cuda_stream;
  s->n = n;
  s->horizon_s = horizon_s;
  s->tick_s = tick_s;
  s->T = (int64_t)Tr;
  s->step_kind = step->kind;
  s->fixed_ticks = step->fixed_ticks;
  s->period_fraction = step->period_fraction;
  s->stepnet = step->kind == SCD_STEP_LEARNED ? step->stepnet : nullptr;
  if (step->kind == SCD_STEP_BAND_TABLE) {
    s->band_edges.assign(step->band_edges_km, step->band_edges_km + (step->n_bands - 1));
    s->band_fracs.assign(step->band_fractions, step->band_fractions + step->n_bands);
  }
  s->box_mode = mode;
  scd_default_tuning(&s->tune);
  if (mode == SCD_BOX_INTERVAL) {
    // the tighter INTERVAL boxes (GEO and HEO ones of a few hundred km)
    // order best with log-compressed space and time weighed 16x: 24 h
    // catalog screen 20.8 -> 19.6 ms, measured; batches keep the defaults
    s->tune.space_warp = 1;
    s->tune.time_scale = 16.0f;
    // their refinement stays selective over longer intervals: a 128th of a
    // period (24 h catalog solve 64.6 ms against 77.3 at a 256th, measured)
    s->tune.refine_start = 128.0f;
  }
  cudaStream_t st = s->stream;
  if (cudaMallocHost(&s->h_ctr_pinned, sizeof(DevCounters)) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return SCD_ERR_CUDA;
  }
  bool ok = s->d_el.ensure(n, st) && s->d_par.ensure(n, st) && s->d_k.ensure(n, st) &&
            s->d_segcnt.ensure(n, st) && s->d_segoff.ensure(n + 1, st) &&
            s->d_ctr.ensure(1, st) && s->d_band.ensure(s->band_edges.size() + s->band_fracs.size() + 1, st);
  if (!ok) {
    scd_scene_destroy(s);
    return SCD_ERR_OOM;
  }
  s->sort_sc.err = &s->d_ctr.p->sort_flags;
  cudaError_t e = cudaMemcpyAsync(s->d_el.p, elems, sizeof(scd_element) * (size_t)n,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !s->band_fracs.empty()) {
    std::vector<double> bt(s->band_edges);
    bt.insert(bt.end(), s->band_fracs.begin(), s->band_fracs.end());
    e = cudaMemcpyAsync(s->d_band.p, bt.data(), sizeof(double) * bt.size(), cudaMemcpyHostToDevice,
                        st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) {
    scd_scene_destroy(s);
    return SCD_ERR_CUDA;
  }
  for (int k = 0; k < 8; ++k) cudaEventCreate(&s->ev[k]);
  s->events_ready = true;
  *out = s;
  return SCD_OK;
}

extern "C" SCD_API int scd_scene_set_elements(scd_scene *s, const scd_element *elems, int64_t n) {
  if (!s || !elems || n != s->n) return SCD_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (!element_ok(elems[i])) return SCD_ERR_INVALID_ARG;
  s->boxes_built = false;
  return cuda_rc(cudaMemcpyAsync(s->d_el.p, elems, sizeof(scd_element) * (size_t)n,
                                 cudaMemcpyHostToDevice, s->stream));
}

extern "C" SCD_API int scd_scene_set_elements_device(scd_scene *s, const scd_element *d_elems,
                                                     int64_t n) {
  if (!s || !d_elems || n != s->n) return SCD_ERR_INVALID_ARG;
  s->boxes_built = false;
  return cuda_rc(cudaMemcpyAsync(s->d_el.p, d_elems, sizeof(scd_element) * (size_t)n,
                                 cudaMemcpyDeviceToDevice, s->stream));
}

extern "C" SCD_API int scd_scene_set_tuning(scd_scene *s, const scd_tuning *t) {
  if (!s || !t || !tuning_ok(t)) return SCD_ERR_INVALID_ARG;
  bool rekey = t->morton_bits != s->tune.morton_bits || t->time_scale != s->tune.time_scale ||
               t->space_warp != s->tune.space_warp || t->split_km != s->tune.split_km;
  s->tune = *t;
  if (rekey) s->boxes_built = false;
  return SCD_OK;
}

extern "C" SCD_API int scd_scene_get_tuning(const scd_scene *s, scd_tuning *t) {
  if (!s || !t) return SCD_ERR_INVALID_ARG;
  *t = s->tune;
  return SCD_OK;
}

extern "C" SCD_API int scd_build_boxes(scd_scene *s) {
  if (!s) return SCD_ERR_INVALID_ARG;
  cudaStream_t st = s->stream;
  if (s->events_ready) cudaEventRecord(s->ev[0], st);
  s->launch_mark = launch_count();
  if (cudaMemsetAsync(s->d_ctr.p, 0, sizeof(DevCounters), st) != cudaSuccess) return SCD_ERR_CUDA;
  if (s->step_kind == SCD_STEP_LEARNED) TRY(learned_steps(s));
  TRY(launch_prepare_objects(s));
  TRY(scan_exclusive_i64(s->d_segcnt.p, s->d_segoff.p, s->n, s->d_scan_tmp, st));
  // the box count sizes every buffer that follows: one 8-byte read
  if (cudaMemcpyAsync(&s->h_ctr_pinned->n_boxes, s->d_segoff.p + s->n, sizeof(int64_t),
                      cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SCD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SCD_ERR_CUDA;
  int64_t N = (int64_t)s->h_ctr_pinned->n_boxes;
  if (N <= 0 || N >= (1ll << 31)) return SCD_ERR_INVALID_ARG;
  s->N = N;
  bool ok = s->d_lo.ensure(N, st) && s->d_hi.ensure(N, st) && s->d_obj.ensure(N, st) &&
            s->d_id.ensure(N, st) && s->d_key32.ensure(N, st) &&
            (s->tune.morton_bits <= 8 || s->d_key64.ensure(N, st));
  if (!ok) return SCD_ERR_OOM;
  TRY(launch_build_boxes(s));
  if (s->events_ready) cudaEventRecord(s->ev[1], st);
  s->boxes_built = true;
  return SCD_OK;
}

static int bits_for(int64_t v) {
  int b = 1;
  while ((1ll << b) <= v) ++b;
  return b;
}

static int find_eager(scd_scene *s, const scd_decomp *d, int dkind, int raw_mode, int ob, int tb);
static int find_graph(scd_scene *s, const scd_decomp *d, int dkind, int ob, int tb);

static void finish_metrics(scd_scene *s, int raw_mode) {
  s->last_node_tests = s->h_ctr.node_tests;
  s->last_leaf_tests = s->h_ctr.leaf_tests;
  s->last_runs = raw_mode ? s->h_ctr.v_raw : s->h_ctr.v_starts;
  s->last_open = raw_mode ? 0 : s->h_ctr.v_ends;
  s->last_launches = launch_count() - s->launch_mark;
  if (s->events_ready) {
    // phases of a replayed graph are not timed: -1
    auto span = [](cudaEvent_t a, cudaEvent_t b) {
      float ms = 0;
      return cudaEventElapsedTime(&ms, a, b) == cudaSuccess ? (double)ms : -1.0;
    };
    s->ms_boxes = span(s->ev[0], s->ev[1]);
    s->ms_sort = span(s->ev[2], s->ev[3]);
    s->ms_build = span(s->ev[3], s->ev[4]);
    s->ms_traverse = span(s->ev[4], s->ev[5]);
    s->ms_canon = span(s->ev[5], s->ev[6]);
    cudaGetLastError();
  }
}

static int find_pairs_impl(scd_scene *s, const scd_decomp *d, int raw_mode) {
  if (!s) return SCD_ERR_INVALID_ARG;
  if (!s->boxes_built) return SCD_ERR_STATE;
  int dkind = d ? d->kind : SCD_DECOMP_NONE;
  scd_decomp scenes_dc;
  if (s->n_scenes > 0) {
    // a batch of scenes: every scene is one cell of one persistent traversal
    if (dkind != SCD_DECOMP_NONE || raw_mode) return SCD_ERR_INVALID_ARG;
    scenes_dc.kind = (scd_decomp_kind)kDecompScenes;
    scenes_dc.p_bands = 0;
    scenes_dc.n_slabs = 0;
    d = &scenes_dc;
    dkind = kDecompScenes;
  } else if (dkind != SCD_DECOMP_NONE) {
    if (dkind == SCD_DECOMP_SLAB_OCT) {
      if (d->n_slabs < 1 || d->n_slabs > 4096) return SCD_ERR_INVALID_ARG;
    } else if (dkind == SCD_DECOMP_ALT_BANDS) {
      if (d->p_bands < 1 || d->p_bands > 4096 || d->p_bands > s->n) return SCD_ERR_INVALID_ARG;
    } else {
      return SCD_ERR_INVALID_ARG;
    }
    if (raw_mode) return SCD_ERR_INVALID_ARG;
  }
  cudaStream_t st = s->stream;
  int ob = bits_for(s->n - 1), tb = bits_for(s->T);
  if (2 * ob + tb > 64) return SCD_ERR_INVALID_ARG;
  int64_t N = s->N;
  s->dkind = dkind;
  s->n_slabs = dkind == SCD_DECOMP_SLAB_OCT ? d->n_slabs : 0;
  s->p_bands = dkind == SCD_DECOMP_ALT_BANDS ? d->p_bands : 0;
  // the decomposed traversal runs on one-box leaves
  const int leaf_saved = s->tune.leaf_size;
  if (dkind != SCD_DECOMP_NONE) s->tune.leaf_size = 1;
  struct Restore {
    scd_scene *s;
    int leaf;
    ~Restore() { s->tune.leaf_size = leaf; }
  } restore{s, leaf_saved};
  if (s->tune.use_graph && !raw_mode) return find_graph(s, d, dkind, ob, tb);
  return find_eager(s, d, dkind, raw_mode, ob, tb);
}

// The find sequence run op by op, with host reads of the counters between
// phases (buffer growth, stack depth, checks).
// Records per box seen so far, per kind of screen (SPEED runs, INTERVAL
// runs, raw cells), starting from catalog-shaped measurements (9.4, 1.5, 22)
// and raised by every large screen (2^20 boxes or more, where a second
// traversal is costly) that needed more; small screens neither learn nor
// use it, and it stays at most 16, so that small crowded scenes cannot make
// a later large one reserve huge buffers.
static std::mutex g_slots_mu;
static double g_slots_per_box[3] = {12.0, 2.0, 24.0};
constexpr int64_t kSlotsLearnBoxes = 1 << 20;

static double slots_per_box(int kind, int64_t N) {
  static const double base[3] = {12.0, 2.0, 24.0};
  if (N < kSlotsLearnBoxes) return base[kind];
  std::lock_guard<std::mutex> lk(g_slots_mu);
  return g_slots_per_box[kind];
}

static void note_slots_per_box(int kind, int64_t N, double ratio) {
  if (N < kSlotsLearnBoxes) return;
  std::lock_guard<std::mutex> lk(g_slots_mu);
  const double r = std::min(16.0, ratio * 1.125);
  if (r > g_slots_per_box[kind]) g_slots_per_box[kind] = r;
}

static int find_eager(scd_scene *s, const scd_decomp *d, int dkind, int raw_mode, int ob, int tb) {
  cudaStream_t st = s->stream;
  int64_t N = s->N;
  if (s->events_ready) cudaEventRecord(s->ev[2], st);
  int64_t M = 0;
  if (dkind == SCD_DECOMP_NONE) {
    // A5: sort box ids along the Morton curve
    int kb = sort_key_bits(s->tune);
    if (s->tune.morton_bits > 8) {
      TRY(radix_sort_u64(s->d_key64.p, s->d_id.p, N, kb, s->sort_sc, st));
    } else {
      TRY(radix_sort_u32(s->d_key32.p, s->d_id.p, N, kb, s->sort_sc, st));
    }
    if (s->events_ready) cudaEventRecord(s->ev[3], st);
    // A6-A7: hierarchy and refit
    TRY(build_hierarchy(s, M));
  } else {
    // A10: references per cell, their sort, the hierarchy and cell roots
    if (s->events_ready) cudaEventRecord(s->ev[3], st);
    TRY(build_decomposed(s, d, M));
    N = s->n_refs;
  }
  if (s->events_ready) cudaEventRecord(s->ev[4], st);
  // A8: traversal, retried with more room when the buffers overflow
  // first guess of the record slots of a new scene: the largest records per
  // box seen so far in this process for the kind of screen (a scene that
  // needs more traverses again with the exact count, and raises the guess)
  const int rkind = raw_mode ? 2 : (s->box_mode == SCD_BOX_INTERVAL ? 1 : 0);
  if (s->pair_cap == 0)
    s->pair_cap = std::max<int64_t>(1 << 16, (int64_t)(N * slots_per_box(rkind, N)));
  bool done = false;
  for (int attempt = 0; attempt < 6 && !done; ++attempt) {
    if (!s->d_starts.ensure(s->pair_cap, st) || (!raw_mode && !s->d_ends.ensure(s->pair_cap, st)) ||
        ((raw_mode || !runs_packed(ob, tb, s->T)) && !s->d_rawval.ensure(s->pair_cap, st)))
      return SCD_ERR_OOM;
    // zero the emission counters, keep the box-build flags
    if (cudaMemsetAsync(s->d_ctr.p, 0, offsetof(DevCounters, extent_bits), st) != cudaSuccess)
      return SCD_ERR_CUDA;
    TRY(traverse(s, M, raw_mode, ob, tb));
    TRY(read_counters(s));
    if (s->h_ctr.trav_flags & ERR_STACK) {
      // a deeper stack, then the same traversal again
      if (s->tune.stack_depth >= 128) return SCD_ERR_INTERNAL;
      s->tune.stack_depth *= 2;
      continue;
    }
    unsigned long long need = raw_mode ? s->h_ctr.n_raw
                                       : std::max(s->h_ctr.n_starts, s->h_ctr.n_ends);
    // the record sort indexes with 32-bit counts
    if (need >= (1ull << 32) - 1) return SCD_ERR_CAPACITY;
    if (need <= (unsigned long long)s->pair_cap) done = true;
    else s->pair_cap = (int64_t)(need + need / 8 + 1024);
    if (N > 0) note_slots_per_box(rkind, N, (double)need / (double)N);
  }
  if (!done) return SCD_ERR_INTERNAL;
  if (s->h_ctr.build_flags & ERR_INVALID) return SCD_ERR_INVALID_ARG;
  if (s->h_ctr.build_flags & ERR_KEPLER) return SCD_ERR_KEPLER_NOCONV;
  if (s->events_ready) cudaEventRecord(s->ev[5], st);
  // A9: canonical list (into host memory: streamed out bucket by bucket)
  s->host_done = false;
  int crc = SCD_ERR_STATE;
  if (s->host_dst && !raw_mode && (int64_t)s->h_ctr.v_starts <= s->host_cap)
    crc = canonicalize_streamed(s, ob, tb, s->host_dst);
  if (crc == SCD_OK) s->host_done = true;
  else if (crc != SCD_ERR_STATE) return crc;
  else TRY(canonicalize(s, raw_mode, ob, tb));
  if (s->events_ready) cudaEventRecord(s->ev[6], st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return SCD_ERR_CUDA;
  if (s->host_done && cudaStreamSynchronize(s->cstream) != cudaSuccess) return SCD_ERR_CUDA;
  unsigned int flags[2] = {0, 0};
  cudaMemcpy(&flags[0], &s->d_ctr.p->trav_flags, sizeof(unsigned int), cudaMemcpyDeviceToHost);
  cudaMemcpy(&flags[1], &s->d_ctr.p->sort_flags, sizeof(unsigned int), cudaMemcpyDeviceToHost);
  if (flags[1] & ERR_SORT) return SCD_ERR_TIMEOUT;
  if (flags[0] & ERR_ZIP) return SCD_ERR_INTERNAL;
  s->graph_M = M;
  finish_metrics(s, raw_mode);
  return SCD_OK;
}

// Everything find_eager does, enqueued without any host wait (sizes from the
// last eager run, counts of the record sorts read on the device), for
// capture into one CUDA graph.
static int enqueue_find(scd_scene *s, const scd_decomp *d, int dkind, int ob, int tb) {
  cudaStream_t st = s->stream;
  int64_t M = 0;
  if (s->events_ready) cudaEventRecord(s->ev[2], st);
  if (dkind == SCD_DECOMP_NONE) {
    int kb = sort_key_bits(s->tune);
    if (s->tune.morton_bits > 8) {
      TRY(radix_sort_u64(s->d_key64.p, s->d_id.p, s->N, kb, s->sort_sc, st));
    } else {
      TRY(radix_sort_u32(s->d_key32.p, s->d_id.p, s->N, kb, s->sort_sc, st));
    }
    if (s->events_ready) cudaEventRecord(s->ev[3], st);
    TRY(build_hierarchy(s, M));
  } else {
    if (s->events_ready) cudaEventRecord(s->ev[3], st);
    TRY(build_decomposed(s, d, M, true));
  }
  if (M != s->graph_M) return SCD_ERR_STATE;
  if (s->events_ready) cudaEventRecord(s->ev[4], st);
  if (cudaMemsetAsync(s->d_ctr.p, 0, offsetof(DevCounters, extent_bits), st) != cudaSuccess)
    return SCD_ERR_CUDA;
  TRY(traverse(s, M, 0, ob, tb));
  if (s->events_ready) cudaEventRecord(s->ev[5], st);
  TRY(canonicalize_dev(s, ob, tb));
  if (s->events_ready) cudaEventRecord(s->ev[6], st);
  return SCD_OK;
}

static void graph_key_of(const scd_scene *s, int64_t key[8]) {
  key[0] = s->dkind;
  key[1] = s->n_slabs * 100000 + s->p_bands;
  key[2] = s->N;
  key[3] = s->pair_cap;
  key[4] = (s->tune.node_width * 10 + s->tune.nodes_per_step) * 100000 +
           s->tune.leaf_size * 1000 + s->tune.stack_depth;
  key[5] = s->tune.morton_bits * 10 + s->tune.space_warp;
  key[6] = (int64_t)(s->tune.time_scale * 1e6f) * 1000000 + (int64_t)(split_of(s->tune) * 10.0f);
  key[7] = s->dkind ? s->n_refs : 0;
}

// Replay the captured find sequence; one read of the counters decides
// whether its sizes still held (else: an eager run, then a new capture).
static int find_graph(scd_scene *s, const scd_decomp *d, int dkind, int ob, int tb) {
  cudaStream_t st = s->stream;
  if (!s->gstream) {
    if (cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->g_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->g_out, cudaEventDisableTiming) != cudaSuccess)
      return SCD_ERR_CUDA;
  }
  int64_t key[8];
  graph_key_of(s, key);
  if (s->graph_ok && memcmp(key, s->graph_key, sizeof(key)) == 0) {
    // the graph runs after everything queued on the caller's stream, and the
    // caller's stream waits for it
    if (cudaEventRecord(s->g_in, st) != cudaSuccess ||
        cudaStreamWaitEvent(s->gstream, s->g_in, 0) != cudaSuccess ||
        cudaGraphLaunch(s->graph_exec, s->gstream) != cudaSuccess ||
        cudaEventRecord(s->g_out, s->gstream) != cudaSuccess ||
        cudaStreamWaitEvent(st, s->g_out, 0) != cudaSuccess)
      return SCD_ERR_CUDA;
    TRY(read_counters(s));
    const DevCounters &c = s->h_ctr;
    if (c.build_flags & ERR_INVALID) return SCD_ERR_INVALID_ARG;
    if (c.build_flags & ERR_KEPLER) return SCD_ERR_KEPLER_NOCONV;
    if (c.sort_flags & ERR_SORT) return SCD_ERR_TIMEOUT;
    bool fits = !(c.trav_flags & (ERR_STACK | ERR_ZIP)) &&
                std::max(c.n_starts, c.n_ends) <= (unsigned long long)s->pair_cap &&
                (!dkind || (int64_t)c.refs_total == s->n_refs);
    if (fits) {
      s->n_out = (int64_t)c.v_starts;
      s->last_graph = 2;
      finish_metrics(s, 0);
      return SCD_OK;
    }
    s->graph_ok = false;
  }
  // eager run (sizes every buffer; its result is the answer), then capture
  TRY(find_eager(s, d, dkind, 0, ob, tb));
  s->last_graph = 0;
  if (s->graph_exec) {
    cudaGraphExecDestroy(s->graph_exec);
    s->graph_exec = nullptr;
  }
  // every buffer the captured sequence touches is sized now: nothing may be
  // allocated while capturing
  if (!s->d_out.grow_keep(s->pair_cap, s->n_out, st) ||
      sort_reserve(s->sort_sc, s->pair_cap, sizeof(unsigned long long),
                   !runs_packed(ob, tb, s->T), st) != SCD_OK ||

      !s->d_tilecnt.ensure((size_t)(s->pair_cap / 2048 + 2), st) ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SCD_OK;  // no graph this time; the eager result stands
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(s->gstream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return SCD_OK;
  }
  s->stream = s->gstream;  // every launch below goes to the captured stream
  int rc = enqueue_find(s, d, dkind, ob, tb);
  cudaError_t e = cudaStreamEndCapture(s->gstream, &g);
  s->stream = st;
  if (rc == SCD_OK && e == cudaSuccess && g &&
      cudaGraphInstantiate(&s->graph_exec, g, 0) == cudaSuccess) {
    graph_key_of(s, s->graph_key);
    s->graph_ok = true;
    s->last_graph = 1;
  } else {
    s->graph_exec = nullptr;
    cudaGetLastError();
  }
  if (g) cudaGraphDestroy(g);
  return SCD_OK;
}

extern "C" SCD_API int scd_find_pairs_device(scd_scene *s, const scd_decomp *d,
                                             const scd_pair **dev_out, int64_t *n_out) {
  if (!dev_out || !n_out) return SCD_ERR_INVALID_ARG;
  TRY(find_pairs_impl(s, d, 0));
  *dev_out = s->d_out.p;
  *n_out = s->n_out;
  return SCD_OK;
}

extern "C" SCD_API int scd_find_raw_cells_device(scd_scene *s, const scd_pair **dev_out,
                                                 int64_t *n_out) {
  if (!dev_out || !n_out) return SCD_ERR_INVALID_ARG;
  TRY(find_pairs_impl(s, nullptr, 1));
  *dev_out = s->d_out.p;
  *n_out = s->n_out;
  return SCD_OK;
}

extern "C" SCD_API int scd_find_pairs(scd_scene *s, const scd_decomp *d, scd_pair *host_out,
                                      int64_t cap, int64_t *n_out) {
  if (!n_out || (cap > 0 && !host_out) || cap < 0) return SCD_ERR_INVALID_ARG;
  s->host_dst = host_out;
  s->host_cap = cap;
  s->host_done = false;
  int rc = find_pairs_impl(s, d, 0);
  // no copy into host_out may still run once the call returns, whatever
  // the path (an error after some buckets were queued included)
  if (s->cstream) cudaStreamSynchronize(s->cstream);
  const bool streamed = s->host_done;
  s->host_dst = nullptr;
  s->host_cap = 0;
  s->host_done = false;
  TRY(rc);
  *n_out = s->n_out;
  if (s->n_out > cap) return SCD_ERR_BUFFER_TOO_SMALL;
  if (s->n_out > 0 && !streamed) {
    if (cudaMemcpyAsync(host_out, s->d_out.p, sizeof(scd_pair) * (size_t)s->n_out,
                        cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
      return SCD_ERR_CUDA;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return SCD_ERR_CUDA;
  }
  return SCD_OK;
}

extern "C" SCD_API int scd_get_boxes(const scd_scene *s, const float **lo4, const float **hi4,
                                     const uint32_t **obj, int64_t *nbox) {
  if (!s || !lo4 || !hi4 || !obj || !nbox) return SCD_ERR_INVALID_ARG;
  if (!s->boxes_built) return SCD_ERR_STATE;
  *lo4 = (const float *)s->d_lo.p;
  *hi4 = (const float *)s->d_hi.p;
  *obj = s->d_obj.p;
  *nbox = s->N;
  return SCD_OK;
}

extern "C" SCD_API int scd_get_steps(const scd_scene *s, const int32_t **steps) {
  if (!s || !steps) return SCD_ERR_INVALID_ARG;
  if (!s->boxes_built) return SCD_ERR_STATE;
  *steps = s->d_k.p;
  return SCD_OK;
}

extern "C" SCD_API int scd_propagate(const scd_element *d_elems, int64_t n, const uint32_t *d_obj,
                                     const double *d_t_s, int64_t m, double *d_out,
                                     void *cuda_stream) {
  if (!d_elems || n <= 0 || m < 0 || (m > 0 && (!d_obj || !d_t_s || !d_out)))
    return SCD_ERR_INVALID_ARG;
  return launch_propagate(d_elems, n, d_obj, d_t_s, m, d_out, (cudaStream_t)cuda_stream);
}

extern "C" SCD_API int scd_batch_find_pairs(scd_scene *const *scenes, int n_scenes,
                                            const scd_decomp *d, scd_pair *const *outs,
                                            const int64_t *caps, int64_t *n_outs) {
  if (!scenes || n_scenes <= 0 || !outs || !caps || !n_outs) return SCD_ERR_INVALID_ARG;
  int worst = SCD_OK;
  for (int k = 0; k < n_scenes; ++k) {
    int rc = scd_find_pairs(scenes[k], d, outs[k], caps[k], &n_outs[k]);
    if (rc == SCD_ERR_BUFFER_TOO_SMALL) worst = rc;
    else if (rc != SCD_OK) return rc;
  }
  return worst;
}

extern "C" SCD_API int scd_batch_scene_create(const scd_element *elems,
                                              const int64_t *scene_offsets,
                                              const double *horizons_s, int n_scenes,
                                              double tick_s, const scd_step_policy *step,
                                              scd_box_mode mode, void *cuda_stream,
                                              scd_scene **out) {
  if (!out || !scene_offsets || !horizons_s || n_scenes < 1 || !(tick_s > 0.0))
    return SCD_ERR_INVALID_ARG;
  *out = nullptr;
  if (scene_offsets[0] != 0) return SCD_ERR_INVALID_ARG;
  int64_t n = scene_offsets[n_scenes];
  std::vector<int32_t> objT((size_t)std::max<int64_t>(n, 1)), objs((size_t)std::max<int64_t>(n, 1));
  double hmax = 0.0;
  for (int k = 0; k < n_scenes; ++k) {
    if (scene_offsets[k + 1] <= scene_offsets[k]) return SCD_ERR_INVALID_ARG;
    double Tq = horizons_s[k] / tick_s, Tr = nearbyint(Tq);
    if (!(horizons_s[k] > 0.0) || !isfinite(horizons_s[k]) ||
        fabs(Tq - Tr) > 1e-9 * std::max(1.0, Tr) || Tr < 1.0 || Tr >= (double)(1 << 24))
      return SCD_ERR_INVALID_ARG;
    hmax = std::max(hmax, horizons_s[k]);
    for (int64_t i = scene_offsets[k]; i < scene_offsets[k + 1]; ++i) {
      objT[(size_t)i] = (int32_t)Tr;
      objs[(size_t)i] = k;
    }
  }
  scd_scene *s = nullptr;
  int rc = scd_scene_create(elems, n, hmax, tick_s, step, mode, cuda_stream, &s);
  if (rc) return rc;
  scd_default_tuning(&s->tune);  // whatever the box mode (measured best for batches)
  cudaStream_t st = s->stream;
  s->n_scenes = n_scenes;
  s->scene_off.assign(scene_offsets, scene_offsets + n_scenes + 1);
  if (!s->d_objT.ensure(n, st) || !s->d_objscene.ensure(n, st) ||
      !s->d_sceneoff.ensure(n_scenes + 1, st) || !s->d_pairoff.ensure(n_scenes + 1, st)) {
    scd_scene_destroy(s);
    return SCD_ERR_OOM;
  }
  if (cudaMemcpyAsync(s->d_objT.p, objT.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(s->d_objscene.p, objs.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaMemcpyAsync(s->d_sceneoff.p, scene_offsets, sizeof(int64_t) * (n_scenes + 1),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    scd_scene_destroy(s);
    return SCD_ERR_CUDA;
  }
  *out = s;
  return SCD_OK;
}

// first pair of each scene in the sorted list: pairs of scene k have
// scene_off[k] <= i < scene_off[k+1]
__global__ void k_pair_offsets(const scd_pair *__restrict__ pr, int64_t np,
                               const int64_t *__restrict__ soff, int ns,
                               int64_t *__restrict__ poff) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > ns) return;
  int64_t key = soff[k];
  int64_t lo = 0, hi = np;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if ((int64_t)pr[mid].i < key) lo = mid + 1; else hi = mid;
  }
  poff[k] = lo;
}

extern "C" SCD_API int scd_batch_scene_offsets(const scd_scene *s, int64_t *host_offsets) {
  if (!s || !host_offsets || s->n_scenes < 1) return SCD_ERR_INVALID_ARG;
  cudaStream_t st = s->stream;
  int ns = s->n_scenes;
  k_pair_offsets<<<(ns + 1 + 127) / 128, 128, 0, st>>>(s->d_out.p, s->n_out, s->d_sceneoff.p, ns,
                                                       s->d_pairoff.p);
  note_launch();
  if (cudaMemcpyAsync(host_offsets, s->d_pairoff.p, sizeof(int64_t) * (ns + 1),
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SCD_ERR_CUDA;
  return SCD_OK;
}

extern "C" SCD_API int scd_last_metrics(const scd_scene *s, char *json, size_t cap) {
  if (!s || !json || cap == 0) return SCD_ERR_INVALID_ARG;
  int w = snprintf(json, cap,
                   "{\"n\": %lld, \"T\": %lld, \"boxes\": %lld, \"node_tests\": %llu, "
                   "\"leaf_tests\": %llu, \"records\": %llu, \"open_runs\": %llu, "
                   "\"pairs\": %lld, "
                   "\"ms_boxes\": %.4f, \"ms_sort\": %.4f, \"ms_build\": %.4f, "
                   "\"ms_traverse\": %.4f, \"ms_canon\": %.4f, \"leaf_size\": %d, "
                   "\"stack_depth\": %d, \"block_threads\": %d, \"morton_bits\": %d, "
                   "\"launches\": %llu, \"refs\": %lld, \"cells\": %d, \"graph\": %d, "
                   "\"narrow_evals\": %llu, \"narrow_evals_fp64\": %llu, \"split_km\": %.1f}",
                   (long long)s->n, (long long)s->T, (long long)s->N, s->last_node_tests,
                   s->last_leaf_tests, s->last_runs, s->last_open, (long long)s->n_out, s->ms_boxes, s->ms_sort,
                   s->ms_build, s->ms_traverse, s->ms_canon, s->tune.leaf_size,
                   s->tune.stack_depth, s->tune.block_threads, s->tune.morton_bits,
                   s->last_launches, (long long)(s->dkind ? s->n_refs : s->N),
                   s->dkind ? s->n_cells : 1, s->last_graph, s->last_np_evals,
                   s->last_np_evals64, (double)split_of(s->tune));
  if (w < 0 || (size_t)w >= cap) return SCD_ERR_BUFFER_TOO_SMALL;
  return SCD_OK;
}

extern "C" SCD_API void scd_scene_destroy(scd_scene *s) {
  if (!s) return;
  cudaStream_t st = s->stream;
  cudaStreamSynchronize(st);
  s->d_el.release(st); s->d_par.release(st); s->d_k.release(st);
  s->d_segcnt.release(st); s->d_segoff.release(st); s->d_scan_tmp.release(st);
  s->d_band.release(st); s->d_ctr.release(st);
  s->d_lo.release(st); s->d_hi.release(st); s->d_obj.release(st);
  s->d_key64.release(st); s->d_key32.release(st); s->d_id.release(st);
  s->s_box.release(st); s->s_obj.release(st);
  s->d_posof.release(st); s->s_nb.release(st);
  s->s_leafkey32.release(st); s->s_leafkey64.release(st);
  s->d_nodes.release(st); s->d_nlo.release(st); s->d_nhi.release(st);
  s->d_qbox.release(st); s->d_qlink.release(st); s->d_w4.release(st);
  s->d_leaflo.release(st); s->d_leafhi.release(st);
  s->d_parent_int.release(st); s->d_parent_leaf.release(st); s->d_flags.release(st);
  s->d_first_last.release(st);
  s->d_starts.release(st); s->d_ends.release(st); s->d_rawval.release(st);
  s->d_tilecnt.release(st);
  s->d_out.release(st);
  s->d_narrow.release(st);
  s->d_npobj.release(st);
  s->sort_sc.release(st);
  s->s_cell.release(st); s->d_first.release(st);
  s->d_refcnt.release(st); s->d_refoff.release(st); s->d_refkey.release(st);
  s->d_refid.release(st); s->d_rr.release(st); s->d_edges.release(st);
  s->d_abits.release(st); s->d_cellroot.release(st);
  s->d_feat.release(st); s->d_ny.release(st); s->d_learned.release(st);
  s->d_objT.release(st); s->d_objscene.release(st); s->d_sceneoff.release(st);
  s->d_pairoff.release(st);
  s->d_part.release(st); s->d_parte.release(st);
  rf_release(s);
  if (s->events_ready)
    for (int k = 0; k < 8; ++k) cudaEventDestroy(s->ev[k]);
  if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
  if (s->gstream) cudaStreamDestroy(s->gstream);
  if (s->g_in) cudaEventDestroy(s->g_in);
  if (s->g_out) cudaEventDestroy(s->g_out);
  if (s->cstream) {
    cudaStreamSynchronize(s->cstream);
    cudaStreamDestroy(s->cstream);
  }
  for (int b = 0; b < scd::kStreamBuckets; ++b)
    if (s->cev[b]) cudaEventDestroy(s->cev[b]);
  if (s->h_ctr_pinned) cudaFreeHost(s->h_ctr_pinned);
  delete s;
}
