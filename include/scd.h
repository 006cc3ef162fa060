/*
 * scd.h -- C ABI of libscd: broad-phase n-to-n screening of orbiting objects
 * over 4D space-time boxes on one GB300 (sm_103a).
 *
 * Method: Bak & Hobbs, "Efficient n-to-n Collision Detection for Space Debris
 * using 4D AABB Trees".  Each object is cut into per-object time segments;
 * each segment becomes a 4D box (its interval occupancy region, Def 7, times
 * its tick interval, Def 8); every pair of boxes of different objects that
 * overlap is a candidate; candidates are reported as a sorted list of
 * (i < j, tick interval) with touching intervals of one pair merged.
 *
 * Conventions shared by every call:
 *  - Every call returns an int status: SCD_OK (0) or a negative SCD_ERR_*.
 *    scd_status_string() names it.  On error no output is partially valid.
 *  - Time is integer ticks of tick_s seconds (Def 6, the discrete-time
 *    problem).  The horizon is T = horizon_s / tick_s ticks (must be a whole
 *    number, T < 2^24); ticks 0..T inclusive are screened, as in Alg 1.
 *  - Boxes are closed on all four axes (Def 2 uses <=).
 *  - A scene owns all device memory it allocates and frees it in
 *    scd_scene_destroy.  Host arrays passed in are copied; the caller keeps
 *    ownership.  A scene is not thread-safe; distinct scenes are independent.
 *  - Work is queued on the CUDA stream given at creation.  Calls that return
 *    host data synchronise that stream.
 *  - Nothing here runs on the CPU apart from argument checks and launch
 *    bookkeeping; if no CUDA device is usable the calls fail with
 *    SCD_ERR_CUDA.
 */
#ifndef SCD_H
#define SCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SCD_API __attribute__((visibility("default")))

enum {
  SCD_OK = 0,
  SCD_ERR_INVALID_ARG = -1,   /* bad size, element, horizon or policy      */
  SCD_ERR_OOM = -2,           /* device allocation failed                  */
  SCD_ERR_BUFFER_TOO_SMALL = -3, /* *n_out holds the count that is needed  */
  SCD_ERR_CUDA = -4,          /* a CUDA runtime call failed                */
  SCD_ERR_KEPLER_NOCONV = -5, /* Kepler's equation did not converge        */
  SCD_ERR_TIMEOUT = -6,       /* a bounded device wait gave up             */
  SCD_ERR_INTERNAL = -7,      /* a device-side consistency check failed    */
  SCD_ERR_STATE = -8,         /* call out of order (e.g. no boxes built)   */
  SCD_ERR_CAPACITY = -9       /* size beyond a fixed built-in capacity     */
};

/* One object (Def 1: position function plus fixed infinity-norm radius).
 * Two-body Kepler elements (Sec. 6.1): semi-major axis a > 0 [km],
 * eccentricity 0 <= e < 1, inclination, right ascension of the ascending
 * node, argument of perigee and mean anomaly at t = 0 [rad], radius >= 0
 * [km].  56 bytes, seven doubles in this order. */
typedef struct {
  double a_km, e, inc_rad, raan_rad, argp_rad, M0_rad, radius_km;
} scd_element;

/* Per-object step length in ticks (Sec. 4: time is tracked per object).
 *  FIXED            k = fixed_ticks for every object
 *  PERIOD_FRACTION  k = floor(P / (period_fraction * tick_s)), P the period
 *  BAND_TABLE       as PERIOD_FRACTION with the fraction looked up by
 *                   perigee altitude a(1-e) - 6378.137 km: n_bands fractions,
 *                   n_bands-1 ascending edges [km]; band b covers
 *                   [edge[b-1], edge[b])
 *  LEARNED          k from a step network (scd_stepnet_*), clamped to
 *                   [P/400, P/50]
 * k is at least one tick.  Arrays are copied at scene creation. */
typedef enum {
  SCD_STEP_FIXED = 0,
  SCD_STEP_PERIOD_FRACTION = 1,
  SCD_STEP_BAND_TABLE = 2,
  SCD_STEP_LEARNED = 3
} scd_step_kind;

typedef struct {
  scd_step_kind kind;
  uint32_t fixed_ticks;
  double period_fraction;
  const double *band_edges_km;
  const double *band_fractions;
  int n_bands;
  const void *stepnet; /* scd_stepnet* for SCD_STEP_LEARNED */
} scd_step_policy;

/* How occ-int (Def 7) bounds a segment [t0, t1]:
 *  SPEED     cube of half-width r + vmax (t1 - t0)/2 around pos((t0+t1)/2),
 *            vmax the perigee speed (vis-viva)
 *  INTERVAL  interval evaluation over the eccentric-anomaly range of the
 *            segment (Sec. 4.5: the single orbital variable is monotone, its
 *            end values bound it), widened by r
 * Both add 1e-6 km and round outward to FP32; both satisfy Properties 1-2. */
typedef enum { SCD_BOX_SPEED = 0, SCD_BOX_INTERVAL = 1 } scd_box_mode;

/* Static decomposition (Sec. 5, Sec. 6.1), solved as independent
 * sub-problems in one launch.
 *  NONE       one problem
 *  ALT_BANDS  p_bands altitude bands with edges at every (n/p)-th sorted
 *             semi-major axis; an object is in every band that its radial
 *             range [a(1-e) - sqrt(3) r, a(1+e) + sqrt(3) r] meets.  Only
 *             pairs joined in the potential-collision graph (Def 9: radial
 *             ranges intersect) are reported.
 *  SLAB_OCT   n_slabs equal tick slabs x the 8 ECI sign octants; the output
 *             equals the NONE output exactly. */
typedef enum {
  SCD_DECOMP_NONE = 0,
  SCD_DECOMP_ALT_BANDS = 1,
  SCD_DECOMP_SLAB_OCT = 2
} scd_decomp_kind;

typedef struct {
  scd_decomp_kind kind;
  int p_bands;
  int n_slabs;
} scd_decomp;

/* One candidate: objects i < j may collide at some tick of [tlo, thi]
 * (closed).  The list is sorted by (i, j, tlo); intervals of one pair never
 * overlap or touch. */
typedef struct {
  uint32_t i, j;
  int32_t tlo, thi;
} scd_pair;

/* Tunables of the tree and traversal (picked by the autotuner). */
typedef struct {
  int leaf_size;      /* boxes per leaf: 1, 2, 4 or 8                      */
  int stack_depth;    /* traversal stack entries: 32, 64 or 128            */
  int block_threads;  /* traversal block size (leaves of several boxes):
                         32..256, a multiple of 32                         */
  int morton_bits;    /* bits per axis of the 4D Morton key: 8, 10, 12, 16
                         (default 12)                                      */
  float time_scale;   /* weight of time against space in the Morton key,
                         (0, 16]: below 1 the horizon takes that share of
                         the time axis's cells; above 1 the scene cube takes
                         1/time_scale of the space axes' cells (default 8).
                         The time axis spans the horizon; in a decomposed
                         screen a tick slab's ticks, in a batch the box's
                         own scene's horizon                               */
  int use_graph;      /* 1: replay find_pairs as one captured CUDA graph    */
  int space_warp;     /* 1: log-compress |x| before quantising (finer keys
                         near Earth, where most boxes are); 0: linear      */
  int nodes_per_step; /* one box per leaf, node width 2: tree nodes each
                         lane visits per traversal step (two independent
                         loads in flight), 1 or 2                          */
  int node_width;     /* one box per leaf: 2 (binary nodes, 36 bytes) or 4
                         (the grandchildren of a binary node in one 128-byte
                         line: one traversal step descends two levels)     */
  float split_km;     /* 0: off.  Otherwise boxes whose largest spatial side
                         exceeds |split_km| km are sorted apart from the
                         others (one key bit above the Morton key, which
                         with 12-bit axes gives up its finest time bit), so
                         each group gets its own subtree and the large boxes
                         do not widen the nodes of the small ones; < 0: the
                         large boxes first (default -1000: each pair of a
                         small and a large box is then found by the small
                         box's query), > 0: after the small ones.  Plain
                         screens apply it with 10- or 12-bit Morton axes
                         (ignored with 8 or 16), decomposed screens and
                         batches always.                                   */
  float refine_start; /* adaptive refinement: the first intervals of object i
                         are L_i ticks long, L_i the largest power of two
                         not above max(1, floor(P_i / (refine_start tick))),
                         P_i its Kepler period; 0: the whole horizon
                         [0, T].  >= 0 and finite (default 256; 128 in a
                         scene of INTERVAL boxes)                          */
} scd_tuning;

typedef struct scd_scene scd_scene;

/* Learned step model (SCD_STEP_LEARNED; not in the paper): a network from 8
 * per-object features to the log of the step in seconds, 8 -> 64 -> 64 -> 1
 * with ReLU, BF16 weights and FP32 accumulation, FP32 master weights trained
 * with AdamW on mean squared error.  Parameters, flat FP32 in this order:
 * W1[8][64], b1[64], W2[64][64], b2[64], w3[64], b3.  Features of an object
 * (scd_stepnet_features): log(a / 6378.137 km), e, sin i, cos i,
 * log(perigee altitude / 100 km), log(apogee altitude / 100 km),
 * log(period / 3600 s), log(1 + number of other objects with |a' - a| <= 50
 * km); altitudes floored at 1 km.  A scene with SCD_STEP_LEARNED uses
 * exp(output) clamped to [P/400, P/50]; every box still bounds its whole
 * segment, so any step keeps the screen sound.  A network must outlive the
 * scenes that use it. */
#define SCD_STEPNET_IN 8
#define SCD_STEPNET_HIDDEN 64
#define SCD_STEPNET_PARAMS 4801
typedef struct scd_stepnet scd_stepnet;

/* Device memory hooks (e.g. a framework's caching allocator).  alloc returns
 * NULL on failure.  Passing NULLs restores cudaMalloc/cudaFree.  Applies to
 * allocations made after the call, process-wide. */
SCD_API int scd_set_allocator(void *(*alloc_fn)(size_t bytes, void *stream, void *ctx),
                              void (*free_fn)(void *ptr, void *stream, void *ctx),
                              void *ctx);

/* Create a scene of n objects (Defs 1, 5-6).  elems: host array of n
 * elements, copied.  horizon_s / tick_s must be a whole number of ticks.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  The scene's
 * tuning starts as scd_default_tuning, with space_warp = 1, time_scale =
 * 16 and refine_start = 128 for INTERVAL boxes (measured best for them).
 * Errors: INVALID_ARG (n <= 0, a <= 0, e outside [0, 1), radius < 0, a NaN,
 * horizon or tick <= 0 or not commensurate, bad policy), OOM, CUDA. */
SCD_API int scd_scene_create(const scd_element *elems, int64_t n, double horizon_s,
                             double tick_s, const scd_step_policy *step,
                             scd_box_mode mode, void *cuda_stream, scd_scene **out);

/* Replace the scene's elements with n new ones from host memory (same n);
 * boxes must be rebuilt. */
SCD_API int scd_scene_set_elements(scd_scene *s, const scd_element *elems, int64_t n);

/* The same, from device memory (n elements in the scd_element layout). */
SCD_API int scd_scene_set_elements_device(scd_scene *s, const scd_element *d_elems, int64_t n);

/* Tuning for later calls; NULL fields are not allowed, use scd_default_tuning. */
SCD_API int scd_scene_set_tuning(scd_scene *s, const scd_tuning *t);
SCD_API int scd_default_tuning(scd_tuning *t);
/* The scene's tuning in force (a find may have deepened the stack after an
 * overflow).  Copied into *t. */
SCD_API int scd_scene_get_tuning(const scd_scene *s, scd_tuning *t);

/* Steps A1-A4: per-object steps, FP64 propagation, outward-rounded FP32
 * boxes and 4D Morton keys (Defs 7-8, Sec. 4.5, Eq. 1).  Asynchronous apart
 * from one read of the box count.  Errors: KEPLER_NOCONV, OOM, CUDA. */
SCD_API int scd_build_boxes(scd_scene *s);

/* Steps A5-A10: sort, hierarchy, refit, traversal and canonical list
 * (Sec. 3.2 query semantics; Sec. 5 decomposition when d != NULL and
 * d->kind != NONE).  host_out: host array of cap pairs.  On success *n_out
 * is the number of pairs written.  If cap is too small: BUFFER_TOO_SMALL,
 * *n_out = the count needed, nothing written.  Synchronous.  When the list
 * fits, an eager find sorts it in buckets of the pairs' first objects and
 * copies each bucket out while the next ones are sorted (the copies overlap
 * the sort when host_out is pinned); the contents equal the device list of
 * scd_find_pairs_device.  On any other error the contents of host_out are
 * unspecified. */
SCD_API int scd_find_pairs(scd_scene *s, const scd_decomp *d, scd_pair *host_out,
                           int64_t cap, int64_t *n_out);

/* The same, leaving the list in device memory owned by the scene; *dev_out
 * stays valid until the next find_pairs call or scd_scene_destroy. */
SCD_API int scd_find_pairs_device(scd_scene *s, const scd_decomp *d,
                                  const scd_pair **dev_out, int64_t *n_out);

/* Every overlapping box pair, unmerged, sorted by (i, j, tlo) (for parity
 * tests of the raw candidate set).  Device memory owned by the scene. */
SCD_API int scd_find_raw_cells_device(scd_scene *s, const scd_pair **dev_out,
                                      int64_t *n_out);

/* One collision witness (Def 4): objects i < j collide at tick t. */
typedef struct {
  uint32_t i, j;
  int32_t t;
} scd_witness;

/* Narrow phase (Def 4, Def 5): the collision witnesses inside a candidate
 * list of the scene.  For each candidate q (i, j, [tlo, thi]) every tick t
 * of the interval is decided by the test of Alg 1: objects i and j collide
 * at t iff their centres, propagated in FP64 (Sec. 6.1), are within
 * r_i + r_j in the infinity norm (Defs 2-3).  Ticks where a bound on the
 * relative motion (perigee speeds, relative velocity and perigee gravity)
 * proves the distance above r_i + r_j are not evaluated; the results are
 * those of testing every tick.
 *   d_pairs   device array of n_pairs candidates with i, j < n and
 *             0 <= tlo <= thi <= T (for example the list of
 *             scd_find_pairs_device); read only.
 *   d_first   device array of n_pairs (or NULL): the first witness tick of
 *             each candidate, -1 if it has none.
 *   d_count   device array of n_pairs (or NULL): the number of witness
 *             ticks of each candidate.
 *   earliest  host pointer (or NULL): the first witness in Alg 1's order
 *             (smallest t, then i, then j) over all candidates, t = -1 if
 *             there is none.  Over the scene's full candidate list this is
 *             the answer of the discrete-time n-to-n problem (Def 5-6).
 * Needs scd_build_boxes (the per-object propagation constants): else
 * SCD_ERR_STATE.  A candidate outside those ranges: SCD_ERR_INVALID_ARG
 * (its outputs are -1 and 0, the others are valid).  n_pairs >= 2^32:
 * SCD_ERR_CAPACITY.  Synchronous on the scene's stream. */
SCD_API int scd_narrow_phase(scd_scene *s, const scd_pair *d_pairs, int64_t n_pairs,
                             int32_t *d_first, uint32_t *d_count, scd_witness *earliest);

/* Adaptive refinement: the interval growing and halving of Alg 5 and Alg 6
 * as data-parallel rounds over all of the scene's objects.  Object i
 * starts with its ticks 0..T cut into intervals of L_i ticks (the last one
 * shorter): L_i is the largest power of two not above
 * max(1, floor(P_i / (f tick))), P_i its Kepler period and f the scene's
 * tuning refine_start, or T + 1 when that is longer or f = 0.  Each round
 * builds the 4D box (Def 8, in the scene's
 * box mode: SPEED or INTERVAL) of every active interval; an interval
 * whose box meets no other object's box is proven collision-free and
 * dropped, one that meets another is halved (ticks [t0, mid], [mid+1, t1]),
 * a single tick that still meets a longer interval waits; two single-tick
 * boxes that meet are a tick candidate, decided by Alg 1's test through
 * scd_narrow_phase.  The result is every collision witness (Def 4) of
 * ticks 0..T, sorted in Alg 1's order (t, then i, then j): the first is the
 * answer of Def 5.  The per-object step policy of the scene plays no part.
 *   host_out     host array of cap witnesses (may be NULL if cap == 0).
 *   n_out        the witness count; cap too small: SCD_ERR_BUFFER_TOO_SMALL
 *                with *n_out set and nothing written.
 *   round_boxes  host array of 64 (or NULL): active intervals per round.
 *   rounds       (or NULL): the rounds taken, at most ceil(log2(max L_i)) + 2.
 * Needs scd_build_boxes (the per-object constants): else SCD_ERR_STATE.
 * Batches of scenes: SCD_ERR_INVALID_ARG.  n > 2^20: SCD_ERR_CAPACITY.
 * Meeting boxes are found per round by a Morton sort of the round's boxes,
 * a radix tree and the persistent traversal; all rounds are queued at once
 * with their sizes on the device.  The scene keeps the rounds' buffers (the
 * capacities that sufficed) and, after the first call of a shape, the
 * rounds' queue as a captured CUDA graph that later calls replay; both are
 * freed with the scene.  Synchronous. */
SCD_API int scd_refine_witnesses(scd_scene *s, scd_witness *host_out, int64_t cap,
                                 int64_t *n_out, int64_t *round_boxes, int *rounds);

/* One span of the continuous-time variant: objects i < j may meet at some
 * real time in [t0, t1] seconds. */
typedef struct {
  uint32_t i, j;
  double t0, t1;
} scd_span;

/* The continuous-time variant of the refinement (Sec. 4.6): the same rounds
 * over closed real intervals, starting from [0, T tick_s] seconds, halved
 * into [t0, mid] and [mid, t1] (the halves share their endpoint), down to
 * the first length <= eps_s; every pair of meeting boxes at that level is
 * one span, the intersection of the two intervals (an instant where two
 * consecutive intervals meet).  No time step: a collision at any real time
 * lies in a span.  Boxes in the scene's box mode.  Spans sorted by (i, j,
 * t0, t1), each once.  Buffers and graph shared with scd_refine_witnesses.
 *   host_out, cap, n_out, round_boxes, rounds: as scd_refine_witnesses.
 * eps_s <= 0: SCD_ERR_INVALID_ARG; eps_s below T tick_s / 2^22:
 * SCD_ERR_CAPACITY.  Needs scd_build_boxes.  Synchronous. */
SCD_API int scd_refine_continuous(scd_scene *s, double eps_s, scd_span *host_out, int64_t cap,
                                  int64_t *n_out, int64_t *round_boxes, int *rounds);

/* The rounds of scd_refine_witnesses (eps_s <= 0) or of
 * scd_refine_continuous at resolution eps_s (eps_s > 0), with every round's
 * boxes copied out, so that each round can be checked against the overlap
 * set of its own boxes: host arrays lo4, hi4 (x, y, z [km], then the
 * interval's first and last unit: ticks, or units of T tick_s / 2^level in
 * the continuous variant) and obj of cap entries receive, round after
 * round, every active interval's FP32 box and object (round_boxes[r] of them
 * for round r, in no particular order).  *n_out: the entries of all rounds;
 * cap too small: SCD_ERR_BUFFER_TOO_SMALL with *n_out set and nothing
 * written.  Errors otherwise as scd_refine_witnesses.  Synchronous. */
SCD_API int scd_refine_trace(scd_scene *s, double eps_s, float *lo4, float *hi4, uint32_t *obj,
                             int64_t cap, int64_t *n_out, int64_t *round_boxes, int *rounds);

/* The scene's boxes in object-major, segment order (device pointers owned
 * by the scene): lo4/hi4 are nbox x 4 floats (x, y, z [km], tick), obj the
 * object of each box. */
SCD_API int scd_get_boxes(const scd_scene *s, const float **lo4, const float **hi4,
                          const uint32_t **obj, int64_t *nbox);

/* Per-object step lengths [ticks] (device, n entries, owned by the scene). */
SCD_API int scd_get_steps(const scd_scene *s, const int32_t **steps);

/* FP64 positions (Sec. 6.1) of objects obj[q] at times t_s[q]: device
 * arrays elems (n), obj (m), t_s (m), out (3 m doubles, x y z [km]).
 * Runs the propagation code of scd_build_boxes.  Asynchronous on stream. */
SCD_API int scd_propagate(const scd_element *d_elems, int64_t n, const uint32_t *d_obj,
                          const double *d_t_s, int64_t m, double *d_out, void *cuda_stream);

/* scd_propagate without any device allocation.  The paper has no
 * counterpart; this exists for callers that cannot allocate device memory
 * when they call: software that must not allocate after start-up (for
 * example on-board or embedded code with a fixed memory budget), hosts whose
 * own allocator this library cannot reach, and latency-bound loops that
 * cannot pay for the device-wide synchronisation of cudaMalloc/cudaFree.
 *
 * Same arguments, layout and result as scd_propagate (obj[q] < n is the
 * caller's duty).  The per-object scratch (112 bytes per object) lives in a
 * fixed array in device memory of SCD_NOALLOC_MAX_OBJECTS entries (3.5 MiB);
 * every GPU that loads the library holds it until the process exits.
 * n > SCD_NOALLOC_MAX_OBJECTS fails with SCD_ERR_CAPACITY before any work.
 * The first call on a device looks up the array's device address with that
 * device current (once per device, safe from several host threads); make
 * that first call before any stream capture.  The address is not looked up
 * again after a reset of the device.  The call
 * is asynchronous on cuda_stream and allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  All calls share the one array
 * and it keeps the last call's contents: calls whose work overlaps on the
 * GPU (different streams or threads) race and must be serialised by the
 * caller.  Every scratch entry a call reads is written earlier in the same
 * call, so nothing needs clearing between calls. */
#define SCD_NOALLOC_MAX_OBJECTS 32768
SCD_API int scd_propagate_noalloc(const scd_element *d_elems, int64_t n, const uint32_t *d_obj,
                                  const double *d_t_s, int64_t m, double *d_out,
                                  void *cuda_stream);

/* A batch of independent scenes screened as one: n_scenes scenes of the
 * concatenated elements (scene k owns elements scene_offsets[k] ..
 * scene_offsets[k+1]-1; scene_offsets[0] = 0, strictly increasing), each
 * with its own horizon horizons_s[k] (a whole number of ticks of tick_s).
 * Every scene becomes one cell: one box build, one reference sort, one tree
 * with a subtree per scene, one persistent traversal over all scenes'
 * boxes, one canonical sort.  scd_build_boxes and scd_find_pairs(_device)
 * then work on the batch (decomposition argument NULL or NONE); the list is
 * sorted by (i, j, tlo) with batch-wide object indices, so each scene's
 * pairs are contiguous; scd_batch_scene_offsets gives where (host array of
 * n_scenes + 1 entries).  Pairs never join objects of different scenes.
 * The batch's tuning starts as scd_default_tuning; each scene's boxes are
 * keyed in a time frame of that scene's own horizon. */
SCD_API int scd_batch_scene_create(const scd_element *elems, const int64_t *scene_offsets,
                                   const double *horizons_s, int n_scenes, double tick_s,
                                   const scd_step_policy *step, scd_box_mode mode,
                                   void *cuda_stream, scd_scene **out);
SCD_API int scd_batch_scene_offsets(const scd_scene *s, int64_t *host_offsets);

/* Screening of separately created scenes (each already with boxes), one
 * after another on their own streams; for one launch over many scenes use
 * scd_batch_scene_create.  outs[s] is a host array of caps[s] pairs;
 * n_outs[s] receives each count.  BUFFER_TOO_SMALL if any cap is too small
 * (all counts still reported). */
SCD_API int scd_batch_find_pairs(scd_scene *const *scenes, int n_scenes, const scd_decomp *d,
                                 scd_pair *const *outs, const int64_t *caps, int64_t *n_outs);

/* Step network: create (He-style initial weights from seed; work is queued
 * on cuda_stream), set/get the FP32 parameters (host arrays of
 * SCD_STEPNET_PARAMS floats; setting resets the optimiser), features of n
 * elements (device arrays; d_feat is n x 8 floats), forward pass (device
 * d_x n x 8, d_y n), gradient of the mean squared error over n samples
 * (device d_t n targets, d_grad SCD_STEPNET_PARAMS floats, *loss_out the
 * loss), one AdamW step (beta 0.9, 0.999, eps 1e-8, decoupled weight decay on
 * the weights), checkpoint save/load (magic "SCDNET01", version, parameter
 * count, optimiser step, FP32 parameters), destroy. */
SCD_API int scd_stepnet_create(void *cuda_stream, uint64_t seed, scd_stepnet **out);
SCD_API int scd_stepnet_set_params(scd_stepnet *net, const float *host_params, int64_t count);
SCD_API int scd_stepnet_get_params(const scd_stepnet *net, float *host_params, int64_t count);
SCD_API int scd_stepnet_features(const scd_element *d_elems, int64_t n, float *d_feat,
                                 void *cuda_stream);
SCD_API int scd_stepnet_forward(const scd_stepnet *net, const float *d_x, int64_t n, float *d_y);
SCD_API int scd_stepnet_grad(scd_stepnet *net, const float *d_x, const float *d_t, int64_t n,
                             float *d_grad, float *loss_out);
SCD_API int scd_stepnet_train_step(scd_stepnet *net, const float *d_x, const float *d_t,
                                   int64_t n, float lr, float weight_decay, float *loss_out);
SCD_API int scd_stepnet_save(const scd_stepnet *net, const char *path);
SCD_API int scd_stepnet_load(scd_stepnet *net, const char *path);
SCD_API void scd_stepnet_destroy(scd_stepnet *net);

/* Candidate count per object: for each of n_pairs device pairs, add one to
 * d_counts[i] and d_counts[j] (device array of n_objects, not cleared here).
 * Used to attribute screening work to objects for step training. */
SCD_API int scd_count_pairs_per_object(const scd_pair *d_pairs, int64_t n_pairs, int64_t n_objects,
                                       uint32_t *d_counts, void *cuda_stream);

/* Metrics of the scene's last find_pairs as one JSON object (box count,
 * node and leaf tests, pair counts, kernel times; launches: the kernels of
 * the last box build and find, or of the last refinement call;
 * narrow_evals and
 * narrow_evals_fp64: the ticks the last scd_narrow_phase evaluated, and
 * those of them it had to decide in FP64).  Writes at most cap bytes
 * including the terminating NUL. */
SCD_API int scd_last_metrics(const scd_scene *s, char *json, size_t cap);

SCD_API void scd_scene_destroy(scd_scene *s);
SCD_API const char *scd_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif
