/*
 * lst.h -- C ABI of the GB300 Line Segment Tracking library (liblst.so).
 *
 * The library runs the data-parallel hot path of Line Segment Tracking
 * (arXiv:2407.18231, Sec. 1) on one NVIDIA GB300 (sm_103a): per event it bins the
 * outer-tracker hits by module, pairs the hits of each module's two sensors into Mini
 * Doublets (MD), links MDs on connected modules into Line Segments (LS), joins LSs that
 * share an MD into T3s and T3s that share an MD into T5s, combines T3s/T5s with
 * inner-tracker seeds (pLS) into pT3s/pT5s, removes duplicates and emits track
 * candidates (TC): pT5s, pT3s, T5s and unlinked pLSs.  Every step runs in the library's
 * own CUDA kernels; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *   - Return LST_OK (0) or a negative lst_status; no C++ exception crosses the ABI.
 *   - Pointers marked "host" are read during the call only; the caller keeps ownership.
 *     Pointers marked "device" must be device memory of the context's GPU.
 *   - A context is used by one host thread at a time (the serving loop owns its context
 *     while it runs).  After a per-event error the context stays usable.
 *   - lst_last_error(ctx) describes the last failure on that context.
 *   - Units: cm, GeV, tesla (B = 3.8 T); floats are IEEE binary32.
 */
#ifndef LST_H
#define LST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lst_status;
#define LST_OK 0
#define LST_ERR_INVALID_ARG (-1)      /* null pointer, zero count where one is required, bad kind */
#define LST_ERR_BAD_INPUT (-2)        /* module id out of range, non-finite coordinate, bad seed */
#define LST_ERR_NO_MAP (-3)           /* lst_build_connection_map has not run */
#define LST_ERR_OOM (-4)              /* device or host allocation failed */
#define LST_ERR_BUDGET (-5)           /* serving: event does not fit the memory budget */
#define LST_ERR_CUDA (-6)             /* a CUDA runtime call failed */
#define LST_ERR_TIMEOUT (-7)          /* a bounded wait for the device ran out */
#define LST_ERR_BUFFER_TOO_SMALL (-8) /* caller buffer smaller than the result */
#define LST_ERR_NOT_FOUND (-9)        /* unknown or released result id */

/* One detector module (48 bytes).  Both sensors of a doublet module form one module
 * (Sec. 1, Fig. 1: every outer-tracker layer is two closely spaced sensors).  A hit names
 * its sensor as det = 2 * module_index + sensor (0 lower, 1 upper).
 *   barrel: surf = lower-sensor radius, gap = radial sensor spacing, [emin, emax) = z extent
 *   endcap: surf = lower-sensor signed z, gap = |z| spacing, [emin, emax) = r extent
 *   (e0x, e0y) / (e1x, e1y): unit vectors of the lower / upper phi edge of the module.
 *   tilt: barrel only, the tilt of the module in the r-z plane in radians (|tilt| < 1.5;
 *   0 = flat, the sensors are the cylinders r = surf and surf + gap).  A tilted module's
 *   lower sensor is the surface (r - surf) cos(tilt) + (z - zc) sin(tilt) = 0 through the
 *   centre zc of its z bin [emin, emax), its upper sensor is one gap along that normal,
 *   and its hits carry both a z and a radial tolerance (the PS coarse coordinate runs
 *   along the tilted surface; Fig. 1's tilted inner-barrel modules).  Endcap: tilt = 0.
 * Rows (ieta = barrel z bin or endcap ring) must be uniform in length within a surface;
 * iphi < nphi numbers the sectors of a row. */
typedef struct lst_module_desc {
  uint8_t subdet;  /* 0 barrel, 1 endcap */
  uint8_t layer;   /* barrel layer 1..6, endcap disk 1..5 */
  int8_t side;     /* 0 barrel, -1 / +1 endcap */
  uint8_t stype;   /* 0 PS (z measured), 1 2S (z = strip centre) */
  uint16_t ieta;
  uint16_t iphi;
  uint16_t nphi;
  uint16_t pad;
  float surf, gap, emin, emax;
  float e0x, e0y, e1x, e1y;
  float tilt;      /* barrel tilt in the r-z plane (rad), 0 = flat; endcap 0 */
} lst_module_desc;

/* Inner-tracker seed, the pLS of Sec. 1 (80 bytes): helix parameters at a reference point
 * and its pixel hits, four (a quad) or three (a triplet, hits in the first three slots).
 * Pixel hits get the ids 4 * pls_index + k (k < n_hits) in track candidates. */
typedef struct lst_pls {
  float px, py, pz;  /* momentum at the reference point, GeV; px = py = 0 is rejected */
  float x0, y0, z0;  /* reference point, cm */
  float hx[4], hy[4], hz[4];
  int32_t charge;    /* +1 or -1 */
  uint32_t n_hits;   /* 4 (quad; 0 is read as 4) or 3 (triplet); other values are rejected */
} lst_pls;

/* One event as host arrays (the library copies them during the call). */
typedef struct lst_event {
  uint32_t n_hits;
  const float *x, *y, *z;  /* host, n_hits each */
  const uint32_t *det;     /* host, n_hits: 2 * module + sensor */
  uint32_t n_pls;
  const lst_pls *pls;      /* host, n_pls (may be NULL when n_pls == 0) */
} lst_event;

/* A batch whose inputs already sit in device memory (events concatenated). */
typedef struct lst_batch_dev {
  uint32_t n_events;
  uint32_t n_hits;         /* total over the batch */
  uint32_t n_pls;          /* total over the batch */
  uint32_t max_event_hits; /* largest event (sizing hint; 0 = unknown) */
  const float *x, *y, *z;  /* device, n_hits */
  const uint32_t *det;     /* device, n_hits */
  const uint32_t *hit_off; /* device, n_events + 1 (hit_off[0] = 0) */
  const lst_pls *pls;      /* device, n_pls */
  const uint32_t *pls_off; /* device, n_events + 1 */
} lst_batch_dev;

/* Context options.  Zero-initialised means defaults. */
typedef struct lst_config {
  int32_t device;        /* CUDA device ordinal (default 0) */
  uint32_t keep_objects; /* 1: every result also keeps all intermediate objects (tests) */
  uint32_t use_graph;    /* lst_run_event / lst_run_batch: 0 default (graph on), 1 force on, 2 force off */
  uint32_t block_size;   /* threads per block of the stage kernels (0 = tuned default) */
  uint32_t blocks_per_sm;/* resident blocks per SM of the persistent grids (0 = default) */
  uint32_t profile;      /* 1: run kernels eagerly with a CUDA event after each (per-kernel times) */
  uint32_t ls_list_cap;  /* LS work split: neighbour MDs staged per warp in shared memory, up to
                            2048 (0 = the library's choice: 512, raised after a run with a
                            longer neighbour list to hold it; 1 = no staging, one warp per MD) */
  uint32_t reserved[9];
} lst_config;

/* Track candidate (Sec. 1 list: pT5, pT3, T5, unlinked pLS).  76 bytes. */
typedef struct lst_tc {
  uint8_t type;        /* LST_TC_PT5 / PT3 / T5 / PLS */
  uint8_t n_ot;        /* outer-tracker hits used (10, 6 or 0) */
  uint8_t n_pix;       /* pixel hits used (4, 3 or 0) */
  uint8_t pad;
  uint32_t obj;        /* index of the object in its own list (pT5, pT3, T5 or pLS) */
  uint32_t pls;        /* pLS index, or 0xFFFFFFFF */
  uint32_t ot[10];     /* input hit indices, 0xFFFFFFFF padded (MD lower, upper, ...) */
  uint32_t pix[4];     /* 4 * pls + k for k < n_pix, 0xFFFFFFFF after */
  float pt;            /* GeV: the pLS pT, or for a T5 0.0113922 / |curvature| */
  float score;         /* selection score (lower is better) */
} lst_tc;

#define LST_TC_PT5 0
#define LST_TC_PT3 1
#define LST_TC_T5 2
#define LST_TC_PLS 3

/* Intermediate objects of one event, for parity checks (keep_objects = 1).
 * All indices are event-local: hits = input order, MDs/T3s/T5s/pLSs = their list. */
#define LST_OBJ_MD 0   /* lst_md_rec */
#define LST_OBJ_LS 1   /* lst_ls_rec */
#define LST_OBJ_T3 2   /* lst_t3_rec */
#define LST_OBJ_T5 3   /* lst_t5_rec */
#define LST_OBJ_PT3 4  /* lst_px_rec */
#define LST_OBJ_PT5 5  /* lst_px_rec */
#define LST_OBJ_PLS 6  /* lst_pls_rec */
typedef struct { uint32_t module, lo, up; } lst_md_rec;
typedef struct { uint32_t md[2]; } lst_ls_rec;
typedef struct { uint32_t md[3]; } lst_t3_rec;
typedef struct { uint32_t md[5]; float score, kfull; uint32_t alive; } lst_t5_rec;
typedef struct { uint32_t pls, obj; float score; uint32_t alive; } lst_px_rec;
typedef struct { uint32_t n_cand; uint32_t cand[36]; uint32_t is_tc; } lst_pls_rec;

typedef struct lst_ctx lst_ctx;
typedef uint64_t lst_result_id;

/* Creates a context on cfg->device (cfg may be NULL), copies the module table to the
 * device and derives every per-module constant the selections need.
 * mods: host, n_mods records.  *out_ctx receives the context (free with lst_destroy).
 * Errors: INVALID_ARG (null, n_mods == 0), BAD_INPUT (bad module record), CUDA, OOM. */
lst_status lst_load_geometry(const lst_module_desc *mods, uint32_t n_mods, const lst_config *cfg,
                             lst_ctx **out_ctx);

/* Builds the module connection map on the host and keeps it resident on the device
 * (Sec. 1: MDs are only linked between modules a precomputed map marks as reachable).
 * The map is a conservative superset: it only prunes module pairs whose anchors can never
 * pass the LS selection.  Errors: INVALID_ARG, OOM, CUDA. */
lst_status lst_build_connection_map(lst_ctx *ctx);

/* Runs the whole chain on one event (the per-event path): the same persistent kernels as a
 * batch, replayed from the context's CUDA graph (plain stream-ordered launches when
 * use_graph = 2).  ev: host arrays.  *out receives a result id (free with lst_release_result).
 * Errors: INVALID_ARG, BAD_INPUT (checked on the device), NO_MAP, OOM, CUDA, TIMEOUT. */
lst_status lst_run_event(lst_ctx *ctx, const lst_event *ev, lst_result_id *out);

/* Runs n events as one batch: one packed upload, one persistent launch per stage, replayed
 * from a CUDA graph.  evs: host array of n events; outs: host array of n result ids. */
lst_status lst_run_batch(lst_ctx *ctx, const lst_event *evs, uint32_t n, lst_result_id *outs);

/* Same as lst_run_batch for inputs already in device memory.  stream: a cudaStream_t of
 * the context's device on which the work is enqueued, or NULL for the context's own
 * stream.  Results stay on the device until lst_batch_finish; the call only enqueues work.
 * Errors: INVALID_ARG, NO_MAP, OOM, CUDA. */
lst_status lst_run_batch_device(lst_ctx *ctx, const lst_batch_dev *batch, void *stream);

/* Waits (bounded by timeout_ms, 0 = no bound) for the last lst_run_batch_device, re-runs it
 * with larger buffers if an object list outgrew its storage, and reports the number of
 * track candidates per event.  n_tc_per_event: host array of batch->n_events (may be NULL).
 * outs: host array of n_events result ids, or NULL to keep nothing on the host. */
lst_status lst_batch_finish(lst_ctx *ctx, uint32_t timeout_ms, uint32_t *n_tc_per_event,
                            lst_result_id *outs);

/* Asynchronous batches (no paper counterpart: a pipelining convenience).  The context has
 * two batch slots.  lst_submit_batch packs n host events into a free slot, uploads them on
 * the slot's stream and queues the chain behind the other slot's batch (the device runs one
 * batch at a time; the upload overlaps the other batch's work), then returns at once with
 * a ticket; the caller's arrays may be reused as soon as it returns.  A caller that keeps
 * one batch in flight while it submits the next overlaps its host work with the device.
 * Errors: INVALID_ARG (null, n == 0, both slots in flight), NO_MAP, OOM, CUDA. */
lst_status lst_submit_batch(lst_ctx *ctx, const lst_event *evs, uint32_t n, uint64_t *ticket);

/* Waits (bounded by timeout_ms, 0 = no bound) for a submitted batch, re-runs it with larger
 * buffers if an object list outgrew its storage, frees its slot and stores its results like
 * lst_run_batch.  n_tc_per_event, outs: host arrays of the batch's n events (either may be
 * NULL).  Errors: NOT_FOUND (unknown or collected ticket), TIMEOUT (the batch stays in
 * flight), BAD_INPUT, OOM, CUDA. */
lst_status lst_collect_batch(lst_ctx *ctx, uint64_t ticket, uint32_t timeout_ms, uint32_t *n_tc_per_event,
                             lst_result_id *outs);

/* Copies the track candidates of a result into buf (host, cap records).  With buf == NULL
 * only *n_out is set (size query).  Errors: NOT_FOUND, BUFFER_TOO_SMALL, INVALID_ARG. */
lst_status lst_get_candidates(lst_ctx *ctx, lst_result_id id, lst_tc *buf, uint32_t cap, uint32_t *n_out);

/* The candidates of n results in one call (no paper counterpart: a batch convenience).
 * ids: host array of n result ids.  counts: host array of n, receives each result's number
 * of candidates.  buf (host, cap records) receives them back to back in ids' order; with
 * buf == NULL only counts and *n_total are set (size query).  Errors: INVALID_ARG,
 * NOT_FOUND (an unknown id; nothing is copied), BUFFER_TOO_SMALL (cap < *n_total). */
lst_status lst_get_candidates_batch(lst_ctx *ctx, const lst_result_id *ids, uint32_t n, lst_tc *buf, uint64_t cap,
                                    uint32_t *counts, uint64_t *n_total);

/* Copies one kind of intermediate object (LST_OBJ_*) of a result kept with keep_objects = 1.
 * buf == NULL is a size query.  Errors: NOT_FOUND, INVALID_ARG (kind, or objects not kept),
 * BUFFER_TOO_SMALL. */
lst_status lst_get_objects(lst_ctx *ctx, lst_result_id id, int32_t kind, void *buf, uint32_t cap,
                           uint32_t *n_out);

/* LST as a seeder (Sec. 2, Table 1: the recovery iteration seeded by "LST pLS quads" or
 * by "LST pLS quads+triplets"): the seeds LST left unlinked -- not used by any surviving
 * pT3 or pT5, the pLS track candidates -- handed on instead of being emitted as tracks.
 * mode LST_SEEDS_QUADS keeps the four-hit seeds, LST_SEEDS_QUADS_TRIPLETS also the
 * three-hit ones.  buf (host, cap records) receives them in seed order; buf == NULL is a
 * size query.  Errors: NOT_FOUND, INVALID_ARG (mode), BUFFER_TOO_SMALL. */
#define LST_SEEDS_QUADS 0
#define LST_SEEDS_QUADS_TRIPLETS 1
typedef struct lst_seed {
  uint32_t pls;     /* seed index in the event's pLS list */
  uint32_t n_pix;   /* 4 or 3 */
  uint32_t pix[4];  /* 4 * pls + k for k < n_pix, 0xFFFFFFFF after */
} lst_seed;
lst_status lst_get_seeds(lst_ctx *ctx, lst_result_id id, int32_t mode, lst_seed *buf, uint32_t cap,
                         uint32_t *n_out);

/* Frees a result's host storage.  Errors: NOT_FOUND. */
lst_status lst_release_result(lst_ctx *ctx, lst_result_id id);

/* Frees the context, its device memory and streams.  NULL is a no-op. */
void lst_destroy(lst_ctx *ctx);

/* Text of the last error on ctx (never NULL; valid until the next call on ctx). */
const char *lst_last_error(lst_ctx *ctx);

/* Static text for a status code. */
const char *lst_status_string(lst_status s);

/* Per-call statistics of the last run on the context (object counts of the whole batch,
 * candidate tests are not counted on the device).  Any pointer may be NULL. */
typedef struct lst_stats {
  uint32_t n_events, n_hits, n_pls, n_md, n_ls, n_t3, n_t5, n_pt3, n_pt5, n_tc;
  uint32_t reruns;        /* re-runs after an object list outgrew its storage */
  uint32_t kernels;       /* kernels launched per run */
  uint64_t device_bytes;  /* device memory held by the context */
  uint64_t ls_candidates; /* MD pairs of connected modules the LS selection tested */
  /* the last lst_serve_replay on the context: batches launched, events in its largest
   * batch, and the most device memory the context and its slots held at once */
  uint32_t served_batches, served_max_batch;
  uint64_t served_peak_bytes;
  uint64_t map_edges;     /* module pairs in the connection map */
} lst_stats;
lst_status lst_get_stats(lst_ctx *ctx, lst_stats *out);

/* Changes the launch configuration of a context (cfg->block_size, blocks_per_sm,
 * ls_list_cap; the other fields are ignored).  Results never depend on it; the next run
 * re-captures its graph.  Errors: INVALID_ARG (out of range, or a batch in flight). */
lst_status lst_set_tuning(lst_ctx *ctx, const lst_config *cfg);

/* Learned T5 selection (Sec. 1: the LST selections include machine-learning methods).  A
 * network of two hidden layers of LST_T5_MLP_HIDDEN rectified units scores each T5
 * candidate and replaces the two curvature-agreement conditions (inner/outer and
 * bridge/full); the full-circle radius and the (a, c, e) r-z condition stay.  With d1, d2
 * the two curvature differences, rhs1, rhs2 the cut tolerances they are held against, k_*
 * the signed curvatures of the inner, outer, bridge and full triples and tol_* their
 * errors, the LST_T5_MLP_INPUTS inputs are (x / (x + y), 0 when both are 0, written x:y):
 *   f0 = d1 : rhs1,  f1 = d2 : rhs2,
 *   f2 = d1 : (|k_in| + |k_out| + 1e-4),  f3 = d2 : (|k_br| + |k_full| + 1e-4),
 *   f4 = (tol_in + tol_out) : (|k_in| + |k_out| + 1e-4),  f5 = |k_full| / k_max,
 *   f6, f7 = r-z residual : tolerance of (a, c, e) and of (b, c, d);
 * then h1 = relu(b1 + W1 f), h2 = relu(b2 + W2 h1), z = b3 + w3 . h2 in binary32, every sum
 * from the bias in index order, and the candidate passes when z > 0.  weights (host,
 * LST_T5_MLP_PARAMS floats) in this order: W1 (16 rows of 8, row j = unit j), b1 (16),
 * W2 (16 rows of 16), b2 (16), w3 (16), b3 (1); the call copies them.  weights == NULL
 * returns to the curvature cuts (the default).  T5 scores, curvatures and everything after
 * the T5 step keep their definitions.  Applies to every later run on the context (its
 * graphs are captured again); the package ships weights trained on synthetic events.
 * Errors: INVALID_ARG (n != LST_T5_MLP_PARAMS, a weight not finite, a batch in flight). */
#define LST_T5_MLP_INPUTS 8
#define LST_T5_MLP_HIDDEN 16
#define LST_T5_MLP_PARAMS 433
lst_status lst_set_t5_selection(lst_ctx *ctx, const float *weights, uint32_t n);

/* Per-kernel device time of the last run in profile mode (CUDA events on the launching
 * stream, summed over the kernel's launches in that run).  buf == NULL is a size query. */
typedef struct lst_profile_entry {
  char name[24];
  uint32_t launches;
  float ms;
} lst_profile_entry;
lst_status lst_get_profile(lst_ctx *ctx, lst_profile_entry *buf, uint32_t cap, uint32_t *n_out);

/* Allocation-free variant of lst_run_event for one small event, for callers that may not
 * allocate device memory while they run (a host framework whose pool allocator owns the
 * GPU, a latency-critical loop that cannot take cudaMalloc's implicit synchronisation, a
 * plug-in in a process that forbids device allocations after start-up).  The paper has no
 * counterpart; this is a deployment convenience.
 * All intermediate lists live in one file-scope device array of 8 MiB that every GPU which
 * loads the library holds until the process exits.  Limits per call: 8192 hits, 512 pLS,
 * 16384 modules in the context, 8192 MDs, 32768 LS, 32768 T3, 16384 T5, 16384 pT3,
 * 16384 pT5; anything larger returns LST_ERR_BUDGET with the list named in lst_last_error.
 * ev: one event (n_events = 1) with device input pointers.  tc_out: device buffer of tc_cap
 * records receiving the track candidates (same records and order as lst_run_event);
 * *n_tc (host) receives their number (also when it exceeds tc_cap, with
 * LST_ERR_BUFFER_TOO_SMALL).  stream: cudaStream_t to run on (NULL = default stream); the
 * call waits for it.  The call performs no cudaMalloc/cudaFree and no allocating library
 * call, its first call on a device included: lst_load_geometry, with the context's device
 * current, looks up the array's device address (cudaGetSymbolAddress, which loads the
 * library's code for that device and commits the array) and loads every kernel the chain
 * launches.  Every call shares the one array and resets what must start at zero, so calls
 * whose work overlaps on the GPU (other streams, other threads) race and must not be
 * issued.  Errors: INVALID_ARG, NO_MAP, BUDGET, BAD_INPUT, BUFFER_TOO_SMALL, CUDA. */
lst_status lst_run_event_static(lst_ctx *ctx, const lst_batch_dev *ev, lst_tc *tc_out, uint32_t tc_cap,
                                uint32_t *n_tc, void *stream);

/* ---- serving: continuous batching of a stream of events (Sec. 2 context: trigger
 * farms reconstruct events as they arrive).  Events are admitted while the device-memory
 * budget allows, packed into open batch slots, and run concurrently on several streams;
 * results are bit-identical to lst_run_event on the same event. ---- */
typedef struct lst_serve_config {
  uint32_t n_slots;          /* concurrent batch slots (streams), >= 1; on PU200-like events at
                                60-80 % of the batched rate, 2 slots of max_batch 16 sharing the
                                device gave the lowest p99 latency */
  uint32_t max_batch;        /* events per slot launch, >= 1 */
  uint64_t memory_budget;    /* bytes of device memory the context and all slots may hold,
                                0 = unbounded.  What the context already holds (geometry,
                                map, its own pipeline) stays; the rest is split evenly over
                                the slots, and a slot admits waiting events into its next
                                batch only while the buffers that batch needs (computed
                                before anything is allocated) fit its share.  An event that
                                alone needs more than a slot's share returns LST_ERR_BUDGET. */
  uint32_t share_device;     /* 0: the slots' batches run on the device one after another
                                (each queued behind the previous launch; a batch's working
                                set fills most of the L2) while the others pack and collect;
                                1: the slots' batches run on the device concurrently */
  uint32_t reserved[7];
} lst_serve_config;

/* Replays a stream of events: event i becomes visible at arrival_s[i] seconds after the
 * call starts (host clock).  latency_s[i] receives completion time - arrival time and
 * n_tc[i] the number of track candidates.  outs (may be NULL) receives result ids.
 * lst_get_stats afterwards reports the batches launched, the largest batch and the peak
 * device memory of the replay.
 * Errors: INVALID_ARG, NO_MAP, BUDGET (an event alone exceeds the budget), OOM, CUDA. */
lst_status lst_serve_replay(lst_ctx *ctx, const lst_serve_config *cfg, const lst_event *evs,
                            const double *arrival_s, uint32_t n, double *latency_s, uint32_t *n_tc,
                            lst_result_id *outs, double *wall_s);

#ifdef __cplusplus
}
#endif
#endif /* LST_H */
