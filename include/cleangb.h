/*
 * cleangb -- tiled Hogbom CLEAN with feedback on one GB300 GPU.
 *
 * C ABI of libcleangb.so.  Method: Wright, Adamek & Armour, "Distribution of
 * the Hogbom CLEAN Algorithm Using Tiled Images with Feedback" (arXiv
 * 2501.01461).
 *
 *   Section 3, first equation:  a minor iteration finds the peak pixel of the
 *       residual and records a component (position, peak x gain).
 *   Section 3, second equation: the residual loses gain x peak x PSF, the
 *       PSF centred on the peak.
 *   Section 2, Fig. 1: the image is split into tiles that are deconvolved in
 *       parallel.
 *   Section 3, Figs. 2-3: at regular intervals every tile's new components,
 *       placed on a full-size image and convolved with the full PSF
 *       ("cross-coupling"), are subtracted from the other tiles (feedback).
 *
 * Readings fixed by this library where the paper is silent:
 *   - the peak is the largest |residual| (its signed value becomes the
 *     component); among equal |residual| the lowest row-major index wins;
 *   - PSF centre = (psf_ny / 2, psf_nx / 2); residual pixels whose PSF index
 *     falls outside the PSF array are left unchanged;
 *   - tile (i, j) of a Ty x Tx grid covers rows [floor(i ny / Ty),
 *     floor((i + 1) ny / Ty)) and columns likewise; tile index t = i Tx + j;
 *   - niter is the total budget: tile t may run floor(niter / T) iterations,
 *     plus one for t < niter mod T (T = Ty Tx);
 *   - a tile stops while |peak| <= threshold; it is checked again after each
 *     feedback;
 *   - the feedback interval K counts minor iterations per tile; a round is up
 *     to K iterations in every tile, then one feedback; a flux trigger may
 *     end a tile's round earlier (clean_params.feedback_trigger); K = 0 with
 *     no trigger means no feedback (independent tiles, Fig. 1(b)); the last
 *     round executed always ends with its feedback;
 *   - feedback applies, to each pixel, the other tiles' components of the
 *     round in list order (tile index, then iteration), each as a rounded
 *     float32 multiply followed by a rounded float32 subtract;
 *   - all arithmetic is float32 with separately rounded multiplies and
 *     subtracts (no fused multiply-add), so results are bit-reproducible.
 *
 * Conventions
 *   - Images are row-major float32.  Device pointers ("d_") are CUDA global
 *     memory owned by the caller; host pointers ("h_") are ordinary (ideally
 *     pinned) host memory.  No call keeps a caller pointer after it returns,
 *     except the PSF borrowed by clean_plan (see there).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered; they synchronise the stream only
 *     where stated (to read a status word or a count back).
 *   - Every call returns a clean_status.  After CLEAN_ERR_CUDA or
 *     CLEAN_ERR_TIMEOUT a plan is poisoned: every later call on it returns
 *     the same code.  No call aborts the process.
 *   - Diagnostics: with the environment variable CLEANGB_REPORT_TIMEOUT set,
 *     the batch and server entry points print to stderr, for each job whose
 *     bounded wait expired, its shape, its unit layout and the tile and
 *     exchange where the wait gave up.
 */
#ifndef CLEANGB_H
#define CLEANGB_H

#include <stdint.h>

#if defined(__GNUC__)
#define CLEAN_API __attribute__((visibility("default")))
#else
#define CLEAN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CLEAN_OK = 0,
  CLEAN_ERR_INVALID_ARG = 1, /* bad parameter or pointer; PSF peak not at centre */
  CLEAN_ERR_NONFINITE = 2,   /* NaN or Inf in the dirty image or the PSF */
  CLEAN_ERR_OOM = 3,         /* device allocation failed */
  CLEAN_ERR_CUDA = 4,        /* a CUDA call failed (plan poisoned) */
  CLEAN_ERR_TIMEOUT = 5,     /* a bounded device wait expired (plan poisoned) */
  CLEAN_ERR_UNSUPPORTED = 6  /* valid request the library cannot serve */
} clean_status;

/* feedback_mode.  The environment variable CLEANGB_FORCE_FEEDBACK
 * (gather, fft or auto), when set, overrides it for every plan created
 * afterwards; clean_stats reports the path in use.  clean_run marks each
 * chunk of rounds with an NVTX range "clean_rounds" for profilers. */
enum { CLEAN_FB_GATHER = 0, CLEAN_FB_FFT = 1, CLEAN_FB_AUTO = 2 };
/* mode */
enum { CLEAN_TILED = 0, CLEAN_UNTILED_GRID = 1 };
/* group_sync */
enum { CLEAN_SYNC_AUTO = 0, CLEAN_SYNC_CLUSTER = 1, CLEAN_SYNC_GRID = 2 };

/* One CLEAN component: pixel (y, x), flux gain x peak (Jy), and the tile
 * that found it.  16 bytes. */
typedef struct {
  int32_t y, x;
  float flux;
  int32_t tile;
} clean_component;

/* The problem as the paper states it (dirty image size, PSF, gain,
 * iteration count, threshold, tile grid, feedback interval) plus execution
 * choices.  Fill with clean_params_default() first. */
typedef struct {
  int32_t ny, nx;            /* dirty image rows, columns (>= 1, ny*nx < 2^31) */
  int32_t psf_ny, psf_nx;    /* PSF rows, columns (>= 1); centre (psf_ny/2, psf_nx/2) */
  float gain;                /* loop gain, 0 < gain <= 1 */
  float threshold;           /* stop a tile while |peak| <= threshold (>= 0) */
  int64_t niter;             /* total minor iterations over all tiles (>= 0) */
  int32_t tiles_y, tiles_x;  /* tile grid, 1 .. min(64, ny) and 1 .. min(64, nx) */
  int32_t feedback_interval; /* K >= 0 minor iterations per tile between feedbacks */
  int32_t feedback_mode;     /* CLEAN_FB_GATHER (exact) | CLEAN_FB_FFT | CLEAN_FB_AUTO */
  int32_t mode;              /* CLEAN_TILED | CLEAN_UNTILED_GRID (needs a 1 x 1 grid) */
  int32_t group_ctas;        /* CTAs per tile in the minor loop; 0 = choose */
  int32_t group_sync;        /* CLEAN_SYNC_*: cluster barrier or bounded grid barrier */
  float feedback_trigger;    /* 0, or in (0, 1): a tile's round also ends once its
                                |peak| <= feedback_trigger x the largest |peak| among
                                the tiles taking part in the round (Section 3: a flux
                                threshold starts the feedback); with K = 0 the rounds
                                end on flux alone */
  int32_t reserved[4];       /* must be 0 */
} clean_params;

typedef struct clean_plan_s* clean_plan_t;

/* Counters of a plan's current run (host struct, filled by clean_stats). */
typedef struct {
  int64_t n_components;   /* components in the list */
  int64_t rounds;         /* rounds that produced at least one component */
  int64_t rounds_launched;/* rounds launched, including no-op rounds */
  int32_t group_ctas;     /* CTAs per tile chosen for the minor loop */
  int32_t group_sync;     /* CLEAN_SYNC_CLUSTER or CLEAN_SYNC_GRID */
  int32_t resident;       /* 1 if each CTA keeps its residual rows in shared memory */
  int32_t feedback_mode;  /* the feedback path in use */
  int32_t sm_count;       /* SMs of the device */
  int32_t feedback_tma;   /* 1 if feedback stages PSF windows with TMA */
  int32_t minor_pipe;     /* 1 if the minor loop streams rows with bulk copies */
  int32_t minor_tmem;     /* 1 if the pipeline keeps each CTA's leading chunks in
                             tensor memory (CLEAN_DEBUG_MINOR_TMEM) */
  int64_t kernel_launches;   /* kernels this plan has launched in total */
  int64_t minor_launches;    /* minor-loop launches timed (CLEAN_DEBUG_TIMING) */
  int64_t feedback_launches; /* feedback launches timed (CLEAN_DEBUG_TIMING) */
  double minor_ms;           /* summed CUDA-event time of the timed minor launches */
  double feedback_ms;        /* summed CUDA-event time of the timed feedback launches */
  int64_t graph_launches;    /* two-round CUDA graphs launched (CLEAN_DEBUG_GRAPHS) */
  int64_t minor_pairs;       /* 1 if the minor loop serves tiles in pairs
                                (CLEAN_DEBUG_MINOR_PAIR) */
  double host_in_ms;         /* last clean_deconvolve_host, CUDA-event times on its
                                stream: input copies (and the PSF check), */
  double host_run_ms;        /* the run (set-up, rounds, status reads), */
  double host_out_ms;        /* output copies */
} clean_stats_t;

/* Fills *p with defaults: gain 0.1, threshold 0, 1 x 1 tiles, K 0, gather
 * feedback, tiled mode, automatic group choice.  Sizes and niter are 0 and
 * must be set.  Returns CLEAN_ERR_INVALID_ARG for p == NULL. */
CLEAN_API int clean_params_default(clean_params* p);

/* Checks *p without touching the GPU.  CLEAN_OK or CLEAN_ERR_INVALID_ARG. */
CLEAN_API int clean_params_check(const clean_params* p);

/* Creates a plan: validates *p (before any CUDA call), then allocates the
 * plan's device state on the current device: residual and model images
 * (4 ny nx bytes each), the component list (16 niter bytes), per-round and
 * per-tile scratch.  d_psf (psf_ny x psf_nx float32, device) is BORROWED:
 * the caller keeps it alive and unchanged until clean_destroy or the next
 * clean_set_psf.  d_psf == NULL makes the plan allocate its own PSF buffer,
 * to be filled by clean_set_psf or clean_deconvolve_host.  A supplied PSF is
 * checked on the device (finite, |P| <= P[centre] everywhere); this call
 * synchronises `stream` for that check.
 * Returns CLEAN_OK, CLEAN_ERR_INVALID_ARG, CLEAN_ERR_NONFINITE, CLEAN_ERR_OOM
 * or CLEAN_ERR_CUDA; *out is NULL on failure. */
CLEAN_API int clean_plan(clean_plan_t* out, const clean_params* p, const float* d_psf,
               void* stream);

/* Replaces the PSF.  on_host = 0: `psf` is a device pointer and is borrowed
 * as in clean_plan (only for plans created with a device PSF).  on_host = 1:
 * `psf` is host memory copied into the plan's own PSF buffer (only for plans
 * created with d_psf == NULL).  Validates and synchronises like clean_plan. */
CLEAN_API int clean_set_psf(clean_plan_t plan, const float* psf, int32_t on_host,
                  void* stream);

/* Runs CLEAN.  d_dirty != NULL starts a new run from that dirty image
 * (device, ny x nx, read only; copied to the residual): the component list,
 * model and budgets are reset.  d_dirty == NULL continues the current run
 * (applying any pending feedback from clean_step first).  Executes up to
 * max_rounds rounds (-1 = until no tile is active: every tile has spent its
 * budget or has |peak| <= threshold), each round being up to K minor
 * iterations per tile followed by one feedback.  Synchronises `stream`
 * between batches of rounds to read the device status (a few bytes).
 * Returns CLEAN_OK, CLEAN_ERR_NONFINITE (dirty image not finite; nothing is
 * computed), CLEAN_ERR_INVALID_ARG, CLEAN_ERR_CUDA or CLEAN_ERR_TIMEOUT. */
CLEAN_API int clean_run(clean_plan_t plan, const float* d_dirty, int32_t max_rounds,
              void* stream);

/* One round of minor loops WITHOUT its feedback (Section 3: the tiles are
 * deconvolved separately between synchronising feedback steps).  The round's
 * components stay pending until clean_feedback (or the next clean_run /
 * clean_step, which apply them first).  Does not synchronise. */
CLEAN_API int clean_step(clean_plan_t plan, void* stream);

/* Applies the pending feedback (Section 3, Figs. 2-3): each component found
 * since the last feedback is subtracted, convolved with the full PSF, from
 * every tile but its own.  No-op if nothing is pending.  Does not
 * synchronise. */
CLEAN_API int clean_feedback(clean_plan_t plan, void* stream);

/* Restored image = model convolved with an elliptical Gaussian clean beam
 * (FWHM bmaj_px, bmin_px pixels; major axis at bpa_rad from +x toward +y;
 * peak 1; offsets (dy, dx) with dy^2 + dx^2 <= r^2, r = floor(5 sigma_major))
 * plus the residual, into d_out (device, ny x nx float32).  The paper
 * compares "reconstructed" images (Section 4, Fig. 4) without defining them;
 * this is the usual Hogbom restoration.  Does not synchronise. */
CLEAN_API int clean_restore(clean_plan_t plan, float bmaj_px, float bmin_px,
                  float bpa_rad, float* d_out, void* stream);

/* Copies the current residual and model (device, ny x nx float32 each) and
 * the component list (device, list order) out of the plan; any output may
 * be NULL.  comps_cap bounds the components written.  n_comps (host, may be
 * NULL) receives the list length; reading it synchronises `stream`. */
CLEAN_API int clean_get(clean_plan_t plan, float* d_residual_out, float* d_model_out,
              clean_component* d_comps_out, int64_t comps_cap,
              int64_t* n_comps, void* stream);

/* Host copy of the list offset at which each recorded round starts (the
 * list is round-major, tile index, then iteration).  Writes up to cap
 * offsets; *n_rounds receives the number of rounds.  Synchronises. */
CLEAN_API int clean_get_rounds(clean_plan_t plan, int64_t* h_offsets, int64_t cap,
                     int64_t* n_rounds, void* stream);

/* Checkpoint / resume of a run between rounds (the paper has no
 * counterpart).  clean_checkpoint copies the plan's run state
 * -- residual, model, component list, round offsets, per-tile budgets,
 * peaks and counts, the control block, the round parity -- into the host
 * buffer h_buf (capacity bytes) and stores its size in *bytes; with h_buf
 * NULL it only reports the size.  The plan must have started a run and not
 * be in the middle of a round (after clean_run or clean_step).  clean_resume
 * loads such a checkpoint into a plan created with identical clean_params
 * and a PSF set (the PSF is not part of the checkpoint); clean_run(plan,
 * NULL, ...) then continues the run, with results identical bit for bit to
 * an uninterrupted run.  A checkpoint of another problem or a corrupt one
 * gives CLEAN_ERR_INVALID_ARG.  Both synchronise `stream`. */
CLEAN_API int clean_checkpoint(clean_plan_t plan, void* h_buf, int64_t capacity,
                               int64_t* bytes, void* stream);
CLEAN_API int clean_resume(clean_plan_t plan, const void* h_buf, int64_t bytes, void* stream);

/* One whole deconvolution with host buffers: copies h_dirty (and h_psf if
 * not NULL; the plan must own its PSF then) to the device, runs to
 * completion, copies residual, model and components back.  Outputs may be
 * NULL.  Synchronises `stream` before returning.  The CUDA-event times of
 * its three phases (inputs in, run, outputs out) are kept for clean_stats. */
CLEAN_API int clean_deconvolve_host(clean_plan_t plan, const float* h_dirty,
                          const float* h_psf, float* h_residual,
                          float* h_model, clean_component* h_comps,
                          int64_t comps_cap, int64_t* n_comps, void* stream);

/* Plain (untiled) Hogbom CLEAN on the whole GPU without allocating any
 * memory.  The paper has no counterpart; this entry point exists for callers
 * that cannot allocate device memory while they run -- for example an
 * imaging pipeline that reserves all of its device memory in one pool at
 * start-up, because cudaMalloc can block, synchronise the device or fail on a
 * fragmented heap, or code inside a framework that owns every allocation.
 * The caller passes the inputs (d_dirty ny x nx, d_psf psf_ny x psf_nx,
 * device, read only) and the outputs (d_residual and d_model ny x nx, device;
 * d_comps room for niter components, device; *n_comps, host, receives the
 * count); gain and threshold as in clean_params, niter from 0 to 2^31 - 1
 * (a tighter cap than clean_params': the whole run is one round, whose
 * component count is a 32-bit word); d_residual may equal d_dirty.  Results
 * are identical to clean_plan + clean_run with CLEAN_UNTILED_GRID.  The
 * kernels' other memory (grid-barrier counters, per-CTA partial peak keys,
 * control words: 16.5 KiB) is a fixed array compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 * Each call looks up that array's device address in the current device's
 * context (cudaGetSymbolAddress, which allocates nothing).  All calls share
 * the array and it keeps the last call's contents (the parts that must
 * start at zero are cleared by each call): calls that overlap on the GPU --
 * on two streams, or from two threads -- race and must be serialised by the
 * caller.  Uses one CTA per SM (fewer for images with fewer rows than SMs),
 * at most 1024 (CLEAN_ERR_UNSUPPORTED beyond).  Synchronises `stream`
 * between its launches to read the status back.
 * Returns CLEAN_OK, CLEAN_ERR_INVALID_ARG (bad size or pointer, PSF peak not
 * at the centre), CLEAN_ERR_NONFINITE, CLEAN_ERR_UNSUPPORTED, CLEAN_ERR_CUDA
 * or CLEAN_ERR_TIMEOUT; it calls no cudaMalloc or cudaFree. */
CLEAN_API int clean_hogbom_noalloc(const float* d_dirty, const float* d_psf, int32_t ny,
                                   int32_t nx, int32_t psf_ny, int32_t psf_nx, float gain,
                                   int64_t niter, float threshold, float* d_residual,
                                   float* d_model, clean_component* d_comps,
                                   int64_t* n_comps, void* stream);

/* ---- Batches: many images deconvolved together ----------------------
 * A batch holds n independent deconvolutions (each its own dirty image, PSF
 * and clean_params, sizes and tile grids free) and runs all of them round by
 * round in shared launches: one minor-loop launch per residual placement with
 * one CTA per (image, tile), largest tiles first, and one feedback launch over
 * every image's blocks.  The paper treats one image; batching changes only
 * which CTA serves which tile, so each image's results are bit for bit those
 * of its own clean_plan + clean_run.  Images with FFT feedback (feedback_mode
 * FFT, or AUTO when the plan picks it) share the minor-loop launches and run
 * their own transforms and kernels for the feedback.  The untiled mode
 * (CLEAN_UNTILED_GRID) is not accepted: a one-tile grid serves instead. */
typedef struct clean_batch_s* clean_batch_t;

/* Creates a batch of n images: params[i] as for clean_plan (checked before
 * any CUDA call), d_psfs[i] device PSFs, BORROWED as in clean_plan.
 * Allocates each image's state.  Synchronises.  CLEAN_OK,
 * CLEAN_ERR_INVALID_ARG, CLEAN_ERR_NONFINITE, CLEAN_ERR_OOM, CLEAN_ERR_CUDA. */
CLEAN_API int clean_batch_create(clean_batch_t* out, int32_t n, const clean_params* params,
                                 const float* const* d_psfs, void* stream);

/* Runs every image: d_dirties != NULL (host array of n device pointers)
 * starts new runs from those dirty images; NULL continues.  At most
 * max_rounds rounds (-1: until no tile of any image is active).  Images that
 * finish early stop costing work.  Synchronises between batches of rounds. */
CLEAN_API int clean_batch_run(clean_batch_t b, const float* const* d_dirties,
                              int32_t max_rounds, void* stream);

/* Image i's residual, model and component list, as clean_get. */
CLEAN_API int clean_batch_get(clean_batch_t b, int32_t i, float* d_residual, float* d_model,
                              clean_component* d_comps, int64_t comps_cap, int64_t* n_comps,
                              void* stream);

/* Rounds and kernels launched by the last runs, components over all images
 * (as of the last status read).  Any output may be NULL. */
CLEAN_API int clean_batch_stats(clean_batch_t b, int64_t* rounds_launched,
                                int64_t* kernel_launches, int64_t* n_components);

/* Round replay from CUDA graphs (on by default): each run of two rounds is
 * one launch of a graph captured after the work lists last changed; results
 * are identical either way.  enable: 1 on, 0 off, -1 leave as is.
 * *graph_launches (may be NULL) receives the graph launches so far.  This
 * is a launch mechanism of this library; the paper has no counterpart. */
CLEAN_API int clean_batch_graphs(clean_batch_t b, int32_t enable, int64_t* graph_launches);

/* Frees the batch and its images' state (not the borrowed PSFs). */
CLEAN_API void clean_batch_destroy(clean_batch_t b);

/* ---- Serving: continuous batching ------------------------------------
 * A server keeps many deconvolution jobs resident on the device and runs
 * them together round by round (the batch machinery above); jobs are added
 * and removed between steps, so a job that arrives while others run starts
 * at the next step and overlaps with them.  Each job's results equal its own
 * clean_plan + clean_run bit for bit, alone or in any mix.  Admission policy
 * (which queued job to add, under which memory budget) belongs to the
 * caller; clean_server_add fails with CLEAN_ERR_OOM when its slots or the
 * device memory run out. */
typedef struct clean_server_s* clean_server_t;

/* A server with room for max_jobs resident jobs. */
CLEAN_API int clean_server_create(clean_server_t* out, int32_t max_jobs, void* stream);

/* Adds a job: params as for clean_plan (CLEAN_TILED), d_psf
 * BORROWED until clean_server_remove, d_dirty read by this call's set-up
 * (stream-ordered) only.  Allocates the job's state and synchronises (PSF
 * check).  *job_id identifies it from then on. */
CLEAN_API int clean_server_add(clean_server_t sv, const clean_params* params, const float* d_psf,
                               const float* d_dirty, int64_t* job_id, void* stream);

/* Runs `rounds` rounds of every unfinished job, then reads their status;
 * *n_running (may be NULL) receives how many jobs still have work.
 * Synchronises. */
CLEAN_API int clean_server_step(clean_server_t sv, int32_t rounds, int32_t* n_running,
                                void* stream);

/* Ids of finished jobs not yet removed (up to cap; *n_done the count). */
CLEAN_API int clean_server_done(clean_server_t sv, int64_t* ids, int32_t cap, int32_t* n_done);

/* A job's residual, model and component list, as clean_get. */
CLEAN_API int clean_server_get(clean_server_t sv, int64_t job_id, float* d_residual,
                               float* d_model, clean_component* d_comps, int64_t comps_cap,
                               int64_t* n_comps, void* stream);

/* Frees a job's state (finished or not); synchronises the device. */
CLEAN_API int clean_server_remove(clean_server_t sv, int64_t job_id);

/* Frees the server and every job still in it. */
CLEAN_API void clean_server_destroy(clean_server_t sv);

/* ---- Measurement: read bandwidth of the L2 -> SM path -----------------
 * The minor loop and the feedback stream PSF windows that stay resident in
 * L2, so their roofline is the rate at which the SMs pull L2-resident data.
 * This call measures it on the current device (the paper has no
 * counterpart).  d_buf (device, 16-byte aligned, caller-owned, read only) of
 * `bytes` bytes should fit well inside L2.  One untimed launch brings it into
 * L2, then one launch reads it `passes` times over, timed with CUDA events on
 * `stream`: method 0 with bulk copies into shared memory (16 KiB each, six
 * in flight per CTA; bytes a multiple of 16384; ctas_per_sm 1 or 2), method
 * 1 with 16-byte vector loads (bytes a multiple of 16; ctas_per_sm 1..4).
 * *bytes_read receives the bytes the timed launch read and *ms its duration.
 * Synchronises `stream`.  CLEAN_OK, CLEAN_ERR_INVALID_ARG, CLEAN_ERR_CUDA, or
 * CLEAN_ERR_TIMEOUT (a copy did not complete within 1 s). */
CLEAN_API int clean_probe_l2_read(const void* d_buf, int64_t bytes, int32_t passes,
                                  int32_t method, int32_t ctas_per_sm, int64_t* bytes_read,
                                  float* ms, void* stream);

/* Fills *out (host) with the plan's counters.  Synchronises. */
CLEAN_API int clean_stats(clean_plan_t plan, clean_stats_t* out, void* stream);

/* Frees everything the plan owns (not the borrowed PSF).  NULL is a no-op.
 * Synchronises the device's work that uses the plan. */
CLEAN_API void clean_destroy(clean_plan_t plan);

/* Static string for a status code. */
CLEAN_API const char* clean_strerror(int status);

/* Test hooks.  clean_debug_set(plan, what, value):
 *   CLEAN_DEBUG_SPIN_LIMIT_NS  bound (ns) of every grid-barrier wait
 *                              (default 2e9); a wait that exceeds it sets
 *                              CLEAN_ERR_TIMEOUT and the kernel returns
 *   CLEAN_DEBUG_FORCE_TIMEOUT  1: the first grid-barrier wait waits for an
 *                              arrival that never comes (it must expire)
 *   CLEAN_DEBUG_FEEDBACK_PATH  feedback kernel: 0 automatic (TMA when the
 *                              PSF is 16-byte aligned with a row pitch that is
 *                              a multiple of 4 floats), 1 plain loads, 2 TMA
 *                              when possible (same results, bit for bit)
 *   CLEAN_DEBUG_GRAPHS         1 (default): clean_run replays each two rounds
 *                              from a CUDA graph captured once per launch
 *                              configuration (not while timing, not for the
 *                              FFT feedback); 0: launch every kernel directly.
 *                              Same results, bit for bit.
 *   CLEAN_DEBUG_MINOR_PATH     minor-loop kernel: 0 automatic (bulk-copy
 *                              pipeline when image and PSF rows are 16-byte
 *                              aligned), 1 plain loads, 2 pipeline when
 *                              possible (same results, bit for bit)
 *   CLEAN_DEBUG_PIPE_CHUNK_PX  pipeline tuning: about this many pixels per
 *                              staged chunk (0: 4096)
 *   CLEAN_DEBUG_PIPE_STAGES    pipeline tuning: at most this many buffers in
 *                              the ring (0: 8); both fail with
 *                              CLEAN_ERR_INVALID_ARG if the ring no longer fits
 *   CLEAN_DEBUG_MINOR_TMEM     1 (default): the pipeline keeps each CTA's
 *                              leading full 128 x 60 chunks (up to 8) in
 *                              tensor memory for the launch when the
 *                              configuration allows it (clean_stats_t.
 *                              minor_tmem); 0: stream every chunk.  Same
 *                              results, bit for bit.
 *   CLEAN_DEBUG_MINOR_PAIR     1 (default): with grid groups, streamed rows and
 *                              an even number of tiles at least 256 pixels
 *                              wide, groups of 2G CTAs serve pairs of tiles
 *                              and alternate between them, so one tile's
 *                              exchange overlaps the other's pass
 *                              (clean_stats_t.minor_pairs); 0: a group per
 *                              tile.  Same results, bit for bit.
 *   CLEAN_DEBUG_TIMING         1: bracket every minor-loop and feedback launch
 *                              with CUDA events on its stream and sum their
 *                              durations into clean_stats (0: off, resets)
 * clean_debug_alloc_limit(bytes): host-side cap on the bytes a plan may
 * allocate (-1 = none); a plan over it fails with CLEAN_ERR_OOM before
 * allocating. */
enum {
  CLEAN_DEBUG_SPIN_LIMIT_NS = 1,
  CLEAN_DEBUG_FORCE_TIMEOUT = 2,
  CLEAN_DEBUG_TIMING = 3,
  CLEAN_DEBUG_FEEDBACK_PATH = 4,
  CLEAN_DEBUG_MINOR_PATH = 5,
  CLEAN_DEBUG_PIPE_CHUNK_PX = 6,
  CLEAN_DEBUG_PIPE_STAGES = 7,
  CLEAN_DEBUG_GRAPHS = 8,
  CLEAN_DEBUG_MINOR_TMEM = 9,
  CLEAN_DEBUG_MINOR_PAIR = 10
};
CLEAN_API int clean_debug_set(clean_plan_t plan, int32_t what, int64_t value);
CLEAN_API void clean_debug_alloc_limit(int64_t bytes);

#ifdef __cplusplus
}
#endif

#endif /* CLEANGB_H */
