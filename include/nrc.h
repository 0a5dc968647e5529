/*
 * nrc.h - C ABI of the GB300 (sm_103a) neural radiance cache hot path.
 *
 * The library computes the per-frame work of a neural radiance cache
 * (Mueller et al., "Real-time Neural Radiance Caching for Path Tracing",
 * ACM TOG 40(4) 2021): inference of the cached scattered radiance for every
 * path vertex that queries the cache (Sec. 3.1), and online training on the
 * frame's training records (Sec. 3.3, 3.5) with the relative L2 loss (Eq. 5)
 * and Adam (Sec. 5).  The network is the bias-free ReLU MLP of Sec. 5
 * ("Architecture"): 64 encoded inputs (Table 1, Sec. 3.6), 5 hidden layers of
 * width 64, 3 linear RGB outputs.
 *
 * Conventions (all entry points):
 *  - Every call returns an nrc_status.  NRC_OK is 0.  On failure the
 *    thread-local string from nrc_last_error_string() says why.  No call
 *    aborts or prints.
 *  - Work is asynchronous on the caller's stream (an nrc_stream is a
 *    cudaStream_t; NULL means the legacy default stream).  Only
 *    nrc_get_state, nrc_set_state, nrc_check_error, nrc_frame_host and
 *    nrc_destroy synchronise that stream.
 *  - The CALLER owns every buffer passed in; the library reads and writes it
 *    only during the stream-ordered execution of the call.  Device pointers
 *    must be device-accessible memory of the current device; record and
 *    output pointers must be 16-byte aligned.
 *  - The LIBRARY owns the cache state created by nrc_create: FP32 master
 *    weights, Adam moments, the step counter, the low-precision weight image
 *    the tensor-core kernels stage into shared memory, scratch for weight
 *    gradient partials, and a device error word.
 *  - Errors: a NULL cache or NULL pointer with n > 0, n < 0, a misaligned
 *    pointer or an out-of-range enum give NRC_ERR_INVALID_ARG and launch
 *    nothing.  n == 0 is a no-op that returns NRC_OK.  A CUDA error gives
 *    NRC_ERR_CUDA; an allocation failure NRC_ERR_OOM; a device-side bounded
 *    wait that gave up sets the error word, reported as NRC_ERR_TIMEOUT by
 *    nrc_check_error.
 *
 * Record layout (query and training records, 16 x float32 = 64 bytes, AoS):
 *    [x0, x1, x2, u_w, v_w, u_n, v_n, r, a0, a1, a2, b0, b1, b2, pad, pad]
 *  x: position in [0,1]^3 (scene-normalised); (u_w, v_w) and (u_n, v_n):
 *  scattered direction and surface normal as spherical coordinates
 *  normalised to [0,1]^2, u = theta/pi, v = phi/(2 pi) (Table 1's sph());
 *  r: roughness; a, b: diffuse and specular reflectance.  Targets are
 *  float32 [n][3] RGB radiance.
 */
#ifndef NRC_H_
#define NRC_H_

#include <stdint.h>

#if defined(__GNUC__)
#define NRC_API __attribute__((visibility("default")))
#else
#define NRC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* nrc_stream; /* identical to cudaStream_t */

typedef enum nrc_status {
  NRC_OK = 0,
  NRC_ERR_INVALID_ARG = 1,
  NRC_ERR_CUDA = 2,
  NRC_ERR_OOM = 3,
  NRC_ERR_TIMEOUT = 4,
  NRC_ERR_UNSUPPORTED = 5,
  NRC_ERR_BUSY = 6, /* not admitted now (memory budget or frame slot in use): retry later */
  NRC_ERR_BOUNDS = 7 /* a device bounds check failed; raised only by a library built with NRC_DEBUG */
} nrc_status;

/* Arithmetic type of the MLP's matrix products.  NRC_FP32: FP32 SIMT FMA
 * (the parity path).  NRC_FP16 / NRC_BF16: tcgen05 tensor-core products with
 * FP32 accumulation; master weights, Adam moments and the loss stay FP32.
 * NRC_FP8: queries with E4M3 operands (tcgen05 kind::f8f6f4, FP32
 * accumulation): each weight matrix scaled by a power of two from its amax,
 * the encoded inputs by 128, and every hidden layer's activations of a row by
 * a power of two from that row's amax (undone exactly in the next epilogue);
 * training as NRC_FP16.  Batched caches, the server and the allocation-free
 * step do not take it. */
enum { NRC_FP32 = 0, NRC_FP16 = 1, NRC_BF16 = 2, NRC_FP8 = 3 };

/* Encoding primitives (Sec. 5, Fig. 7): CHEAP replaces the sine by the
 * triangle wave tri(x) = 2|x mod 2 - 1| - 1 and the one-blob Gaussian by the
 * quartic 15/16 (1 - x^2)^2; EXACT keeps sine and Gaussian. */
enum { NRC_ENC_CHEAP = 0, NRC_ENC_EXACT = 1 };

/* Normalisation of the relative L2 loss (Eq. 5): LUMINANCE divides every
 * channel by the squared luminance (Rec. 709 weights) of the prediction;
 * PER_CHANNEL divides each channel by its own squared prediction. */
enum { NRC_LOSS_LUMINANCE = 0, NRC_LOSS_PER_CHANNEL = 1 };

/* Execution path.  FUSED: one fused kernel per stage (encoding fused into the
 * first layer, activations on chip).  PLAIN: a separate FP32 kernel per layer
 * with every activation round-tripping through HBM (a reference point). */
enum { NRC_PATH_FUSED = 0, NRC_PATH_PLAIN = 1 };

enum {
  NRC_OPT_ADAM = 0,
  NRC_OPT_SHAMPOO = 1
};

typedef struct nrc_config {
  int32_t width;         /* hidden width; 64 (128: plain FP32 path only, the width-128 variant) */
  int32_t hidden_layers; /* number of hidden layers; 5 (1..8) */
  int32_t dtype;         /* NRC_FP32 | NRC_FP16 | NRC_BF16 */
  int32_t enc_mode;      /* NRC_ENC_CHEAP | NRC_ENC_EXACT */
  int32_t loss_mode;     /* NRC_LOSS_LUMINANCE | NRC_LOSS_PER_CHANNEL */
  int32_t path;          /* NRC_PATH_FUSED | NRC_PATH_PLAIN */
  float pad_value;       /* value of the 2 padding inputs; 1.0 (Sec. 3.6) */
  float lr;              /* Adam learning rate; 1e-2 */
  float beta1, beta2;    /* Adam decay rates; 0.9, 0.99 */
  float adam_eps;        /* Adam epsilon; 1e-8 */
  float loss_eps;        /* epsilon of Eq. 5; 0.01 */
  uint64_t seed;         /* seed of the Xavier-uniform initial weights */
  int32_t ema;           /* 1: keep the weight average of Sec. 3.3, Eq. 2 (read as the bias-corrected
                            average EMA_t = ((1-a) W_t + a eta_{t-1} EMA_{t-1}) / eta_t, eta_t = 1 - a^t),
                            updated by every training step, and query the cache with it; 0 (default):
                            query with the trained weights */
  float ema_alpha;       /* a of Eq. 2; 0.99 */
  int32_t refl_factor;   /* 1: reflectance factorisation (Sec. 5): the prediction is the network output
                            times the record's diffuse + specular albedo (a + b, per channel), in queries and
                            in the training loss; 0 (default) */
  int32_t optimizer;     /* NRC_OPT_ADAM (default; Sec. 5) | NRC_OPT_SHAMPOO (the second-order variant
                            Sec. 5 reports; read as Gupta et al. 2018 with the exponential statistics, root
                            interval and Adam grafting of Anil et al. 2020: per weight matrix
                            W -= lr * D ||A|| / ||D||, D = L^-1/4 m^ R^-1/4, A = Adam's step) */
  int32_t shampoo_interval; /* steps between inverse-root updates; 4 (once per frame) */
  float shampoo_eps;     /* relative regulariser eps * tr(S)/n added to each statistic; 1e-4 */
} nrc_config;

typedef struct nrc_cache nrc_cache;

/* Fills *cfg with the defaults listed above. */
NRC_API void nrc_default_config(nrc_config* cfg);

/* Creates a cache: allocates its state on the current device and draws
 * Xavier-uniform weights U(+-sqrt(6/(fan_in+fan_out))) from SplitMix64(seed)
 * (weights layer after layer, row-major [out][in], FP64 then rounded to
 * FP32); Adam moments and the step counter start at zero.  The weight upload
 * is ordered on `stream`.  *out receives the handle.  Returns
 * NRC_ERR_UNSUPPORTED for widths other than 64 or a dtype the device lacks. */
NRC_API nrc_status nrc_create(const nrc_config* cfg, nrc_stream stream, nrc_cache** out);

/* Frees the cache after synchronising its internal work.  NULL is a no-op. */
NRC_API nrc_status nrc_destroy(nrc_cache* cache);

/* Number of weights (FP32 elements of nrc_get_state's `weights`). */
NRC_API int64_t nrc_param_count(const nrc_cache* cache);

/* Input encoding (Sec. 3.6, Table 1): records[n][16] (device) ->
 * out[n][64] (device) in out_dtype (NRC_FP32 | NRC_FP16 | NRC_BF16).
 * Features: 12 frequency features of each position axis (axis-major, sine or
 * triangle wave of 2^d * pi * x, d = 0..11), one-blob k = 4 of u_w, v_w,
 * u_n, v_n and of 1 - exp(-r), the six albedos, two pad entries. */
NRC_API nrc_status nrc_encode(nrc_cache* cache, const float* records, int64_t n, void* out, int32_t out_dtype,
                      nrc_stream stream);

/* Cache query (Sec. 3.1; Sec. 4 fully fused network): rgb[n][3] (device) =
 * MLP(encode(records[n][16])) with the current weights. */
NRC_API nrc_status nrc_infer(nrc_cache* cache, const float* records, int64_t n, float* rgb, nrc_stream stream);

/* Training-record shuffle and batch gather (Sec. 3.5): for j < batch,
 * rec_out[j] = pool[perm(step * batch + j)] and tgt_out[j] = target[same],
 * perm(i) = (a*i + c) mod n_pool with a, c drawn from SplitMix64(frame_seed)
 * (a = 1 + 4 (h mod floor(n_pool/4)) raised by 2 until gcd(a, n_pool) = 1,
 * c = h' mod n_pool).  Requires (step+1)*batch <= n_pool < 2^31.  All
 * pointers are device pointers; tgt_out may be NULL (target then unused). */
NRC_API nrc_status nrc_gather(const float* pool, const float* target, int64_t n_pool, int64_t batch, uint64_t frame_seed,
                      int32_t step, float* rec_out, float* tgt_out, nrc_stream stream);

/* One optimisation step (Sec. 3.3: several per frame, each on a disjoint
 * slice of the shuffled records): gather batch `step_in_frame` of the frame's
 * pool (as nrc_gather), encode, forward, relative L2 loss (Eq. 5) averaged
 * over the 3*batch terms, backward pass, then Adam on the FP32 master weights
 * (step counter t incremented first).  pool[n_pool][16], target[n_pool][3]
 * are device pointers; loss_out (device, 1 float, may be NULL) receives the
 * batch's loss before the update.  Requires (step_in_frame+1)*batch <=
 * n_pool and batch <= 1048576. */
NRC_API nrc_status nrc_train_step(nrc_cache* cache, const float* pool, const float* target, int64_t n_pool, int64_t batch,
                          uint64_t frame_seed, int32_t step_in_frame, float* loss_out, nrc_stream stream);

/* One frame (Sec. 3.1-3.5): the cache query rgb = infer(queries) with the
 * weights before this frame's training, then n_steps train steps on the
 * pool (steps 0 .. n_steps-1 of frame_seed's shuffle).  loss_out (device,
 * n_steps floats, may be NULL) receives each step's loss.  Device pointers.
 * Since the queries read the weights from before the frame's training, the
 * two are independent: for NRC_FP16 / NRC_BF16 caches on the fused path with
 * Adam (width 64, at most 5 hidden layers, at most 64 steps) the whole frame is ONE persistent
 * launch in which some CTAs run the training steps (grid barriers between
 * the steps, Adam inside the launch) while the others answer the queries,
 * and the training CTAs answer queries once the steps are done.  Its
 * outputs equal nrc_infer's bit for bit; its weights equal those of
 * n_steps x nrc_train_step up to FP32 summation order (the weight-gradient
 * partials come from a different number of CTAs).  Other caches run the
 * query launch and then each step's launches.  The fused launch keeps all
 * its CTAs resident at once (cooperative launch): it needs the whole GPU
 * and NRC_ERR_CUDA is returned if the device cannot host it. */
NRC_API nrc_status nrc_frame(nrc_cache* cache, const float* queries, int64_t n_queries, float* rgb, const float* pool,
                     const float* target, int64_t n_pool, int64_t batch, int32_t n_steps, uint64_t frame_seed,
                     float* loss_out, nrc_stream stream);

/* How nrc_frame splits the fused launch: train_ctas = 0 (default) chooses
 * the number of training CTAs per frame from a model of the frame's length
 * (the training's dependent chain against the SM time of all the work), and
 * runs a frame without queries as separate launches (faster for training
 * alone); 1 .. SM count fixes it (capped at the batch's 128-row tiles) and
 * takes the fused launch for frames without queries too; -1 runs every frame
 * as separate launches (queries, then each step's gradient and Adam kernels).
 * Host-side setting; INVALID_ARG outside [-1, SM count]. */
NRC_API nrc_status nrc_set_frame_ctas(nrc_cache* cache, int32_t train_ctas);

/* The number of training CTAs nrc_frame would use for this frame shape, or
 * -1 if the frame would not take the fused launch. */
NRC_API int32_t nrc_frame_ctas(const nrc_cache* cache, int64_t n_queries, int64_t batch, int32_t n_steps);

/* nrc_frame with HOST buffers: copies queries, pool and target host->device
 * into library-owned staging buffers (grown on demand), runs the frame, and
 * copies rgb[n_queries][3] and the n_steps losses (loss_out, host, may be
 * NULL) back.  Synchronises `stream` before returning.  Pinned host memory
 * gives asynchronous copies. */
NRC_API nrc_status nrc_frame_host(nrc_cache* cache, const float* queries, int64_t n_queries, float* rgb, const float* pool,
                          const float* target, int64_t n_pool, int64_t batch, int32_t n_steps, uint64_t frame_seed,
                          float* loss_out, nrc_stream stream);

/* Copies the state out (host pointers, each nrc_param_count floats; any may
 * be NULL): FP32 weights layer after layer, row-major [out][in]; Adam first
 * and second moments in the same layout; *step = Adam step counter.
 * Synchronises `stream`. */
NRC_API nrc_status nrc_get_state(nrc_cache* cache, float* weights, float* adam_m, float* adam_v, int64_t* step,
                         nrc_stream stream);

/* Replaces the state (host pointers as in nrc_get_state; NULL moments are
 * zeroed; weights must not be NULL) and rebuilds the low-precision weight
 * image.  Synchronises `stream`. */
NRC_API nrc_status nrc_set_state(nrc_cache* cache, const float* weights, const float* adam_m, const float* adam_v,
                         int64_t step, nrc_stream stream);

/* Selects NRC_PATH_FUSED or NRC_PATH_PLAIN for later calls. */
NRC_API nrc_status nrc_set_path(nrc_cache* cache, int32_t path);

/* Synchronises `stream`, then reads and clears the device error word:
 * NRC_ERR_TIMEOUT if a bounded device wait gave up since the last check;
 * NRC_ERR_BOUNDS if a device bounds check of an NRC_DEBUG build failed (the
 * access it guarded was skipped; the results of the calls since the last
 * check are then undefined). */
NRC_API nrc_status nrc_check_error(nrc_cache* cache, nrc_stream stream);

/* Number of kernels the library launched on this cache since creation. */
NRC_API int64_t nrc_launch_count(const nrc_cache* cache);

/* ----------------------------------------------------------------------
 * Batched caches: several independent caches (each with its own weights,
 * Adam state and training data) served together.  All caches of a batch must
 * have been created with identical configurations (FP16 or BF16), on the
 * same device.  The batch object owns its descriptors and the weight-gradient
 * partials of batched training steps; the caches stay owned by the caller.
 */
typedef struct nrc_batch nrc_batch;

/* Plans batched calls over caches[0 .. n_caches-1] (host array of handles). */
NRC_API nrc_status nrc_batch_create(nrc_cache* const* caches, int32_t n_caches, nrc_batch** out);

/* Frees the batch (not the caches) after synchronising the device. */
NRC_API nrc_status nrc_batch_destroy(nrc_batch* batch);

/* Cache queries of every cache in ONE persistent launch (Sec. 4's fused
 * network per cache): rgb[c][n[c]][3] = MLP_c(encode(records[c][n[c]][16])).
 * records, n and rgb are host arrays of n_caches entries; records[c] and
 * rgb[c] are device pointers as in nrc_infer.  With unit_tiles 0 (the
 * default) each CTA takes one contiguous range of all the caches' 128-row
 * tiles (cache after cache, equal counts); otherwise the work is cut into
 * units of up to unit_tiles tiles of one cache, taken by the CTAs from a
 * device counter.  Each row is computed exactly as nrc_infer computes it.
 * Descriptors are uploaded (asynchronously) only when they differ from the
 * previous call's, so the launch can be captured in a CUDA graph and
 * replayed for the same buffers. */
NRC_API nrc_status nrc_batch_infer(nrc_batch* batch, const float* const* records, const int64_t* n,
                                   float* const* rgb, nrc_stream stream);

/* One training step of every cache in one gradient launch and one Adam
 * launch: cache c trains on batch `step` of frame_seed[c]'s shuffle of its
 * pool (as nrc_train_step), batch[c] <= 65536 records (0 skips the cache).
 * The CTAs (at most one per SM in all) are shared out so that the largest
 * number of 128-record tiles any CTA trains is as small as possible.  All
 * arguments are host arrays of n_caches entries; pool[c], target[c] and
 * loss_out[c] (may be NULL, as may loss_out itself) are device pointers. */
NRC_API nrc_status nrc_batch_train_step(nrc_batch* batch, const float* const* pool, const float* const* target,
                                        const int64_t* n_pool, const int64_t* batch_size,
                                        const uint64_t* frame_seed, int32_t step, float* const* loss_out,
                                        nrc_stream stream);

/* nrc_batch_train_step with the frame seeds in DEVICE memory: frame_seed_dev
 * is a device array of n_caches uint64 (8-byte aligned), read by the gradient
 * kernel when it runs, which derives each cache's shuffle from it.  The step's
 * descriptors then do not depend on the seeds; they are uploaded only when
 * they differ from the previous upload (pools, batches, step, loss pointers),
 * so repeated calls launch the two kernels only and can be captured in a CUDA
 * graph together with nrc_batch_infer.  Replays train on whatever seeds the
 * array holds then (write it, stream-ordered, before each replay).  Same
 * results as nrc_batch_train_step with those seeds. */
NRC_API nrc_status nrc_batch_train_step_dev(nrc_batch* batch, const float* const* pool, const float* const* target,
                                            const int64_t* n_pool, const int64_t* batch_size,
                                            const uint64_t* frame_seed_dev, int32_t step, float* const* loss_out,
                                            nrc_stream stream);

/* Sets the work-unit size of nrc_batch_infer (1 .. 4096 tiles; 0, the
 * default: one contiguous range per CTA). */
NRC_API nrc_status nrc_batch_set_unit_tiles(nrc_batch* batch, int32_t unit_tiles);

/* Training partition of nrc_batch_train_step.  0 (default): the CTAs (one
 * per SM in all) are shared out so that the largest number of tiles any CTA
 * trains is as small as possible.
 * T > 0 (up to 4096): cache c gets ceil(tiles_c / T) CTAs, tiles_c = its
 * batch in 128-record tiles, whatever the other caches train; its weight
 * gradients are then summed in the same order as when it trains alone, so
 * its result is bit-identical alone and in any mix. */
NRC_API nrc_status nrc_batch_set_train_tiles(nrc_batch* batch, int32_t train_tiles);

/* Autotuner: runs nrc_batch_infer on the given buffers with each candidate
 * work-unit size (0 and 5 .. 160 tiles), keeps the fastest (CUDA-event timing; it
 * synchronises the stream) and reports it in *chosen (may be NULL). */
NRC_API nrc_status nrc_batch_autotune(nrc_batch* batch, const float* const* records, const int64_t* n,
                                      float* const* rgb, nrc_stream stream, int32_t* chosen);

/* ----------------------------------------------------------------------
 * Serving runtime: frames streamed from several viewports, each with its own
 * cache, batched continuously onto this GPU (the paper renders one viewport;
 * this is the multi-viewport serving form of its per-frame work, Sec. 3.4 and
 * Fig. 4: per frame, cache queries for every pixel's path vertex, then the
 * frame's training steps).
 *
 * A viewport keeps resident on the device, owned by the server: its cache
 * (weights, Adam state), its training-record pool with targets, and n_slots
 * frame buffers (query records in, RGB out, per-step losses).  It is admitted
 * only if that memory fits the server's budget.  The caller writes a frame's
 * query records into a slot's buffer, the training pool into the pool buffer
 * (both with work complete before it submits), and submits the frame; a
 * scheduler thread batches pending frames -- in arrival order, at most one
 * per viewport -- into one persistent query launch followed by train_steps
 * batched training steps (viewport v's frame trains on batch k of the
 * frame seed's shuffle of its pool in step k, Sec. 3.5), keeping at most
 * max_inflight batches queued on the server's stream.  Frames arriving while
 * a batch runs join the next batch.  Every viewport trains with the same CTA
 * partition alone and in any mix (train_tiles), so a frame's outputs and the
 * viewport's weights are bit-identical whatever else is served.
 */
typedef struct nrc_server nrc_server;

typedef struct nrc_server_config {
  uint64_t memory_budget; /* bytes all viewports may keep resident (default 16 GiB) */
  int32_t max_viewports;  /* viewports open at once (default 16) */
  int32_t max_inflight;   /* batches queued on the GPU at once (default 2) */
  int32_t train_steps;    /* training steps per frame (default 4) */
  int32_t train_batch;    /* records per training step (default 16384, <= 65536) */
  int32_t train_tiles;    /* 128-record tiles per training CTA (default 4) */
  int32_t unit_tiles;     /* 128-row tiles per query work unit (default 0: one contiguous range per CTA) */
} nrc_server_config;

/* One finished frame.  Times are CLOCK_MONOTONIC nanoseconds (nrc_now_ns). */
typedef struct nrc_frame_done {
  int32_t viewport;
  int32_t slot;
  int64_t tag;          /* the caller's tag from nrc_server_submit */
  int64_t n_queries;
  int64_t arrival_ns;   /* the caller's arrival time from nrc_server_submit */
  int64_t submit_ns;    /* when nrc_server_submit accepted it */
  int64_t launch_ns;    /* when its batch was issued */
  int64_t done_ns;      /* when the stream reached the end of its batch */
  int32_t batch_frames; /* frames in its batch */
  int32_t failed;       /* 1 if its batch failed to launch (see nrc_server_poll's status) */
} nrc_frame_done;

typedef struct nrc_server_info {
  uint64_t memory_used;
  uint64_t memory_budget;
  int64_t frames_done;
  int64_t batches;
  int64_t queries_done;
  int64_t pending;
  int32_t viewports;
  int32_t inflight;
} nrc_server_info;

NRC_API void nrc_server_default_config(nrc_server_config* cfg);

/* Monotonic clock of the frame timings, in nanoseconds. */
NRC_API int64_t nrc_now_ns(void);

/* Creates a server for caches of configuration *cache_cfg (NRC_FP16 or
 * NRC_BF16; every viewport's cache must equal it but for the seed) on the
 * current device, with its own non-blocking stream and scheduler thread. */
NRC_API nrc_status nrc_server_create(const nrc_server_config* cfg, const nrc_config* cache_cfg, nrc_server** out);

/* Waits for every submitted frame, stops the thread, frees all viewports. */
NRC_API nrc_status nrc_server_destroy(nrc_server* server);

/* Admits a viewport: creates its cache from *cache_cfg (Xavier init from
 * cache_cfg->seed) and allocates its pool (n_pool >= train_steps x
 * train_batch records) and n_slots (1..8) frame buffers of max_queries
 * records.  NRC_ERR_BUSY if the memory would exceed the budget or all
 * viewport entries are in use (nothing allocated; retry after a close).
 * *id_out receives the viewport id. */
NRC_API nrc_status nrc_server_open_viewport(nrc_server* server, const nrc_config* cache_cfg, int64_t max_queries,
                                            int64_t n_pool, int32_t n_slots, int32_t* id_out);

/* Waits for the viewport's frames, then frees its cache and buffers. */
NRC_API nrc_status nrc_server_close_viewport(nrc_server* server, int32_t id);

/* Device pointers of a slot's buffers (server-owned): records [max_queries][16]
 * (caller writes), rgb [max_queries][3] and losses [train_steps] (valid once
 * the frame is reported done).  Any out-pointer may be NULL. */
NRC_API nrc_status nrc_server_viewport_buffers(nrc_server* server, int32_t id, int32_t slot, float** records,
                                               float** rgb, float** losses);

/* Device pointers of the viewport's training pool [n_pool][16] and targets
 * [n_pool][3] (caller writes) and its cache handle (for nrc_get_state /
 * nrc_set_state after nrc_server_drain; the server owns it). */
NRC_API nrc_status nrc_server_viewport_pool(nrc_server* server, int32_t id, float** pool, float** target,
                                            nrc_cache** cache);

/* Queues frame `tag` of viewport `id`: n_queries (<= max_queries) records in
 * slot `slot`, training shuffle seeded by frame_seed.  NRC_ERR_BUSY while the
 * slot's previous frame is in flight.  Does not block. */
NRC_API nrc_status nrc_server_submit(nrc_server* server, int32_t id, int32_t slot, int64_t n_queries,
                                     uint64_t frame_seed, int64_t arrival_ns, int64_t tag);

/* Moves up to max_out finished frames into out[] (*n_out of them), waiting up
 * to timeout_ms for the first if none is ready.  Returns the first error a
 * batch met, if any (its frames are reported with failed = 1). */
NRC_API nrc_status nrc_server_poll(nrc_server* server, nrc_frame_done* out, int32_t max_out, int32_t timeout_ms,
                                   int32_t* n_out);

/* Holds (paused != 0) or releases (0) the scheduler: while held, submitted
 * frames wait and no batch is issued; on release the pending frames are
 * batched as usual (in arrival order, at most one per viewport per batch).
 * A renderer can hold, submit every viewport's frame of a display interval
 * and release them into one batch.  nrc_server_drain,
 * nrc_server_close_viewport and nrc_server_destroy release a held server. */
NRC_API nrc_status nrc_server_pause(nrc_server* server, int32_t paused);

/* Blocks until every submitted frame is done and the stream is idle. */
NRC_API nrc_status nrc_server_drain(nrc_server* server);

NRC_API nrc_status nrc_server_query(nrc_server* server, nrc_server_info* out);

/* Training step that allocates nothing (the paper has no counterpart; this
 * serves callers that cannot allocate device memory when they train -- e.g.
 * a renderer whose engine hands out every device allocation itself under a
 * fixed budget, or a frame loop that must not take the device-wide
 * synchronisation cudaMalloc / cudaFree can imply).
 *
 * Runs the same training step as nrc_train_step for a cache with config
 * *cfg (dtype NRC_FP16 or NRC_BF16, width 64, 1..5 hidden layers; the
 * constants checked as nrc_create checks them) -- equal to it up to FP32
 * summation order, since its weight-gradient partials come from at most 64
 * CTAs -- on state
 * the CALLER owns, all device pointers: weights, adam_m, adam_v
 * (nrc_param_count floats each, layout of nrc_get_state; read and updated
 * in place) and *step_counter (device int64, incremented).  pool, target,
 * n_pool, batch (<= 65536), frame_seed, step_in_frame and loss_out as in
 * nrc_train_step; err_out (device int32, may be NULL) receives the device
 * error word of this call (0, or NRC's timeout bit 1).
 *
 * Scratch lives in file-scope device arrays of fixed size: 64
 * weight-gradient partials of 20,676 floats (5.3 MB), a 43,008-byte 16-bit
 * weight image and an error word.  Sizes beyond that (other widths, more
 * layers, batch > 65536) are rejected with NRC_ERR_INVALID_ARG before
 * anything is launched.  No cudaMalloc, cudaFree or allocating library
 * routine is called.  The arrays come into being when the CUDA runtime loads
 * their module on a device, and stay until exit; with lazy module loading
 * (the CUDA default) that happens at the first call on each device, which
 * looks up their device addresses with cudaGetSymbolAddress (with that device
 * current), so that first call lowers the device's free memory by about
 * 6 MB and no later call changes it.  A call with batch 0 (cfg checked; the
 * other pointers may be NULL) makes that first lookup and launches nothing:
 * make it at start-up, before any stream capture.  Every call shares the arrays: each call rebuilds the weight
 * image and clears the error word before using them, and calls whose work
 * overlaps on the GPU (other streams, other threads) race on the scratch and
 * must be serialised by the caller. */
NRC_API nrc_status nrc_train_step_noalloc(const nrc_config* cfg, float* weights, float* adam_m, float* adam_v,
                                          int64_t* step_counter, const float* pool, const float* target,
                                          int64_t n_pool, int64_t batch, uint64_t frame_seed,
                                          int32_t step_in_frame, float* loss_out, int32_t* err_out,
                                          nrc_stream stream);

/* Weight average of a cache created with cfg.ema = 1 (Sec. 3.3, Eq. 2): copies
 * the nrc_param_count FP32 averaged weights (layout of nrc_get_state) to the
 * host buffer ema (synchronises the stream).  Before the first training step
 * the average equals the weights; nrc_set_state restarts it at the weights
 * it sets.  NRC_ERR_UNSUPPORTED for a cache without an average. */
NRC_API nrc_status nrc_get_ema(nrc_cache* cache, float* ema, nrc_stream stream);

/* Replaces the weight average (host buffer, nrc_param_count floats) and the
 * 16-bit image the queries read (synchronises the stream). */
NRC_API nrc_status nrc_set_ema(nrc_cache* cache, const float* ema, nrc_stream stream);

/* ----------------------------------------------------------------------
 * Training-record pipeline around the cache query (Sec. 3.3 self-training,
 * Sec. 3.4 path termination with the area-spread heuristic, Eqs. 3-4,
 * Sec. 3.5 one training path per screen tile).  Input: the vertices a path
 * tracer produced for every pixel, n_vertices per pixel, 24 floats each:
 *   0-2 position x_i, 3-4 direction towards x_{i-1} and 5-6 normal (both
 *   (theta/pi, phi/(2 pi))), 7 roughness, 8-10 diffuse and 11-13 specular
 *   albedo (0-13 are the query record's first 14 floats), 14 pdf (solid angle)
 *   of the direction that reached x_i, 15 |cos| of that direction with the
 *   normal at x_i, 16-18 emitted radiance, 19-21 throughput weight of the
 *   bounce leaving x_i (BSDF cos / pdf), 22 a uniform for Russian roulette,
 *   23 unused.
 * Decisions: the rendering path ends at the first x_n (n >= 1, 0-based) whose
 * spread (sum_{i=1..n} sqrt(|x_{i-1} - x_i|^2 / (pdf_i cos_i)))^2 exceeds
 * c a_0, a_0 = |camera - x_0|^2 / (4 pi cos_0), or at the last vertex; every
 * tile x tile block of pixels has one training path, the pixel at offset
 * (tile_ox, tile_oy); its suffix restarts the sum at x_n and ends at the first
 * x_m past the threshold -- or, in tiles t with t % 16 == unbiased_phase,
 * continues from each vertex j >= n with probability rr_survive (roulette
 * uniform < rr_survive; weight 1/rr_survive) and ends where it stops.  These
 * decisions are computed with round-to-nearest FP32 operations in a fixed
 * order (include no fused multiply-adds), hence reproducible. */
typedef struct nrc_paths {
  const float* vertices; /* device, [width*height][n_vertices][24], pixels row-major, 16-byte aligned */
  int32_t width, height, n_vertices; /* 2 <= n_vertices <= 64 */
  float camera[3];       /* x_{-1}: the camera position */
} nrc_paths;

typedef struct nrc_path_params {
  float c;               /* spread threshold; 0.01 (Sec. 3.4) */
  int32_t tile;          /* side of a training tile in pixels */
  int32_t tile_ox, tile_oy; /* this frame's offset of the training pixel in each tile, in [0, tile) */
  int32_t unbiased_phase; /* tiles with t % 16 == phase get a roulette-only suffix (u = 1/16); -1: none */
  float rr_survive;      /* roulette survival probability of those suffixes; 0.8 */
} nrc_path_params;

/* Number of training tiles, ceil(width/tile) * ceil(height/tile) (0 on bad sizes). */
NRC_API int64_t nrc_paths_tile_count(int32_t width, int32_t height, int32_t tile);

/* Tile side for the next frame so that the training records approach
 * `target` (Sec. 3.5's adaptive tiling): tile * sqrt(generated / target),
 * rounded, in [1, 256]. */
NRC_API int32_t nrc_paths_adapt_tile(int32_t tile, int64_t generated, int64_t target);

/* Terminates every pixel's rendering path and picks the training paths.
 * Outputs (device, caller-owned): render_queries [pixels][16] (the record of
 * each terminal vertex, for nrc_infer), render_emitted [pixels][3] (emitted
 * light along the path, throughput-weighted), render_throughput [pixels][3]
 * (throughput from the camera to the terminal vertex), tiles [n_tiles][4]
 * int32 {pixel or -1, n, m, unbiased} and tail_queries [n_tiles][16] (the
 * record of x_m, the training path's self-training query; rows of tiles
 * without a training path are left as they are).  tail_queries may be
 * render_queries + 16 * pixels, so that one nrc_infer over pixels + n_tiles
 * records answers both.  Record and tile buffers must be 16-byte aligned. */
NRC_API nrc_status nrc_paths_terminate(const nrc_paths* paths, const nrc_path_params* params,
                                       float* render_queries, float* render_emitted, float* render_throughput,
                                       int32_t* tiles, float* tail_queries, nrc_stream stream);

/* Length of the offsets scratch nrc_paths_records needs for n_tiles training
 * tiles: n_tiles entries plus one per 2048 tiles (the scan's block totals). */
NRC_API int64_t nrc_paths_offsets_count(int64_t n_tiles);

/* Self-training records (Sec. 3.3): for each training path, in tile order, the
 * records of x_0 .. x_{m-1} with targets L_j = w_j (Le_{j+1} + L_{j+1}) from
 * L_m = tail_rgb[t] (the cache's value at x_m; 0 where the roulette ended an
 * unbiased suffix).  Writes min(total, max_records) records into pool
 * [max][16] and targets [max][3]; offsets (device int64 scratch of
 * nrc_paths_offsets_count(n_tiles) entries) receives in its first n_tiles
 * entries each path's first record, *count (device int64) the total. */
NRC_API nrc_status nrc_paths_records(const nrc_paths* paths, const nrc_path_params* params, const int32_t* tiles,
                                     const float* tail_rgb, float* pool, float* targets, int64_t max_records,
                                     int64_t* offsets, int64_t* count, nrc_stream stream);

/* Pixel radiance: image = render_emitted + render_throughput * rgb (rgb: the
 * cache's value at each terminal vertex), all [n][3] device arrays. */
NRC_API nrc_status nrc_paths_composite(const float* render_emitted, const float* render_throughput,
                                       const float* rgb, int64_t n, float* image, nrc_stream stream);

/* Fault injection for tests (faults made on the host; nothing here
 * faults the GPU).  nrc_debug_fail_device_allocs: after `after` more device
 * allocations by this library (process-wide), the next `count` fail as if the
 * device were out of memory; the call that needed them returns NRC_ERR_OOM and
 * frees what it had allocated.  (0, 0) switches it off. */
NRC_API void nrc_debug_fail_device_allocs(int32_t after, int32_t count);

/* Runs, on `stream`, a one-thread kernel that waits through the library's
 * bounded device wait on an mbarrier nothing arrives at, with a limit of
 * limit_us microseconds (1 .. 2,000,000; the kernels use 2 s).  The wait gives
 * up, sets the cache's error word and returns: the next nrc_check_error
 * reports NRC_ERR_TIMEOUT and the cache stays usable. */
NRC_API nrc_status nrc_debug_wait_timeout(nrc_cache* cache, int32_t limit_us, nrc_stream stream);

/* Why the last failing call on this thread failed ("" if none). */
NRC_API const char* nrc_last_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* NRC_H_ */
