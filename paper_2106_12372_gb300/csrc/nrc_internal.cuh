// Internal declarations of the GB300 neural radiance cache library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "nrc.h"

namespace nrc {

constexpr int kRecFloats = 16;  // 64-byte record
constexpr int kEncDims = 64;    // Table 1: 62 features + 2 pad (Sec. 3.6)
constexpr int kOutDims = 3;     // RGB
constexpr int kMaxMats = 9;     // hidden layers <= 8
constexpr int kTile = 128;      // batch rows per tensor-core tile (MMA M)
constexpr int kQuerySlots = 5;  // 128-row tiles in flight per SM in the width-64 query kernels
constexpr int kOutPad = 16;     // output layer padded to N = 16 for the MMA
constexpr int kMaxBatch = 1 << 16;  // training records per step

// Device error word bits.
constexpr int kErrTimeout = 1;
constexpr int kErrBounds = 2;  // a device bounds check of an NRC_DEBUG build failed

// NRC_DCHECK(cond, err): in a build with NRC_DEBUG defined, evaluates cond
// and, where it is false, sets kErrBounds in the error word *err and yields
// false, so that the caller skips the access it guards; otherwise it is the
// constant true and the guarded access always runs.
#ifdef NRC_DEBUG
#define NRC_DCHECK(cond, err) ((cond) ? true : (atomicOr((err), ::nrc::kErrBounds), false))
#else
#define NRC_DCHECK(cond, err) true
#endif
// Bounded device waits give up after this many nanoseconds.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// Fault injection for tests (nrc_debug_fail_device_allocs): after
// g_alloc_skip more device allocations, the next g_alloc_fail ones fail as if
// the device were out of memory.
extern int g_alloc_skip, g_alloc_fail;
cudaError_t dev_alloc_bytes(void** p, size_t bytes);
// Raises a kernel's dynamic shared-memory limit to at least `bytes`.  `done`
// (one per kernel instance) remembers the largest limit set so far, so that
// the attribute is set once per increase, never lowered, and concurrent first
// launches from several host threads are safe.
template <typename K>
inline cudaError_t ensure_smem(K kernel, int bytes, std::atomic<int>* done) {
  if (done->load(std::memory_order_acquire) >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  int cur = done->load(std::memory_order_relaxed);
  while (cur < bytes && !done->compare_exchange_weak(cur, bytes, std::memory_order_acq_rel)) {
  }
  return cudaSuccess;
}

// Every device allocation of the library goes through here.
template <class T>
inline cudaError_t dev_alloc(T** p, size_t bytes) {
  return dev_alloc_bytes(reinterpret_cast<void**>(p), bytes);
}

struct NetShape {
  int n_mats;              // hidden_layers + 1
  int dims[kMaxMats + 1];  // d_0 = 64, d_1..d_H = width, d_L = 3
  int w_off[kMaxMats + 1]; // FP32 element offset of matrix l (row-major [out][in])
  int n_params;
};

// Elements between consecutive weight-gradient partials: the n_params
// gradients, the loss sum, padded to a multiple of 4 floats so that every
// partial starts 16-byte aligned (the tensor-core kernel stores float4).
__host__ __device__ __forceinline__ size_t partial_stride(int n_params) {
  return (size_t(n_params) + 1 + 3) & ~size_t(3);
}

// Byte layout of the 16-bit weight image for the tensor-core kernels: matrix
// l is stored as N_l = round_up(d_{l+1}, 16) rows of K_l = d_l elements,
// K-major with the 128-byte swizzle (8-row atoms of 1024 bytes; 16-byte chunk
// c of row n stored at chunk c ^ (n % 8)), so that one bulk copy puts it in
// shared memory exactly as the tcgen05 descriptors read it.  Only K = 64 is
// supported (one 128-byte swizzle row per matrix row).
struct ImageShape {
  int off[kMaxMats + 1];  // byte offset of matrix l; off[n_mats] = total bytes
  int rows[kMaxMats];     // N_l
};

struct Cache {
  nrc_config cfg;
  NetShape net;
  ImageShape img;
  float* w = nullptr;     // FP32 master weights [n_params]
  float* m = nullptr;     // Adam first moment
  float* v = nullptr;     // Adam second moment
  long long* t = nullptr; // Adam step counter (device)
  uint8_t* wimg = nullptr;        // 16-bit weight image (tensor-core path)
  uint8_t* wimg8 = nullptr;       // E4M3 image of the queried weights (NRC_FP8), + per-layer 1/scale
  bool wimg8_dirty = true;        // the weights changed since wimg8 was built
  float* ema = nullptr;           // weight average of Eq. 2 (cfg.ema), FP32 [n_params]
  uint8_t* wimg_ema = nullptr;    // its 16-bit image (what queries read when cfg.ema)
  // Shampoo (cfg.optimizer): gradient, statistics L_l/R_l and their inverse
  // fourth roots (each 64 x 64, block 2l = L_l, 2l+1 = R_l), per-block ||A||^2
  float* sh_g = nullptr;
  float* sh_stats = nullptr;
  float* sh_roots = nullptr;
  float* sh_anorm = nullptr;
  float* partials = nullptr;      // [max_partials][partial_stride] weight-gradient partials; loss at [n_params]
  int max_partials = 0;
  int* err = nullptr;     // device error word
  // plain-path scratch (grown on demand)
  float* plain_buf = nullptr;
  size_t plain_bytes = 0;
  // nrc_frame_host staging (grown on demand)
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // nrc_frame_host pipeline (created on first use): query uploads, queries and
  // read-backs on their own streams, the queries on a snapshot of the image
  cudaStream_t s_h2d = nullptr, s_query = nullptr, s_d2h = nullptr;
  cudaEvent_t ev_pipe[20] = {};
  uint8_t* wimg_snap = nullptr;
  // fused frame (k_frame_tc, created on first use): the training's working
  // weight images and the launch's device counters; frame_ctas = training
  // CTAs (0: chosen per frame by frame_split(), -1: separate launches)
  uint8_t* wimg_work = nullptr;
  uint8_t* wimg_ema_work = nullptr;
  unsigned* frame_sync = nullptr;
  int frame_ctas = 0;
  long long launches = 0;
  int sm_count = 0;
  int device = 0;
};

// One cache of a batched query: its weight image and its query buffers.
struct BatchCache {
  const uint8_t* wimg;
  const float* rec;
  float* rgb;
  int64_t n;
};
// A run of 128-row tiles [tile_begin, tile_end) of one cache.
struct BatchUnit {
  int cache;
  int tile_begin;
  int tile_end;
};

// The work of one CTA of a batched training step: tiles tile_begin,
// tile_begin + tile_step, ... < tile_end of one cache's batch.
struct TrainJob {
  const float* pool;
  const float* target;
  int64_t n_pool;
  int64_t batch;
  uint64_t a, c;       // the batch's shuffle (Sec. 3.5)
  const uint64_t* seed;  // device: the frame seed to derive a, c from in the kernel (null: a, c as given)
  int step;
  int tile_begin, tile_end, tile_step;
  const uint8_t* wimg;
  float* partial;      // this CTA's weight-gradient partial
  long long* t_ctr;
  int bump_t;          // the cache's first CTA advances its Adam step counter
  float inv3n;
};

// Adam over one cache of a batched step: its state and its partials.
struct AdamJob {
  float* w;
  float* m;
  float* v;
  float* ema;          // null: no weight average
  uint8_t* wimg_ema;
  const long long* t_ctr;
  const float* partials;
  int n_partials;
  uint8_t* wimg;
  float grad_scale;
  float* loss_out;
};

// ---------------------------------------------------------------- host side
void set_error(const char* fmt, ...);
nrc_status cuda_status(cudaError_t e, const char* what);

// Validates a configuration (enums, sizes, optimiser and loss constants):
// NRC_OK, or the status nrc_create returns for it (message set).
nrc_status check_cfg(const nrc_config* cfg);

void make_net_shape(const nrc_config& cfg, NetShape* s);
void make_image_shape(const NetShape& s, ImageShape* img);

// Shuffle parameters (Sec. 3.5): perm(i) = (a*i + c) mod n_pool.
void lcg_params(int64_t n_pool, uint64_t frame_seed, uint64_t* a, uint64_t* c);

// The frame's shuffle of a pool of n_pool records (Sec. 3.5): the full-period
// LCG i -> (a i + c) mod n_pool whose multiplier and increment come from
// SplitMix64 (Steele, Lea & Flood 2014) of frame_seed; a is 1 mod 4 and
// coprime to n_pool, the Hull-Dobell conditions.  Host and device compute it
// alike (lcg_params is this on the host).
__host__ __device__ __forceinline__ uint64_t splitmix64_next(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ void lcg_shuffle(int64_t n_pool, uint64_t frame_seed, uint64_t* a_out,
                                                     uint64_t* c_out) {
  const uint64_t N = uint64_t(n_pool);
  uint64_t st = frame_seed;
  const uint64_t h = splitmix64_next(st);
  const uint64_t h2 = splitmix64_next(st);
  uint64_t a = N >= 4 ? 1 + 4 * (h % (N / 4)) : 1;
  auto gcd = [](uint64_t x, uint64_t y) {
    while (y) {
      const uint64_t t = x % y;
      x = y;
      y = t;
    }
    return x;
  };
  while (N > 1 && gcd(a, N) != 1) a += 2;
  *a_out = a;
  *c_out = N ? h2 % N : 0;
}

// Kernel launchers (each returns the launch's cudaError_t).
// Grows the weight-gradient partial buffer to at least `count` partials.
cudaError_t ensure_partials(Cache* c, int count);

cudaError_t launch_gather(const float* pool, const float* target, int64_t n_pool, int64_t batch, uint64_t a,
                          uint64_t c, int step, float* rec_out, float* tgt_out, cudaStream_t st);
cudaError_t launch_encode(const float* rec, int64_t n, void* out, int out_dtype, int enc_mode, float pad,
                          cudaStream_t st);
cudaError_t launch_infer_simt(Cache* c, const float* rec, int64_t n, float* rgb, cudaStream_t st);
// What one training CTA trains: its cache's data, state and images, and its
// place among the cache's T training CTAs (b), with the cache's own grid
// barrier counter.  The frame kernel's training CTAs all train the frame's
// cache; a batched training launch gives each CTA one cache of the batch.
struct TrainView {
  const float* pool;
  const float* target;
  int64_t n_pool;
  int64_t batch;
  uint64_t a, c;          // the shuffle (Sec. 3.5)
  const uint64_t* seed;   // device: the frame seed to derive a, c from (null: as given)
  int step0;              // index of the first step (its batch of the shuffle)
  int T, b;
  float* w;
  float* m;
  float* v;
  float* ema;             // null: no weight average
  long long* t_ctr;
  const uint8_t* img_in;  // image of the weights the first step starts from
  uint8_t* img_work;      // the image every step writes
  uint8_t* img_ema_work;
  float* partials;        // [T][partial_stride]
  unsigned* bar;          // the T CTAs' grid barrier counter
  float* loss_out;
  float inv3n;
};

// Batched training with the frame kernel's training role (k_frame.cu): one
// cooperative launch of n_views <= SM-count CTAs, CTA k training views[k]
// (device array) for n_steps steps; counters: n_counters - 1 barrier
// counters (the views' bar) and a retire counter, zero at launch and left zero.
bool train_views_ok(const Cache* proto);
cudaError_t launch_train_views(const Cache* proto, const TrainView* views, int n_views, unsigned* counters,
                               int n_counters, int n_steps, cudaStream_t st);
// Width-128 FP16 / BF16 queries on the tensor cores (k_tc128.cu).
cudaError_t launch_infer_tc128(Cache* c, const float* rec, int64_t n, float* rgb, cudaStream_t st);
cudaError_t launch_train_simt(Cache* c, const float* pool, const float* target, int64_t n_pool, int64_t batch,
                              uint64_t a, uint64_t cc, int step, int* n_partials, cudaStream_t st);
cudaError_t launch_adam(Cache* c, int n_partials, float grad_scale, float* loss_out, cudaStream_t st);
cudaError_t launch_build_image(Cache* c, cudaStream_t st);
// Shampoo step after a gradient launch (replaces launch_adam when cfg.optimizer).
cudaError_t launch_shampoo(Cache* c, int n_partials, float grad_scale, float* loss_out, cudaStream_t st);
constexpr size_t kShampooStatFloats = 64 * 64;  // one statistic (or root), 64 x 64
// 16-bit image of an arbitrary FP32 weight set of c's shape into img.
cudaError_t launch_build_image_of(const Cache* c, const float* w, uint8_t* img, cudaStream_t st);
// What queries read: the weight average when the cache keeps one.
inline const float* query_weights(const Cache* c) { return c->cfg.ema ? c->ema : c->w; }
inline const uint8_t* query_image(const Cache* c) { return c->cfg.ema ? c->wimg_ema : c->wimg; }
cudaError_t launch_step_increment(Cache* c, cudaStream_t st);
// Waits, through the kernels' bounded mbarrier wait, on an mbarrier that
// nothing arrives at; gives up after limit_ns and sets kErrTimeout in *err.
cudaError_t launch_wait_probe(int* err, unsigned long long limit_ns, cudaStream_t st);
// image: the weight image to read (nullptr: the cache's queried image)
cudaError_t launch_infer_tc(Cache* c, const float* rec, int64_t n, float* rgb, cudaStream_t st,
                            const uint8_t* image = nullptr);
// E4M3 image (64-byte swizzle, matrix l at img8_offset(net, l)) of the queried
// weights with its per-layer 1/scale floats after the last matrix.
int img8_offset(const NetShape& net, int l);
constexpr int kImg8ScaleBytes = 48;  // per-layer 1/scale floats (kMaxMats of 12), a multiple of 16 bytes
cudaError_t launch_build_image_fp8(Cache* c, cudaStream_t st);
cudaError_t launch_infer_fp8(Cache* c, const float* rec, int64_t n, float* rgb, cudaStream_t st);
inline bool fp16_like(int dtype) { return dtype == NRC_FP16 || dtype == NRC_FP8; }
// One persistent launch over the units of several caches (device arrays);
// proto supplies the shape, dtype and encoding shared by all of them.
cudaError_t launch_infer_batched(const Cache* proto, const BatchCache* caches, const BatchUnit* units, int n_units,
                                 unsigned* counter, int grid, cudaStream_t st, const int* unit_off = nullptr);
cudaError_t launch_train_tc(Cache* c, const float* pool, const float* target, int64_t n_pool, int64_t batch,
                            uint64_t a, uint64_t cc, int step, int* n_partials, float* grad_scale, cudaStream_t st);
// One training launch over several caches (device array of per-CTA jobs) and
// one Adam launch over their weights.
cudaError_t launch_train_batched(const Cache* proto, const TrainJob* jobs, int n_jobs, cudaStream_t st);
cudaError_t launch_adam_batched(const Cache* proto, const AdamJob* jobs, int n_jobs, cudaStream_t st);
// One persistent launch for a frame's queries and its n_steps training steps
// (k_frame_tc): n_train CTAs train while the others answer queries.
cudaError_t launch_frame_tc(Cache* c, const float* rec, int64_t n_q, float* rgb, const float* pool, const float* target,
                            int64_t n_pool, int64_t batch, int n_steps, uint64_t a, uint64_t cc, float* loss_out,
                            int n_train, cudaStream_t st);
// Training CTAs of a fused frame chosen from a model of the frame's length.
int frame_split(const Cache* c, int64_t n_q, int64_t batch, int n_steps);
// Plain per-layer FP32 path.
cudaError_t plain_infer(Cache* c, const float* rec, int64_t n, float* rgb, cudaStream_t st);
cudaError_t plain_train(Cache* c, const float* pool, const float* target, int64_t n_pool, int64_t batch,
                        uint64_t a, uint64_t cc, int step, float* loss_out, cudaStream_t st);

// ------------------------------------------------------------- device side
// Input encoding of one record (Sec. 3.6, Table 1; Sec. 5 cheap primitives).
// Writes the 64 features in order: x0 d=0..11, x1, x2 (frequency), one-blob
// of u_w, v_w, u_n, v_n, 1-exp(-r) (4 bins each), a0..a2, b0..b2, pad, pad.

// Triangle wave standing in for sin(pi*y) (Fig. 7): tri(y - 1/2) with
// tri(t) = 2|t mod 2 - 1| - 1, evaluated as |4 frac(y/2 - 1/4) - 2| - 1.
// For y = 2^d x with x in [0, 1] the only rounding is in y/2 - 1/4 (at most
// 2^-25), i.e. at most ~1.2e-7 in the result.
__device__ __forceinline__ float tri_sin(float y) {
  const float t = fmaf(y, 0.5f, -0.25f);
  const float f = t - floorf(t);
  return fabsf(fmaf(4.0f, f, -2.0f)) - 1.0f;
}

// Clamped antiderivative of the quartic kernel 15/16 (1 - y^2)^2:
// Q(y) = 15/16 y (1 - 2/3 y^2 + 1/5 y^4) on [-1, 1], +-1/2 outside.
__device__ __forceinline__ float quartic_cdf(float y) {
  y = fminf(1.0f, fmaxf(-1.0f, y));
  const float y2 = y * y;
  return y * fmaf(y2, fmaf(y2, 0.1875f, -0.625f), 0.9375f);
}

// Twice the mass of a standard Gaussian between 0 and y (bins are scaled by k).
__device__ __forceinline__ float gauss_cdf2(float y) { return erff(y * 0.70710678118654752f); }

template <int MODE>
__device__ __forceinline__ void oneblob4(float s, float* out) {
  // Bin i of k = 4 holds the kernel mass over [i/4, (i+1)/4]; kernel width 1/4.
  const float ks = 4.0f * s;
  float prev = (MODE == 0) ? quartic_cdf(-ks) : gauss_cdf2(-ks);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float hi = float(i + 1) - ks;
    const float cur = (MODE == 0) ? quartic_cdf(hi) : gauss_cdf2(hi);
    out[i] = (MODE == 0) ? cur - prev : 0.5f * (cur - prev);
    prev = cur;
  }
}

// Packed FP32 pairs: one instruction computes both lanes, each rounded exactly
// as the scalar operation, so the paired code below gives the same bits as
// its scalar form with half the arithmetic instructions.
struct F2 {
  float x, y;
};
__device__ __forceinline__ F2 fma_x2(F2 a, F2 b, F2 c) {
  F2 d;
  asm("{\n\t.reg .b64 a, b, c;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\tmov.b64 c, {%6, %7};\n\t"
      "fma.rn.f32x2 a, a, b, c;\n\tmov.b64 {%0, %1}, a;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ F2 sub_x2(F2 a, F2 b) {
  F2 d;
  asm("{\n\t.reg .b64 a, b;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\tsub.rn.f32x2 a, a, b;\n\t"
      "mov.b64 {%0, %1}, a;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ F2 mul_x2(F2 a, F2 b) {
  F2 d;
  asm("{\n\t.reg .b64 a, b;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\tmul.rn.f32x2 a, a, b;\n\t"
      "mov.b64 {%0, %1}, a;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// quartic_cdf of two arguments
__device__ __forceinline__ F2 quartic_cdf_x2(F2 y) {
  y.x = fminf(1.0f, fmaxf(-1.0f, y.x));
  y.y = fminf(1.0f, fmaxf(-1.0f, y.y));
  const F2 y2 = mul_x2(y, y);
  return mul_x2(y, fma_x2(y2, fma_x2(y2, F2{0.1875f, 0.1875f}, F2{-0.625f, -0.625f}), F2{0.9375f, 0.9375f}));
}

// oneblob4<0> of two values side by side (a's bins to oa, b's to ob)
__device__ __forceinline__ void oneblob4_quartic_x2(float a, float b, float* oa, float* ob) {
  const F2 ks = mul_x2(F2{4.0f, 4.0f}, F2{a, b});
  F2 prev = quartic_cdf_x2(F2{-ks.x, -ks.y});
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const F2 cur = quartic_cdf_x2(sub_x2(F2{float(i + 1), float(i + 1)}, ks));
    const F2 m = sub_x2(cur, prev);
    oa[i] = m.x;
    ob[i] = m.y;
    prev = cur;
  }
}

template <int MODE>
__device__ __forceinline__ void encode_record(const float* r, float pad, float* f) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (MODE == 0) {
      // tri(2^d x - 1/2) = |4 frac(2^(d-1) x - 1/4) - 2| - 1; 2^(d-1) x is exact
      const F2 xx{r[j], r[j]};
#pragma unroll
      for (int d = 0; d < 12; d += 2) {
        const F2 t = fma_x2(xx, F2{float(1 << d) * 0.5f, float(2 << d) * 0.5f}, F2{-0.25f, -0.25f});
        const F2 u = fma_x2(F2{4.0f, 4.0f}, sub_x2(t, F2{floorf(t.x), floorf(t.y)}), F2{-2.0f, -2.0f});
        f[12 * j + d] = fabsf(u.x) - 1.0f;
        f[12 * j + d + 1] = fabsf(u.y) - 1.0f;
      }
    } else {
#pragma unroll
      for (int d = 0; d < 12; ++d) f[12 * j + d] = sinpif(r[j] * float(1 << d));
    }
  }
  if (MODE == 0) {
    oneblob4_quartic_x2(r[3], r[4], f + 36, f + 40);
    oneblob4_quartic_x2(r[5], r[6], f + 44, f + 48);
  } else {
    oneblob4<MODE>(r[3], f + 36);
    oneblob4<MODE>(r[4], f + 40);
    oneblob4<MODE>(r[5], f + 44);
    oneblob4<MODE>(r[6], f + 48);
  }
  oneblob4<MODE>(-expm1f(-r[7]), f + 52);
#pragma unroll
  for (int j = 0; j < 6; ++j) f[56 + j] = r[8 + j];
  f[62] = pad;
  f[63] = pad;
}

// Half of the 64 features: half 0 -> features 0..31 (x0 d=0..11, x1 d=0..11,
// x2 d=0..7); half 1 -> features 32..63 (x2 d=8..11, the five one-blobs, the
// albedos, the pad).  Same arithmetic as encode_record.
template <int MODE>
__device__ __forceinline__ void encode_record_half(const float* r, float pad, int half, float* f) {
  if (half == 0) {
#pragma unroll
    for (int d = 0; d < 12; ++d) {
      f[d] = (MODE == 0) ? tri_sin(r[0] * float(1 << d)) : sinpif(r[0] * float(1 << d));
      f[12 + d] = (MODE == 0) ? tri_sin(r[1] * float(1 << d)) : sinpif(r[1] * float(1 << d));
    }
#pragma unroll
    for (int d = 0; d < 8; ++d) f[24 + d] = (MODE == 0) ? tri_sin(r[2] * float(1 << d)) : sinpif(r[2] * float(1 << d));
  } else {
#pragma unroll
    for (int d = 8; d < 12; ++d) f[d - 8] = (MODE == 0) ? tri_sin(r[2] * float(1 << d)) : sinpif(r[2] * float(1 << d));
    oneblob4<MODE>(r[3], f + 4);
    oneblob4<MODE>(r[4], f + 8);
    oneblob4<MODE>(r[5], f + 12);
    oneblob4<MODE>(r[6], f + 16);
    oneblob4<MODE>(-expm1f(-r[7]), f + 20);
#pragma unroll
    for (int j = 0; j < 6; ++j) f[24 + j] = r[8 + j];
    f[30] = pad;
    f[31] = pad;
  }
}

__device__ __forceinline__ void load_record(const float* rec, int64_t row, float* r) {
  const float4* p = reinterpret_cast<const float4*>(rec + row * kRecFloats);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 v = __ldg(p + q);
    r[4 * q + 0] = v.x;
    r[4 * q + 1] = v.y;
    r[4 * q + 2] = v.z;
    r[4 * q + 3] = v.w;
  }
}

// Byte offset of element (n, k) of a 16-bit K-major matrix with 128-byte rows
// in the 128-byte-swizzled layout.
__host__ __device__ __forceinline__ uint32_t sw128_offset(uint32_t n, uint32_t k) {
  return (n >> 3) * 1024u + (n & 7u) * 128u + ((((k >> 3) ^ n) & 7u) << 4) + (k & 7u) * 2u;
}

// Byte offset of element (row n, input k) of matrix l in the 16-bit weight
// image: matrices with more than 64 inputs are stored as blocks of 64
// inputs (each block rows x 128 B, 128-byte swizzled), block after block.
// For 64 inputs or fewer it is sw128_offset within the matrix.
__host__ __device__ __forceinline__ uint32_t img_offset(const ImageShape& img, int l, uint32_t n, uint32_t k) {
  return uint32_t(img.off[l]) + (k >> 6) * uint32_t(img.rows[l]) * 128u + sw128_offset(n, k & 63u);
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while its predecessor in the stream still runs;
// pdl_wait() blocks until the predecessor has completed and its writes are
// visible, pdl_launch_dependents() lets the successor start early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// b^t for integer t >= 0 by repeated squaring in FP32: exact for t = 1, about
// 2 log2(t) roundings otherwise (FP64 arithmetic is slow on this part).
__device__ __forceinline__ float pow_int(float b, long long t) {
  float r = 1.0f;
  while (t > 0) {
    if (t & 1) r *= b;
    b *= b;
    t >>= 1;
  }
  return r;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace nrc

// The C ABI's opaque cache handle is the library's cache state.
struct nrc_cache : nrc::Cache {};
