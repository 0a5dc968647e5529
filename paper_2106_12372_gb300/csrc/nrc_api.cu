// C ABI of the neural radiance cache library (include/nrc.h): argument
// checking, cache state ownership, and the launch sequences of each call.
#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "nrc_internal.cuh"

namespace nrc {

int g_alloc_skip = 0, g_alloc_fail = 0;
static std::mutex g_alloc_mu;

cudaError_t dev_alloc_bytes(void** p, size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_alloc_skip > 0) {
      --g_alloc_skip;
    } else if (g_alloc_fail > 0) {
      --g_alloc_fail;
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  return cudaMalloc(p, bytes);
}


static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

nrc_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return NRC_OK;
  set_error("%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return NRC_ERR_OOM;
  return NRC_ERR_CUDA;
}

void make_net_shape(const nrc_config& cfg, NetShape* s) {
  std::memset(s, 0, sizeof(*s));
  s->n_mats = cfg.hidden_layers + 1;
  s->dims[0] = kEncDims;
  for (int l = 1; l <= cfg.hidden_layers; ++l) s->dims[l] = cfg.width;
  s->dims[s->n_mats] = kOutDims;
  int off = 0;
  for (int l = 0; l < s->n_mats; ++l) {
    s->w_off[l] = off;
    off += s->dims[l] * s->dims[l + 1];
  }
  s->w_off[s->n_mats] = off;
  s->n_params = off;
}

void make_image_shape(const NetShape& s, ImageShape* img) {
  std::memset(img, 0, sizeof(*img));
  int off = 0;
  for (int l = 0; l < s.n_mats; ++l) {
    img->off[l] = off;
    img->rows[l] = (s.dims[l + 1] + 15) / 16 * 16;
    off += img->rows[l] * s.dims[l] * 2;
  }
  img->off[s.n_mats] = off;
}

static uint64_t splitmix64(uint64_t& state) {
  // Steele, Lea & Flood 2014.
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void lcg_params(int64_t n_pool, uint64_t frame_seed, uint64_t* a_out, uint64_t* c_out) {
  lcg_shuffle(n_pool, frame_seed, a_out, c_out);
}

// Xavier-uniform initial weights from SplitMix64 (stream 2 of the seed):
// layer after layer, row-major [out][in], U(-a, a), a = sqrt(6/(fan_in+fan_out)).
static void xavier_init(const NetShape& s, uint64_t seed, std::vector<float>& w) {
  w.resize(size_t(s.n_params));
  uint64_t state = seed * 0x100000001B3ull + 2ull;
  for (int l = 0; l < s.n_mats; ++l) {
    const double lim = std::sqrt(6.0 / double(s.dims[l] + s.dims[l + 1]));
    for (int p = s.w_off[l]; p < s.w_off[l + 1]; ++p) {
      const double u = double(splitmix64(state) >> 11) * (1.0 / 9007199254740992.0);
      w[size_t(p)] = float((2.0 * u - 1.0) * lim);
    }
  }
}

cudaError_t ensure_partials(Cache* c, int count) {
  if (count <= c->max_partials) return cudaSuccess;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  cudaFree(c->partials);
  c->partials = nullptr;
  c->max_partials = 0;
  e = dev_alloc(&c->partials, size_t(count) * partial_stride(c->net.n_params) * 4);
  if (e == cudaSuccess) c->max_partials = count;
  return e;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

nrc_status check_cfg(const nrc_config* cfg) {
  if (!cfg) return set_error("cfg is NULL"), NRC_ERR_INVALID_ARG;
  if (cfg->hidden_layers < 1 || cfg->hidden_layers > kMaxMats - 1)
    return set_error("hidden_layers must be in [1, %d]", kMaxMats - 1), NRC_ERR_INVALID_ARG;
  if (cfg->width != 64 && cfg->width != 128) return set_error("width %d unsupported (64 or 128)", cfg->width), NRC_ERR_UNSUPPORTED;
  if (cfg->width != 64) {
    // width 128: FP32 on the plain path, or FP16/BF16 queries on the tensor cores (trained on the plain FP32
    // kernels); Adam only, and at most 7 hidden layers on the tensor cores (the 16-bit weight image stays in
    // shared memory)
    const bool plain32 = cfg->dtype == NRC_FP32 && cfg->path == NRC_PATH_PLAIN;
    const bool tc16 = (cfg->dtype == NRC_FP16 || cfg->dtype == NRC_BF16) && cfg->hidden_layers <= 7 && !cfg->ema;
    if (cfg->optimizer != NRC_OPT_ADAM || !(plain32 || tc16))
      return set_error("width 128: dtype NRC_FP32 on the plain path, or NRC_FP16 / NRC_BF16 with at most 7 hidden "
                       "layers and no weight average; Adam only"),
             NRC_ERR_UNSUPPORTED;
  }
  if (cfg->dtype < NRC_FP32 || cfg->dtype > NRC_FP8) return set_error("unknown dtype %d", cfg->dtype), NRC_ERR_INVALID_ARG;
  if (cfg->enc_mode != NRC_ENC_CHEAP && cfg->enc_mode != NRC_ENC_EXACT)
    return set_error("unknown enc_mode %d", cfg->enc_mode), NRC_ERR_INVALID_ARG;
  if (cfg->loss_mode != NRC_LOSS_LUMINANCE && cfg->loss_mode != NRC_LOSS_PER_CHANNEL)
    return set_error("unknown loss_mode %d", cfg->loss_mode), NRC_ERR_INVALID_ARG;
  if (cfg->path != NRC_PATH_FUSED && cfg->path != NRC_PATH_PLAIN)
    return set_error("unknown path %d", cfg->path), NRC_ERR_INVALID_ARG;
  if (!(cfg->lr > 0.0f) || !(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f) || !(cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f) ||
      !(cfg->adam_eps >= 0.0f) || !(cfg->loss_eps > 0.0f) || !std::isfinite(cfg->pad_value))
    return set_error("invalid optimiser or loss constants"), NRC_ERR_INVALID_ARG;
  if ((cfg->ema != 0 && cfg->ema != 1) || (cfg->ema && !(cfg->ema_alpha >= 0.0f && cfg->ema_alpha < 1.0f)))
    return set_error("ema must be 0 or 1 and ema_alpha in [0, 1)"), NRC_ERR_INVALID_ARG;
  if (cfg->refl_factor != 0 && cfg->refl_factor != 1) return set_error("refl_factor must be 0 or 1"), NRC_ERR_INVALID_ARG;
  if ((cfg->optimizer != NRC_OPT_ADAM && cfg->optimizer != NRC_OPT_SHAMPOO) || cfg->shampoo_interval < 1 ||
      !(cfg->shampoo_eps >= 0.0f))
    return set_error("optimizer must be NRC_OPT_ADAM or NRC_OPT_SHAMPOO, shampoo_interval >= 1, shampoo_eps >= 0"),
           NRC_ERR_INVALID_ARG;
  return NRC_OK;
}

static nrc_status check_pool(const nrc_cache* c, const float* pool, const float* target, int64_t n_pool,
                             int64_t batch, int32_t step) {
  if (!c) return set_error("cache is NULL"), NRC_ERR_INVALID_ARG;
  if (batch < 0 || n_pool < 0 || step < 0) return set_error("negative size or step"), NRC_ERR_INVALID_ARG;
  if (batch == 0) return NRC_OK;
  if (batch > kMaxBatch) return set_error("batch %lld above %d", (long long)batch, kMaxBatch), NRC_ERR_INVALID_ARG;
  if (n_pool >= (int64_t(1) << 31)) return set_error("n_pool must be below 2^31"), NRC_ERR_INVALID_ARG;
  if ((int64_t(step) + 1) * batch > n_pool)
    return set_error("(step+1)*batch = %lld exceeds n_pool = %lld", (long long)((int64_t(step) + 1) * batch),
                     (long long)n_pool),
           NRC_ERR_INVALID_ARG;
  if (!pool || !target) return set_error("pool or target is NULL"), NRC_ERR_INVALID_ARG;
  if (!aligned16(pool)) return set_error("pool must be 16-byte aligned"), NRC_ERR_INVALID_ARG;
  return NRC_OK;
}

// Shampoo statistics start at zero with the step counter (nrc_create, nrc_set_state).
static cudaError_t reset_shampoo(Cache* c, cudaStream_t st) {
  if (c->cfg.optimizer != NRC_OPT_SHAMPOO) return cudaSuccess;
  const size_t sh_bytes = size_t(2 * c->net.n_mats) * kShampooStatFloats * 4;
  cudaError_t e = cudaMemsetAsync(c->sh_stats, 0, sh_bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->sh_roots, 0, sh_bytes, st);
  return e;
}
}  // namespace nrc


using namespace nrc;

extern "C" {

const char* nrc_last_error_string(void) { return g_err; }

void nrc_default_config(nrc_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->width = 64;
  cfg->hidden_layers = 5;
  cfg->dtype = NRC_FP16;
  cfg->enc_mode = NRC_ENC_CHEAP;
  cfg->loss_mode = NRC_LOSS_LUMINANCE;
  cfg->path = NRC_PATH_FUSED;
  cfg->pad_value = 1.0f;
  cfg->lr = 1e-2f;
  cfg->beta1 = 0.9f;
  cfg->beta2 = 0.99f;
  cfg->adam_eps = 1e-8f;
  cfg->loss_eps = 0.01f;
  cfg->seed = 2106;
  cfg->ema = 0;
  cfg->ema_alpha = 0.99f;
  cfg->refl_factor = 0;
  cfg->optimizer = NRC_OPT_ADAM;
  cfg->shampoo_interval = 4;
  cfg->shampoo_eps = 1e-4f;
}

namespace nrc {
// Restarts the weight average at the current weights (cache creation,
// nrc_set_state): EMA_0 is never read by Eq. 2 (eta_0 = 0), but queries made
// before the first training step see it.
static cudaError_t reset_ema(Cache* c, cudaStream_t st) {
  if (!c->cfg.ema) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(c->ema, c->w, size_t(c->net.n_params) * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && c->cfg.dtype != NRC_FP32)
    e = cudaMemcpyAsync(c->wimg_ema, c->wimg, size_t(c->img.off[c->net.n_mats]), cudaMemcpyDeviceToDevice, st);
  return e;
}
}  // namespace nrc

int64_t nrc_param_count(const nrc_cache* c) { return c ? c->net.n_params : 0; }

int64_t nrc_launch_count(const nrc_cache* c) { return c ? c->launches : 0; }

static void free_cache(nrc_cache* c) {
  cudaFree(c->w);
  cudaFree(c->m);
  cudaFree(c->v);
  cudaFree(c->t);
  cudaFree(c->wimg);
  cudaFree(c->ema);
  cudaFree(c->wimg_ema);
  cudaFree(c->wimg8);
  cudaFree(c->sh_g);
  cudaFree(c->sh_stats);
  cudaFree(c->sh_roots);
  cudaFree(c->sh_anorm);
  cudaFree(c->partials);
  cudaFree(c->err);
  cudaFree(c->plain_buf);
  cudaFree(c->stage);
  cudaFree(c->wimg_snap);
  cudaFree(c->wimg_work);
  cudaFree(c->wimg_ema_work);
  cudaFree(c->frame_sync);
  for (cudaEvent_t e : c->ev_pipe)
    if (e) cudaEventDestroy(e);
  if (c->s_h2d) cudaStreamDestroy(c->s_h2d);
  if (c->s_query) cudaStreamDestroy(c->s_query);
  if (c->s_d2h) cudaStreamDestroy(c->s_d2h);
  delete c;
}

nrc_status nrc_create(const nrc_config* cfg, nrc_stream stream, nrc_cache** out) {
  if (!out) return set_error("out is NULL"), NRC_ERR_INVALID_ARG;
  *out = nullptr;
  nrc_status s = check_cfg(cfg);
  if (s != NRC_OK) return s;
  nrc_cache* c = new (std::nothrow) nrc_cache();
  if (!c) return set_error("host allocation failed"), NRC_ERR_OOM;
  c->cfg = *cfg;
  make_net_shape(*cfg, &c->net);
  make_image_shape(c->net, &c->img);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess && cfg->dtype != NRC_FP32) {
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, c->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, c->device);
    if (major != 10) {
      delete c;
      return set_error("tensor-core path needs an sm_10x device (found sm_%d%d)", major, minor), NRC_ERR_UNSUPPORTED;
    }
  }
  const size_t np = size_t(c->net.n_params);
  c->max_partials = 0;
  if (e == cudaSuccess) e = dev_alloc(&c->w, np * 4);
  if (e == cudaSuccess) e = dev_alloc(&c->m, np * 4);
  if (e == cudaSuccess) e = dev_alloc(&c->v, np * 4);
  if (e == cudaSuccess) e = dev_alloc(&c->t, sizeof(long long));
  if (e == cudaSuccess) e = dev_alloc(&c->wimg, size_t(c->img.off[c->net.n_mats]) + 1024);
  if (e == cudaSuccess) e = dev_alloc(&c->err, sizeof(int));
  if (e == cudaSuccess && cfg->ema) e = dev_alloc(&c->ema, np * 4);
  if (e == cudaSuccess && cfg->dtype == NRC_FP8)
    e = dev_alloc(&c->wimg8, size_t(img8_offset(c->net, c->net.n_mats)) + kImg8ScaleBytes);
  if (e == cudaSuccess && cfg->ema) e = dev_alloc(&c->wimg_ema, size_t(c->img.off[c->net.n_mats]) + 1024);
  const size_t sh_bytes = size_t(2 * c->net.n_mats) * kShampooStatFloats * 4;
  if (e == cudaSuccess && cfg->optimizer == NRC_OPT_SHAMPOO) e = dev_alloc(&c->sh_g, np * 4);
  if (e == cudaSuccess && cfg->optimizer == NRC_OPT_SHAMPOO) e = dev_alloc(&c->sh_stats, sh_bytes);
  if (e == cudaSuccess && cfg->optimizer == NRC_OPT_SHAMPOO) e = dev_alloc(&c->sh_roots, sh_bytes);
  if (e == cudaSuccess && cfg->optimizer == NRC_OPT_SHAMPOO) e = dev_alloc(&c->sh_anorm, (np + 31) / 32 * 4);
  if (e != cudaSuccess) {
    nrc_status st = cuda_status(e, "nrc_create allocation");
    free_cache(c);
    return st;
  }
  std::vector<float> w0;
  xavier_init(c->net, cfg->seed, w0);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  e = cudaMemcpyAsync(c->w, w0.data(), np * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->m, 0, np * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->v, 0, np * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->t, 0, sizeof(long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->wimg, 0, size_t(c->img.off[c->net.n_mats]) + 1024, st);
  if (e == cudaSuccess) e = launch_build_image(c, st);
  if (e == cudaSuccess) e = reset_ema(c, st);
  if (e == cudaSuccess) e = reset_shampoo(c, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // w0 is a host temporary
  if (e != cudaSuccess) {
    nrc_status s2 = cuda_status(e, "nrc_create upload");
    free_cache(c);
    return s2;
  }
  c->launches += cfg->dtype != NRC_FP32 ? 1 : 0;
  *out = c;
  return NRC_OK;
}

nrc_status nrc_destroy(nrc_cache* c) {
  if (!c) return NRC_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_cache(c);
  return cuda_status(e, "nrc_destroy");
}

nrc_status nrc_set_path(nrc_cache* c, int32_t path) {
  if (!c) return set_error("cache is NULL"), NRC_ERR_INVALID_ARG;
  if (path != NRC_PATH_FUSED && path != NRC_PATH_PLAIN) return set_error("unknown path %d", path), NRC_ERR_INVALID_ARG;
  if (path == NRC_PATH_FUSED && c->cfg.width != 64 && c->cfg.dtype != NRC_FP16 && c->cfg.dtype != NRC_BF16)
    return set_error("the fused kernels take width 64, or width 128 in FP16 / BF16"), NRC_ERR_UNSUPPORTED;
  c->cfg.path = path;
  return NRC_OK;
}

nrc_status nrc_encode(nrc_cache* c, const float* rec, int64_t n, void* out, int32_t out_dtype, nrc_stream stream) {
  if (!c) return set_error("cache is NULL"), NRC_ERR_INVALID_ARG;
  if (n < 0) return set_error("n < 0"), NRC_ERR_INVALID_ARG;
  if (out_dtype < NRC_FP32 || out_dtype > NRC_BF16) return set_error("unknown out_dtype"), NRC_ERR_INVALID_ARG;
  if (n == 0) return NRC_OK;
  if (!rec || !out) return set_error("NULL pointer"), NRC_ERR_INVALID_ARG;
  if (!aligned16(rec) || !aligned16(out)) return set_error("pointers must be 16-byte aligned"), NRC_ERR_INVALID_ARG;
  if (n > (int64_t(1) << 40)) return set_error("n too large"), NRC_ERR_INVALID_ARG;
  c->launches += 1;
  return cuda_status(launch_encode(rec, n, out, out_dtype, c->cfg.enc_mode, c->cfg.pad_value,
                                   reinterpret_cast<cudaStream_t>(stream)),
                     "nrc_encode");
}

static nrc_status infer_impl(nrc_cache* c, const float* rec, int64_t n, float* rgb, cudaStream_t st) {
  cudaError_t e;
  if (c->cfg.path == NRC_PATH_PLAIN) {
    e = plain_infer(c, rec, n, rgb, st);
  } else if (c->cfg.width == 128) {
    e = launch_infer_tc128(c, rec, n, rgb, st);
    c->launches += 1;
  } else if (c->cfg.dtype == NRC_FP8) {
    e = cudaSuccess;
    if (c->wimg8_dirty) {
      e = launch_build_image_fp8(c, st);
      c->wimg8_dirty = false;
      c->launches += 1;
    }
    if (e == cudaSuccess) e = launch_infer_fp8(c, rec, n, rgb, st);
    c->launches += 1;
  } else if (c->cfg.dtype == NRC_FP32) {
    e = launch_infer_simt(c, rec, n, rgb, st);
    c->launches += 1;
  } else {
    e = launch_infer_tc(c, rec, n, rgb, st);
    c->launches += 1;
  }
  return cuda_status(e, "nrc_infer");
}

nrc_status nrc_infer(nrc_cache* c, const float* rec, int64_t n, float* rgb, nrc_stream stream) {
  if (!c) return set_error("cache is NULL"), NRC_ERR_INVALID_ARG;
  if (n < 0) return set_error("n < 0"), NRC_ERR_INVALID_ARG;
  if (n == 0) return NRC_OK;
  if (!rec || !rgb) return set_error("NULL pointer"), NRC_ERR_INVALID_ARG;
  if (!aligned16(rec) || !aligned16(rgb)) return set_error("pointers must be 16-byte aligned"), NRC_ERR_INVALID_ARG;
  if (n > (int64_t(1) << 40)) return set_error("n too large"), NRC_ERR_INVALID_ARG;
  return infer_impl(c, rec, n, rgb, reinterpret_cast<cudaStream_t>(stream));
}

nrc_status nrc_gather(const float* pool, const float* target, int64_t n_pool, int64_t batch, uint64_t frame_seed,
                      int32_t step, float* rec_out, float* tgt_out, nrc_stream stream) {
  if (batch < 0 || n_pool < 0 || step < 0) return set_error("negative size or step"), NRC_ERR_INVALID_ARG;
  if (batch == 0) return NRC_OK;
  if (n_pool >= (int64_t(1) << 31)) return set_error("n_pool must be below 2^31"), NRC_ERR_INVALID_ARG;
  if ((int64_t(step) + 1) * batch > n_pool) return set_error("(step+1)*batch exceeds n_pool"), NRC_ERR_INVALID_ARG;
  if (!pool || !rec_out || (tgt_out && !target)) return set_error("NULL pointer"), NRC_ERR_INVALID_ARG;
  if (!aligned16(pool) || !aligned16(rec_out)) return set_error("pointers must be 16-byte aligned"), NRC_ERR_INVALID_ARG;
  uint64_t a, cc;
  lcg_params(n_pool, frame_seed, &a, &cc);
  return cuda_status(launch_gather(pool, target, n_pool, batch, a, cc, step, rec_out, tgt_out,
                                   reinterpret_cast<cudaStream_t>(stream)),
                     "nrc_gather");
}

static nrc_status train_impl(nrc_cache* c, const float* pool, const float* target, int64_t n_pool, int64_t batch,
                             uint64_t frame_seed, int32_t step, float* loss_out, cudaStream_t st) {
  c->wimg8_dirty = true;
  uint64_t a, cc;
  lcg_params(n_pool, frame_seed, &a, &cc);
  cudaError_t e;
  if (c->cfg.path == NRC_PATH_PLAIN || c->cfg.width != 64) {
    // (width 128 trains on the plain FP32 kernels; their Adam writes the 16-bit image the queries read)
    e = plain_train(c, pool, target, n_pool, batch, a, cc, step, loss_out, st);
    return cuda_status(e, "nrc_train_step (plain)");
  }
  int n_partials = 0;
  float grad_scale = 1.0f;
  if (c->cfg.dtype == NRC_FP32)
    e = launch_train_simt(c, pool, target, n_pool, batch, a, cc, step, &n_partials, st);
  else
    e = launch_train_tc(c, pool, target, n_pool, batch, a, cc, step, &n_partials, &grad_scale, st);
  if (e != cudaSuccess) return cuda_status(e, "nrc_train_step (gradient)");
  if (c->cfg.optimizer == NRC_OPT_SHAMPOO) {
    e = launch_shampoo(c, n_partials, grad_scale, loss_out, st);
    c->launches += 4;
    return cuda_status(e, "nrc_train_step (shampoo)");
  }
  e = launch_adam(c, n_partials, grad_scale, loss_out, st);
  c->launches += 2;
  return cuda_status(e, "nrc_train_step (adam)");
}

nrc_status nrc_train_step(nrc_cache* c, const float* pool, const float* target, int64_t n_pool, int64_t batch,
                          uint64_t frame_seed, int32_t step, float* loss_out, nrc_stream stream) {
  nrc_status s = check_pool(c, pool, target, n_pool, batch, step);
  if (s != NRC_OK || batch == 0) return s;
  return train_impl(c, pool, target, n_pool, batch, frame_seed, step, loss_out, reinterpret_cast<cudaStream_t>(stream));
}

namespace nrc {
// The fused frame kernel takes the 16-bit tensor-core path with Adam at
// width 64 and up to 5 hidden layers.  A frame without queries runs as
// separate launches unless the training CTAs are set: alone, the training
// is faster there (the Adam kernel spreads the reduction over every SM and
// programmatic dependent launch overlaps the next step's gather).
static bool fused_frame_ok(const Cache* c, int64_t n_q, int64_t batch, int32_t n_steps) {
  const nrc_config& k = c->cfg;
  return c->frame_ctas >= 0 && (n_q > 0 || c->frame_ctas > 0) && k.path == NRC_PATH_FUSED &&
         (k.dtype == NRC_FP16 || k.dtype == NRC_BF16) &&
         k.optimizer == NRC_OPT_ADAM && k.width == 64 && c->net.n_mats <= 6 && n_steps > 0 && n_steps <= 64 && batch > 0 &&
         (n_q + kTile - 1) / kTile < (int64_t(1) << 31);
}
}  // namespace nrc

nrc_status nrc_set_frame_ctas(nrc_cache* c, int32_t train_ctas) {
  if (!c) return set_error("cache is NULL"), NRC_ERR_INVALID_ARG;
  if (train_ctas < -1 || train_ctas > c->sm_count)
    return set_error("train_ctas must be -1, 0 or 1..%d", c->sm_count), NRC_ERR_INVALID_ARG;
  c->frame_ctas = train_ctas;
  return NRC_OK;
}

int32_t nrc_frame_ctas(const nrc_cache* c, int64_t n_queries, int64_t batch, int32_t n_steps) {
  if (!c || n_queries < 0 || batch <= 0 || n_steps <= 0 || !fused_frame_ok(c, n_queries, batch, n_steps)) return -1;
  const int64_t tiles = (batch + kTile - 1) / kTile;
  const int t = c->frame_ctas > 0 ? c->frame_ctas : frame_split(c, n_queries, batch, n_steps);
  return int32_t(std::min<int64_t>(t, tiles));
}

namespace nrc {
static nrc_status frame_impl(nrc_cache* c, const float* queries, int64_t n_q, float* rgb, const float* pool,
                             const float* target, int64_t n_pool, int64_t batch, int32_t n_steps, uint64_t frame_seed,
                             float* loss_out, nrc_stream stream, bool allow_fused) {
  if (!c) return set_error("cache is NULL"), NRC_ERR_INVALID_ARG;
  if (n_q < 0 || n_steps < 0) return set_error("negative size"), NRC_ERR_INVALID_ARG;
  if (n_q > 0 && (!queries || !rgb || !aligned16(queries) || !aligned16(rgb)))
    return set_error("queries/rgb NULL or misaligned"), NRC_ERR_INVALID_ARG;
  if (n_steps > 0 && batch > 0) {
    nrc_status s = check_pool(c, pool, target, n_pool, batch, n_steps - 1);
    if (s != NRC_OK) return s;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (allow_fused && fused_frame_ok(c, n_q, batch, n_steps)) {
    // one persistent launch: the queries and the training steps side by side
    uint64_t a, cc;
    lcg_params(n_pool, frame_seed, &a, &cc);
    const int ctas = c->frame_ctas > 0 ? c->frame_ctas : frame_split(c, n_q, batch, n_steps);
    c->wimg8_dirty = true;
    c->launches += 1;
    return cuda_status(launch_frame_tc(c, queries, n_q, rgb, pool, target, n_pool, batch, n_steps, a, cc, loss_out,
                                       ctas, st),
                       "nrc_frame (fused)");
  }
  if (n_q > 0) {
    nrc_status s = infer_impl(c, queries, n_q, rgb, st);
    if (s != NRC_OK) return s;
  }
  if (batch > 0) {
    for (int k = 0; k < n_steps; ++k) {
      nrc_status s = train_impl(c, pool, target, n_pool, batch, frame_seed, k, loss_out ? loss_out + k : nullptr, st);
      if (s != NRC_OK) return s;
    }
  }
  return NRC_OK;
}
}  // namespace nrc

nrc_status nrc_frame(nrc_cache* c, const float* queries, int64_t n_q, float* rgb, const float* pool,
                     const float* target, int64_t n_pool, int64_t batch, int32_t n_steps, uint64_t frame_seed,
                     float* loss_out, nrc_stream stream) {
  return frame_impl(c, queries, n_q, rgb, pool, target, n_pool, batch, n_steps, frame_seed, loss_out, stream, true);
}

namespace nrc {
// nrc_frame_host for the tensor-core path, pipelined: the queries go up in
// chunks on s_h2d, each chunk is answered on s_query as soon as it has landed
// and comes back on s_d2h, while the frame's training steps run on the
// caller's stream against the pool (uploaded first).  The queries read a
// snapshot of the starting weight image, so that they see the weights from
// before the frame's training, as the sequential frame does.
constexpr int kPipeChunks = 8;
static nrc_status frame_host_pipelined(nrc_cache* c, const float* queries, int64_t n_q, float* rgb, const float* pool,
                                       const float* target, int64_t n_pool, int64_t batch, int32_t n_steps,
                                       uint64_t frame_seed, float* loss_out, float* dq, float* dr, float* dp, float* dt,
                                       float* dl, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (!c->wimg_snap) {  // set-up, resumable after a failure: each resource is made once
    if (!c->s_h2d) e = cudaStreamCreateWithFlags(&c->s_h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess && !c->s_query) e = cudaStreamCreateWithFlags(&c->s_query, cudaStreamNonBlocking);
    if (e == cudaSuccess && !c->s_d2h) e = cudaStreamCreateWithFlags(&c->s_d2h, cudaStreamNonBlocking);
    for (int i = 0; i < 20 && e == cudaSuccess; ++i)
      if (!c->ev_pipe[i]) e = cudaEventCreateWithFlags(&c->ev_pipe[i], cudaEventDisableTiming);
    const size_t img_bytes = size_t(c->img.off[c->net.n_mats]) + 1024;
    if (e == cudaSuccess) e = dev_alloc(&c->wimg_snap, img_bytes);
    if (e != cudaSuccess) return cuda_status(e, "nrc_frame_host pipeline set-up");
  }
  cudaEvent_t ev_start = c->ev_pipe[0], ev_snap = c->ev_pipe[1], ev_pool = c->ev_pipe[2], ev_train = c->ev_pipe[3];
  cudaEvent_t* ev_h = c->ev_pipe + 4;
  cudaEvent_t* ev_q = c->ev_pipe + 12;
  // the caller's earlier work, then the weight snapshot (stream order on st)
  e = cudaEventRecord(ev_start, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->wimg_snap, query_image(c), size_t(c->img.off[c->net.n_mats]), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(ev_snap, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_h2d, ev_start, 0);
  if (e == cudaSuccess && n_pool > 0 && pool) e = cudaMemcpyAsync(dp, pool, size_t(n_pool) * 64, cudaMemcpyHostToDevice, c->s_h2d);
  if (e == cudaSuccess && n_pool > 0 && target)
    e = cudaMemcpyAsync(dt, target, size_t(n_pool) * 12, cudaMemcpyHostToDevice, c->s_h2d);
  if (e == cudaSuccess) e = cudaEventRecord(ev_pool, c->s_h2d);
  // training on the caller's stream once the pool is up
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_pool, 0);
  if (e != cudaSuccess) return cuda_status(e, "nrc_frame_host");
  if (n_steps > 0 && batch > 0) {
    // the training steps as separate launches: they share the GPU with the
    // query chunks on the other streams, where a cooperative grid would wait
    // for SMs
    nrc_status s = frame_impl(c, dq, 0, dr, dp, dt, n_pool, batch, n_steps, frame_seed, loss_out ? dl : nullptr,
                              reinterpret_cast<nrc_stream>(st), false);
    if (s != NRC_OK) return s;
  }
  e = cudaEventRecord(ev_train, st);
  // queries in chunks of whole 128-row tiles
  const int64_t tiles = (n_q + kTile - 1) / kTile;
  const int chunks = int(std::min<int64_t>(kPipeChunks, std::max<int64_t>(1, tiles / 512)));
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_query, ev_snap, 0);
  for (int k = 0; k < chunks && e == cudaSuccess; ++k) {
    const int64_t b = tiles * k / chunks * kTile, en = std::min<int64_t>(n_q, tiles * (k + 1) / chunks * kTile);
    if (en <= b) continue;
    cudaStream_t hs = c->s_h2d;
    e = cudaMemcpyAsync(dq + b * 16, queries + b * 16, size_t(en - b) * 64, cudaMemcpyHostToDevice, hs);
    if (e == cudaSuccess) e = cudaEventRecord(ev_h[k], hs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_query, ev_h[k], 0);
    if (e == cudaSuccess) e = launch_infer_tc(c, dq + b * 16, en - b, dr + b * 3, c->s_query, c->wimg_snap);
    c->launches += 1;
    if (e == cudaSuccess) e = cudaEventRecord(ev_q[k], c->s_query);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_d2h, ev_q[k], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rgb + b * 3, dr + b * 3, size_t(en - b) * 12, cudaMemcpyDeviceToHost, c->s_d2h);
  }
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_d2h, ev_train, 0);
  if (e == cudaSuccess && loss_out && n_steps > 0)
    e = cudaMemcpyAsync(loss_out, dl, size_t(n_steps) * 4, cudaMemcpyDeviceToHost, c->s_d2h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_d2h);
  return cuda_status(e, "nrc_frame_host");
}
}  // namespace nrc

nrc_status nrc_frame_host(nrc_cache* c, const float* queries, int64_t n_q, float* rgb, const float* pool,
                          const float* target, int64_t n_pool, int64_t batch, int32_t n_steps, uint64_t frame_seed,
                          float* loss_out, nrc_stream stream) {
  if (!c) return set_error("cache is NULL"), NRC_ERR_INVALID_ARG;
  if (n_q < 0 || n_pool < 0 || n_steps < 0 || batch < 0) return set_error("negative size"), NRC_ERR_INVALID_ARG;
  if ((n_q > 0 && (!queries || !rgb)) || (n_steps > 0 && batch > 0 && (!pool || !target)))
    return set_error("NULL pointer"), NRC_ERR_INVALID_ARG;
  auto up16 = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t bq = up16(size_t(n_q) * 64), br = up16(size_t(n_q) * 12), bp = up16(size_t(n_pool) * 64),
               bt = up16(size_t(n_pool) * 12), bl = up16(size_t(n_steps) * 4);
  const size_t need = bq + br + bp + bt + bl;
  if (need > c->stage_bytes) {
    cudaDeviceSynchronize();
    cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
    cudaError_t e = dev_alloc(&c->stage, need);
    if (e != cudaSuccess) return cuda_status(e, "nrc_frame_host staging");
    c->stage_bytes = need;
  }
  uint8_t* base = static_cast<uint8_t*>(c->stage);
  float* dq = reinterpret_cast<float*>(base);
  float* dr = reinterpret_cast<float*>(base + bq);
  float* dp = reinterpret_cast<float*>(base + bq + br);
  float* dt = reinterpret_cast<float*>(base + bq + br + bp);
  float* dl = reinterpret_cast<float*>(base + bq + br + bp + bt);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n_q > 0 && c->cfg.path == NRC_PATH_FUSED && c->cfg.width == 64 &&
      (c->cfg.dtype == NRC_FP16 || c->cfg.dtype == NRC_BF16))
    return frame_host_pipelined(c, queries, n_q, rgb, pool, target, n_pool, batch, n_steps, frame_seed, loss_out, dq, dr,
                                dp, dt, dl, st);
  cudaError_t e = cudaSuccess;
  if (n_q > 0) e = cudaMemcpyAsync(dq, queries, size_t(n_q) * 64, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n_pool > 0 && pool) e = cudaMemcpyAsync(dp, pool, size_t(n_pool) * 64, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n_pool > 0 && target)
    e = cudaMemcpyAsync(dt, target, size_t(n_pool) * 12, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "nrc_frame_host upload");
  nrc_status s = nrc_frame(c, dq, n_q, dr, dp, dt, n_pool, batch, n_steps, frame_seed, loss_out ? dl : nullptr, stream);
  if (s != NRC_OK) return s;
  if (n_q > 0) e = cudaMemcpyAsync(rgb, dr, size_t(n_q) * 12, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && loss_out && n_steps > 0)
    e = cudaMemcpyAsync(loss_out, dl, size_t(n_steps) * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_status(e, "nrc_frame_host download");
}

nrc_status nrc_get_state(nrc_cache* c, float* w, float* m, float* v, int64_t* step, nrc_stream stream) {
  if (!c) return set_error("cache is NULL"), NRC_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t bytes = size_t(c->net.n_params) * 4;
  cudaError_t e = cudaSuccess;
  long long t = 0;
  if (w) e = cudaMemcpyAsync(w, c->w, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && m) e = cudaMemcpyAsync(m, c->m, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && v) e = cudaMemcpyAsync(v, c->v, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&t, c->t, sizeof(t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (step) *step = t;
  return cuda_status(e, "nrc_get_state");
}

nrc_status nrc_set_state(nrc_cache* c, const float* w, const float* m, const float* v, int64_t step,
                         nrc_stream stream) {
  if (!c || !w) return set_error("cache or weights NULL"), NRC_ERR_INVALID_ARG;
  if (step < 0) return set_error("step < 0"), NRC_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t bytes = size_t(c->net.n_params) * 4;
  long long t = step;
  cudaError_t e = cudaMemcpyAsync(c->w, w, bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = m ? cudaMemcpyAsync(c->m, m, bytes, cudaMemcpyHostToDevice, st) : cudaMemsetAsync(c->m, 0, bytes, st);
  if (e == cudaSuccess) e = v ? cudaMemcpyAsync(c->v, v, bytes, cudaMemcpyHostToDevice, st) : cudaMemsetAsync(c->v, 0, bytes, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->t, &t, sizeof(t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_build_image(c, st);
  if (e == cudaSuccess) e = reset_ema(c, st);
  if (e == cudaSuccess) e = reset_shampoo(c, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  c->wimg8_dirty = true;
  return cuda_status(e, "nrc_set_state");
}

nrc_status nrc_get_ema(nrc_cache* c, float* ema, nrc_stream stream) {
  if (!c || !ema) return set_error("cache or output NULL"), NRC_ERR_INVALID_ARG;
  if (!c->cfg.ema) return set_error("the cache keeps no weight average (cfg.ema = 0)"), NRC_ERR_UNSUPPORTED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(ema, c->ema, size_t(c->net.n_params) * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_status(e, "nrc_get_ema");
}

nrc_status nrc_set_ema(nrc_cache* c, const float* ema, nrc_stream stream) {
  if (!c || !ema) return set_error("cache or input NULL"), NRC_ERR_INVALID_ARG;
  if (!c->cfg.ema) return set_error("the cache keeps no weight average (cfg.ema = 0)"), NRC_ERR_UNSUPPORTED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(c->ema, ema, size_t(c->net.n_params) * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && c->cfg.dtype != NRC_FP32) e = launch_build_image_of(c, c->ema, c->wimg_ema, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  c->wimg8_dirty = true;
  return cuda_status(e, "nrc_set_ema");
}

void nrc_debug_fail_device_allocs(int32_t after, int32_t count) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc_skip = after > 0 ? after : 0;
  g_alloc_fail = count > 0 ? count : 0;
}

nrc_status nrc_debug_wait_timeout(nrc_cache* c, int32_t limit_us, nrc_stream stream) {
  if (!c) return set_error("cache is NULL"), NRC_ERR_INVALID_ARG;
  if (limit_us < 1 || limit_us > 2000000) return set_error("limit_us must be in [1, 2000000]"), NRC_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return cuda_status(launch_wait_probe(c->err, 1000ull * (unsigned long long)limit_us, st), "nrc_debug_wait_timeout");
}

nrc_status nrc_check_error(nrc_cache* c, nrc_stream stream) {
  if (!c) return set_error("cache is NULL"), NRC_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int h = 0;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_status(e, "nrc_check_error");
  // a frame launch that gave up may have left its counters part-way
  if (h != 0 && c->frame_sync) e = cudaMemset(c->frame_sync, 0, 64);
  if (e != cudaSuccess) return cuda_status(e, "nrc_check_error");
  if (h & kErrBounds) return set_error("a device bounds check failed (NRC_DEBUG build; the access was skipped)"), NRC_ERR_BOUNDS;
  if (h & kErrTimeout) return set_error("a bounded device wait timed out"), NRC_ERR_TIMEOUT;
  return NRC_OK;
}

}  // extern "C"
