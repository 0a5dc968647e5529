// Allocation-free training step (nrc_train_step_noalloc).
//
// Some callers cannot allocate device memory at the point where they train:
// a renderer whose engine reserves and hands out every device allocation
// itself under a fixed budget, or a frame loop that must not take the
// device-wide synchronisation that cudaMalloc / cudaFree can imply.  This
// entry point runs the same tensor-core training step as nrc_train_step on
// state the caller owns (weights, Adam moments, step counter) and keeps its
// scratch -- the per-CTA weight-gradient partials, the 16-bit weight image
// and the error word -- in file-scope device arrays of fixed size, which
// every GPU that loads the library holds until the process exits.
#include <mutex>

#include "nrc_internal.cuh"

namespace nrc {

// Capacity of the static scratch.
constexpr int kNaPartials = 64;        // training CTAs (each loops over its share of 128-row tiles)
constexpr int kNaMaxMats = 6;          // width 64, at most 5 hidden layers
constexpr int kNaParams = 5 * 64 * 64 + 64 * 3;  // 20,672 weights of the width-64, 5-hidden-layer net
constexpr int kNaImageBytes = 5 * 64 * 64 * 2 + 16 * 64 * 2;  // 43,008 bytes
constexpr size_t kNaPartialFloats = size_t(kNaPartials) * ((size_t(kNaParams) + 1 + 3) & ~size_t(3));

static __device__ __align__(256) float g_na_partials[kNaPartialFloats];  // 5.3 MB
static __device__ __align__(1024) uint8_t g_na_image[kNaImageBytes];
static __device__ __align__(256) int g_na_err;

struct NaScratch {
  bool ready = false;
  float* partials = nullptr;
  uint8_t* image = nullptr;
  int* err = nullptr;
  int sm_count = 0;
};

constexpr int kNaMaxDevices = 64;
static NaScratch g_na_dev[kNaMaxDevices];
static std::mutex g_na_mutex;

// Device addresses of the static arrays on the current device.  In host
// code the arrays' names are host-side stand-ins, not device addresses, so
// the kernels get the addresses looked up here (once per device, with that
// device current).
static nrc_status na_scratch(int device, NaScratch** out) {
  if (device < 0 || device >= kNaMaxDevices) return set_error("device index %d out of range", device), NRC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  NaScratch& s = g_na_dev[device];
  if (!s.ready) {
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.partials), g_na_partials);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.image), g_na_image);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.err), g_na_err);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return cuda_status(e, "nrc_train_step_noalloc set-up");
    s.ready = true;
  }
  *out = &s;
  return NRC_OK;
}

}  // namespace nrc

using namespace nrc;

extern "C" nrc_status nrc_train_step_noalloc(const nrc_config* cfg, float* weights, float* adam_m, float* adam_v,
                                             int64_t* step_counter, const float* pool, const float* target,
                                             int64_t n_pool, int64_t batch, uint64_t frame_seed,
                                             int32_t step_in_frame, float* loss_out, int32_t* err_out,
                                             nrc_stream stream) {
  if (!cfg) return set_error("cfg is NULL"), NRC_ERR_INVALID_ARG;
  if (cfg->width == 64) {  // the general checks of nrc_create first (constants, enums)
    const nrc_status cs = check_cfg(cfg);
    if (cs != NRC_OK) return cs;
  }
  if (cfg->width != 64 || cfg->hidden_layers < 1 || cfg->hidden_layers > kNaMaxMats - 1)
    return set_error("nrc_train_step_noalloc: width must be 64 and hidden_layers 1..%d (static scratch holds %d "
                     "weights)", kNaMaxMats - 1, kNaParams),
           NRC_ERR_INVALID_ARG;
  if (cfg->dtype != NRC_FP16 && cfg->dtype != NRC_BF16)
    return set_error("nrc_train_step_noalloc: dtype must be NRC_FP16 or NRC_BF16"), NRC_ERR_UNSUPPORTED;
  if (cfg->enc_mode != NRC_ENC_CHEAP && cfg->enc_mode != NRC_ENC_EXACT)
    return set_error("unknown enc_mode %d", cfg->enc_mode), NRC_ERR_INVALID_ARG;
  if (cfg->loss_mode != NRC_LOSS_LUMINANCE && cfg->loss_mode != NRC_LOSS_PER_CHANNEL)
    return set_error("unknown loss_mode %d", cfg->loss_mode), NRC_ERR_INVALID_ARG;
  if (cfg->ema)
    return set_error("nrc_train_step_noalloc keeps no weight average (cfg->ema must be 0)"), NRC_ERR_UNSUPPORTED;
  if (cfg->refl_factor != 0 && cfg->refl_factor != 1) return set_error("refl_factor must be 0 or 1"), NRC_ERR_INVALID_ARG;
  if (cfg->optimizer != NRC_OPT_ADAM)
    return set_error("nrc_train_step_noalloc trains with Adam only"), NRC_ERR_UNSUPPORTED;
  if (batch < 0 || n_pool < 0 || step_in_frame < 0) return set_error("negative size or step"), NRC_ERR_INVALID_ARG;
  if (batch > 0) {
    if (batch > kMaxBatch)
      return set_error("nrc_train_step_noalloc: batch %lld above the maximum %d", (long long)batch, kMaxBatch),
             NRC_ERR_INVALID_ARG;
    if (n_pool >= (int64_t(1) << 31)) return set_error("n_pool must be below 2^31"), NRC_ERR_INVALID_ARG;
    if ((int64_t(step_in_frame) + 1) * batch > n_pool)
      return set_error("(step+1)*batch exceeds n_pool"), NRC_ERR_INVALID_ARG;
    if (!weights || !adam_m || !adam_v || !step_counter || !pool || !target)
      return set_error("nrc_train_step_noalloc: NULL state or input pointer"), NRC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(pool) & 15u) || (reinterpret_cast<uintptr_t>(weights) & 15u))
      return set_error("pool and weights must be 16-byte aligned"), NRC_ERR_INVALID_ARG;
  }

  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_status(e, "nrc_train_step_noalloc");
  NaScratch* s = nullptr;
  nrc_status st = na_scratch(device, &s);
  if (st != NRC_OK) return st;
  if (batch == 0) return NRC_OK;  // the set-up alone (the first call on a device)

  // A view of the caller's state plus the static scratch, shaped like a cache
  // so that the ordinary launchers run unchanged; nothing in it is allocated.
  Cache c;
  c.cfg = *cfg;
  c.cfg.path = NRC_PATH_FUSED;
  make_net_shape(c.cfg, &c.net);
  make_image_shape(c.net, &c.img);
  c.w = weights;
  c.m = adam_m;
  c.v = adam_v;
  c.t = reinterpret_cast<long long*>(step_counter);
  c.wimg = s->image;
  c.partials = s->partials;
  c.max_partials = kNaPartials;
  c.err = s->err;
  c.sm_count = s->sm_count < kNaPartials ? s->sm_count : kNaPartials;  // caps the grid at the partial count
  c.device = device;

  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  uint64_t a, cc;
  lcg_params(n_pool, frame_seed, &a, &cc);
  e = cudaMemsetAsync(s->err, 0, sizeof(int), cs);
  if (e == cudaSuccess) e = launch_build_image(&c, cs);
  int n_partials = 0;
  float grad_scale = 1.0f;
  if (e == cudaSuccess) e = launch_train_tc(&c, pool, target, n_pool, batch, a, cc, step_in_frame, &n_partials,
                                            &grad_scale, cs);
  if (e == cudaSuccess) e = launch_adam(&c, n_partials, grad_scale, loss_out, cs);
  if (e == cudaSuccess && err_out) e = cudaMemcpyAsync(err_out, s->err, sizeof(int), cudaMemcpyDeviceToDevice, cs);
  return cuda_status(e, "nrc_train_step_noalloc");
}
