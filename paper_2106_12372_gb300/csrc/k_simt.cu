// FP32 SIMT kernels: record gather, standalone encoding, fused FP32 inference
// and training (the parity path), fused weight-gradient reduction + Adam, and
// the 16-bit weight image builder.
#include "nrc_internal.cuh"

namespace nrc {

// ------------------------------------------------------------------ gather
// Sec. 3.5: batch `step` takes pool[perm(step*batch + j)], perm(i) = (a*i + c) mod n_pool.
__global__ void k_gather(const float4* __restrict__ pool, const float* __restrict__ target, int64_t n_pool,
                         int64_t batch, uint64_t a, uint64_t c, int step, float4* __restrict__ rec_out,
                         float* __restrict__ tgt_out) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= batch) return;
  const uint64_t i = uint64_t(step) * uint64_t(batch) + uint64_t(j);
  const int64_t src = int64_t((a * i + c) % uint64_t(n_pool));
#pragma unroll
  for (int q = 0; q < 4; ++q) rec_out[j * 4 + q] = __ldg(pool + src * 4 + q);
  if (tgt_out) {
#pragma unroll
    for (int q = 0; q < 3; ++q) tgt_out[j * 3 + q] = __ldg(target + src * 3 + q);
  }
}

cudaError_t launch_gather(const float* pool, const float* target, int64_t n_pool, int64_t batch, uint64_t a,
                          uint64_t c, int step, float* rec_out, float* tgt_out, cudaStream_t st) {
  const int threads = 256;
  const int64_t blocks = (batch + threads - 1) / threads;
  k_gather<<<unsigned(blocks), threads, 0, st>>>(reinterpret_cast<const float4*>(pool), target, n_pool, batch, a, c,
                                                 step, reinterpret_cast<float4*>(rec_out), tgt_out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ encode
template <int MODE, typename T>
__global__ void k_encode(const float* __restrict__ rec, int64_t n, T* __restrict__ out, float pad) {
  const int64_t row = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (row >= n) return;
  float r[kRecFloats], f[kEncDims];
  load_record(rec, row, r);
  encode_record<MODE>(r, pad, f);
  T* o = out + row * kEncDims;
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int q = 0; q < 16; ++q)
      reinterpret_cast<float4*>(o)[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        T lo, hi;
        if constexpr (std::is_same<T, __half>::value) {
          lo = __float2half_rn(f[8 * q + 2 * e]);
          hi = __float2half_rn(f[8 * q + 2 * e + 1]);
        } else {
          lo = __float2bfloat16_rn(f[8 * q + 2 * e]);
          hi = __float2bfloat16_rn(f[8 * q + 2 * e + 1]);
        }
        w[e] = uint32_t(*reinterpret_cast<uint16_t*>(&lo)) | (uint32_t(*reinterpret_cast<uint16_t*>(&hi)) << 16);
      }
      reinterpret_cast<uint4*>(o)[q] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

cudaError_t launch_encode(const float* rec, int64_t n, void* out, int out_dtype, int enc_mode, float pad,
                          cudaStream_t st) {
  const int threads = 128;
  const unsigned blocks = unsigned((n + threads - 1) / threads);
#define NRC_ENC(MODE)                                                                                 \
  if (out_dtype == NRC_FP32)                                                                          \
    k_encode<MODE, float><<<blocks, threads, 0, st>>>(rec, n, static_cast<float*>(out), pad);         \
  else if (out_dtype == NRC_FP16)                                                                     \
    k_encode<MODE, __half><<<blocks, threads, 0, st>>>(rec, n, static_cast<__half*>(out), pad);       \
  else                                                                                                \
    k_encode<MODE, __nv_bfloat16><<<blocks, threads, 0, st>>>(rec, n, static_cast<__nv_bfloat16*>(out), pad);
  if (enc_mode == NRC_ENC_CHEAP) {
    NRC_ENC(0)
  } else {
    NRC_ENC(1)
  }
#undef NRC_ENC
  return cudaGetLastError();
}

// ------------------------------------------------------ fused FP32 layers
// One thread owns one batch row; its activations live in registers; the
// weights of the whole network sit in shared memory (row-major [out][in]) and
// are read as float4 broadcasts.  Width 64 only.

// z[o] = sum_i W[o][i] h[i] for 64 outputs, with the ReLU of Sec. 5.
__device__ __forceinline__ void dense64_relu(const float* __restrict__ W, const float* h, float* z) {
#pragma unroll
  for (int o = 0; o < 64; ++o) {
    const float4* wr = reinterpret_cast<const float4*>(W + o * 64);
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float4 wv = wr[q];
      s = fmaf(wv.x, h[4 * q], s);
      s = fmaf(wv.y, h[4 * q + 1], s);
      s = fmaf(wv.z, h[4 * q + 2], s);
      s = fmaf(wv.w, h[4 * q + 3], s);
    }
    z[o] = fmaxf(s, 0.0f);
  }
}

// Linear RGB output layer (3 x 64).
__device__ __forceinline__ void dense_out(const float* __restrict__ W, const float* h, float* y) {
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    const float4* wr = reinterpret_cast<const float4*>(W + o * 64);
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float4 wv = wr[q];
      s = fmaf(wv.x, h[4 * q], s);
      s = fmaf(wv.y, h[4 * q + 1], s);
      s = fmaf(wv.z, h[4 * q + 2], s);
      s = fmaf(wv.w, h[4 * q + 3], s);
    }
    y[o] = s;
  }
}

__device__ __forceinline__ void stage_weights(float* sw, const float* __restrict__ w, int n_params) {
  const float4* src = reinterpret_cast<const float4*>(w);
  float4* dst = reinterpret_cast<float4*>(sw);
  for (int i = threadIdx.x; i < n_params / 4; i += blockDim.x) dst[i] = __ldg(src + i);
  for (int i = (n_params / 4) * 4 + threadIdx.x; i < n_params; i += blockDim.x) sw[i] = w[i];
}

template <int MODE>
__global__ void __launch_bounds__(128) k_infer_simt(const float* __restrict__ rec, int64_t n, float* __restrict__ rgb,
                                                    const float* __restrict__ w, const __grid_constant__ NetShape net, float pad,
                                                    int factor) {
  extern __shared__ float4 smem_f4[];
  float* sw = reinterpret_cast<float*>(smem_f4);
  stage_weights(sw, w, net.n_params);
  __syncthreads();
  for (int64_t row = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; row < n; row += int64_t(gridDim.x) * blockDim.x) {
    float r[kRecFloats], h[64], z[64];
    load_record(rec, row, r);
    encode_record<MODE>(r, pad, h);
    for (int l = 0; l < net.n_mats - 1; ++l) {
      dense64_relu(sw + net.w_off[l], h, z);
#pragma unroll
      for (int i = 0; i < 64; ++i) h[i] = z[i];
    }
    float y[3];
    dense_out(sw + net.w_off[net.n_mats - 1], h, y);
    if (factor) {  // reflectance factorisation (Sec. 5): times diffuse + specular albedo
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) y[ch] *= r[8 + ch] + r[11 + ch];
    }
    rgb[row * 3 + 0] = y[0];
    rgb[row * 3 + 1] = y[1];
    rgb[row * 3 + 2] = y[2];
  }
}

cudaError_t launch_infer_simt(Cache* c, const float* rec, int64_t n, float* rgb, cudaStream_t st) {
  const size_t smem = size_t(c->net.n_params) * 4;
  static std::atomic<int> attr_done[2];
  const int mode = c->cfg.enc_mode;
  cudaError_t e = mode == 0 ? ensure_smem(k_infer_simt<0>, int(smem), &attr_done[0])
                            : ensure_smem(k_infer_simt<1>, int(smem), &attr_done[1]);
  if (e != cudaSuccess) return e;
  const int64_t want = (n + 127) / 128;
  const int64_t cap = int64_t(c->sm_count) * 2;
  const unsigned blocks = unsigned(want < cap ? want : cap);
  if (mode == 0)
    k_infer_simt<0><<<blocks, 128, smem, st>>>(rec, n, rgb, query_weights(c), c->net, c->cfg.pad_value,
                                               c->cfg.refl_factor);
  else
    k_infer_simt<1><<<blocks, 128, smem, st>>>(rec, n, rgb, query_weights(c), c->net, c->cfg.pad_value,
                                               c->cfg.refl_factor);
  return cudaGetLastError();
}

// --------------------------------------------------- fused FP32 training
// One CTA of 64 threads per 64 gathered batch rows.  Shared memory holds the
// weights, every layer's input activations H_l (feature-major, row stride 65)
// and the current delta (feature-major, row stride 68 for float4 reads).
// Each CTA writes the weight gradient of its rows and its loss sum to its own
// partial; the Adam kernel sums the partials in a fixed order.
constexpr int kTrainRows = 64;
constexpr int kHStride = kTrainRows + 1;
constexpr int kDStride = kTrainRows + 4;

__device__ __forceinline__ void relative_l2(const float* y, const float* t, int loss_mode, float eps, float* g,
                                            float* loss_row) {
  // Eq. 5 with the luminance (or per-channel) normalisation; g = dL/dy up to
  // the 1/(3N) factor, which the caller applies.
  const float lum = 0.2126f * y[0] + 0.7152f * y[1] + 0.0722f * y[2];
  float acc = 0.0f;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    const float den = (loss_mode == NRC_LOSS_LUMINANCE ? lum * lum : y[ch] * y[ch]) + eps;
    const float inv = 1.0f / den;
    const float diff = y[ch] - t[ch];
    acc = fmaf(diff * diff, inv, acc);
    g[ch] = 2.0f * diff * inv;
  }
  *loss_row = acc;
}

template <int MODE>
__global__ void __launch_bounds__(kTrainRows) k_train_simt(const float* __restrict__ pool, const float* __restrict__ target,
                                                         int64_t n_pool, int64_t batch, uint64_t a, uint64_t c,
                                                         int step, const float* __restrict__ w, const __grid_constant__ NetShape net,
                                                         float pad, int loss_mode, float loss_eps, float inv3n,
                                                         float* __restrict__ partials, long long* __restrict__ t_ctr,
                                                         int factor) {
  extern __shared__ float4 smem_f4[];
  float* sw = reinterpret_cast<float*>(smem_f4);
  float* Hs = sw + ((net.n_params + 3) & ~3);       // [n_mats][64][kHStride]
  float* Ds = Hs + net.n_mats * 64 * kHStride;       // [64][kDStride]
  Ds = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(Ds) + 15) & ~uintptr_t(15));
  __shared__ float red[kTrainRows / 32];
  const int tid = threadIdx.x;
  if (blockIdx.x == 0 && tid == 0) *t_ctr += 1;  // Adam's t for the update that follows
  stage_weights(sw, w, net.n_params);

  const int64_t j = int64_t(blockIdx.x) * kTrainRows + tid;
  const bool valid = j < batch;
  float h[64], z[64];
  float tg[3] = {0.f, 0.f, 0.f};
  float fac[3] = {1.f, 1.f, 1.f};
  if (valid) {
    const uint64_t i = uint64_t(step) * uint64_t(batch) + uint64_t(j);
    const int64_t src = int64_t((a * i + c) % uint64_t(n_pool));
    float r[kRecFloats];
    load_record(pool, src, r);
    encode_record<MODE>(r, pad, h);
    if (factor) {
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) fac[ch] = r[8 + ch] + r[11 + ch];
    }
    tg[0] = __ldg(target + src * 3);
    tg[1] = __ldg(target + src * 3 + 1);
    tg[2] = __ldg(target + src * 3 + 2);
  } else {
#pragma unroll
    for (int i = 0; i < 64; ++i) h[i] = 0.0f;
  }
  __syncthreads();
  // forward, keeping every layer's input
  for (int l = 0; l < net.n_mats - 1; ++l) {
    float* Hl = Hs + l * 64 * kHStride;
#pragma unroll
    for (int i = 0; i < 64; ++i) Hl[i * kHStride + tid] = h[i];
    dense64_relu(sw + net.w_off[l], h, z);
#pragma unroll
    for (int i = 0; i < 64; ++i) h[i] = z[i];
  }
  {
    float* Hl = Hs + (net.n_mats - 1) * 64 * kHStride;
#pragma unroll
    for (int i = 0; i < 64; ++i) Hl[i * kHStride + tid] = h[i];
  }
  float y[3], g[3], loss_row;
  dense_out(sw + net.w_off[net.n_mats - 1], h, y);
  // factorisation: the loss sees y * f, the network output the gradient times f
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) y[ch] *= fac[ch];
  relative_l2(y, tg, loss_mode, loss_eps, g, &loss_row);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) g[ch] *= fac[ch];
  if (!valid) {
    g[0] = g[1] = g[2] = 0.0f;
    loss_row = 0.0f;
  }
  float* P = partials + size_t(blockIdx.x) * partial_stride(net.n_params);
  // backward: d holds delta_{l+1} of this row
  float d[64];
#pragma unroll
  for (int o = 0; o < 64; ++o) d[o] = o < 3 ? g[o] * inv3n : 0.0f;
  for (int l = net.n_mats - 1; l >= 0; --l) {
    const int dout = net.dims[l + 1];
    __syncthreads();  // previous layer's readers of Ds are done
    for (int o = 0; o < dout; ++o) Ds[o * kDStride + tid] = d[o];
    __syncthreads();
    // dW_l[o][i] = sum over this CTA's rows of delta_{l+1}[o] H_l[i]; thread = input i
    {
      const float* Hl = Hs + l * 64 * kHStride + tid * kHStride;
      float acc[64];
#pragma unroll
      for (int o = 0; o < 64; ++o) acc[o] = 0.0f;
      for (int r0 = 0; r0 < kTrainRows; r0 += 4) {
        const float h0 = Hl[r0], h1 = Hl[r0 + 1], h2 = Hl[r0 + 2], h3 = Hl[r0 + 3];
        if (dout == 64) {
#pragma unroll
          for (int o = 0; o < 64; ++o) {
            const float4 dv = *reinterpret_cast<const float4*>(Ds + o * kDStride + r0);
            acc[o] = fmaf(dv.x, h0, acc[o]);
            acc[o] = fmaf(dv.y, h1, acc[o]);
            acc[o] = fmaf(dv.z, h2, acc[o]);
            acc[o] = fmaf(dv.w, h3, acc[o]);
          }
        } else {
#pragma unroll
          for (int o = 0; o < 3; ++o) {
            const float4 dv = *reinterpret_cast<const float4*>(Ds + o * kDStride + r0);
            acc[o] = fmaf(dv.x, h0, acc[o]);
            acc[o] = fmaf(dv.y, h1, acc[o]);
            acc[o] = fmaf(dv.z, h2, acc[o]);
            acc[o] = fmaf(dv.w, h3, acc[o]);
          }
        }
      }
      float* Pl = P + net.w_off[l];
      if (dout == 64) {
#pragma unroll
        for (int o = 0; o < 64; ++o) Pl[o * 64 + tid] = acc[o];
      } else {
#pragma unroll
        for (int o = 0; o < 3; ++o) Pl[o * 64 + tid] = acc[o];
      }
    }
    if (l == 0) break;
    // delta_l = (W_l^T delta_{l+1}) * [H_l > 0]
    {
      const float* Wl = sw + net.w_off[l];
      float nd[64];
#pragma unroll
      for (int i = 0; i < 64; ++i) nd[i] = 0.0f;
      if (dout == 64) {
#pragma unroll 4
        for (int o = 0; o < 64; ++o) {
          const float4* wr = reinterpret_cast<const float4*>(Wl + o * 64);
          const float dv = Ds[o * kDStride + tid];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float4 wv = wr[q];
            nd[4 * q] = fmaf(wv.x, dv, nd[4 * q]);
            nd[4 * q + 1] = fmaf(wv.y, dv, nd[4 * q + 1]);
            nd[4 * q + 2] = fmaf(wv.z, dv, nd[4 * q + 2]);
            nd[4 * q + 3] = fmaf(wv.w, dv, nd[4 * q + 3]);
          }
        }
      } else {
        for (int o = 0; o < 3; ++o) {
          const float4* wr = reinterpret_cast<const float4*>(Wl + o * 64);
          const float dv = Ds[o * kDStride + tid];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float4 wv = wr[q];
            nd[4 * q] = fmaf(wv.x, dv, nd[4 * q]);
            nd[4 * q + 1] = fmaf(wv.y, dv, nd[4 * q + 1]);
            nd[4 * q + 2] = fmaf(wv.z, dv, nd[4 * q + 2]);
            nd[4 * q + 3] = fmaf(wv.w, dv, nd[4 * q + 3]);
          }
        }
      }
      const float* Hl = Hs + l * 64 * kHStride;
#pragma unroll
      for (int i = 0; i < 64; ++i) d[i] = Hl[i * kHStride + tid] > 0.0f ? nd[i] : 0.0f;
    }
  }
  // loss partial: fixed-order block sum
  float s = loss_row;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) {
    float tot = 0.0f;
    for (int k = 0; k < kTrainRows / 32; ++k) tot += red[k];
    P[net.n_params] = tot * inv3n;
  }
}

size_t train_simt_smem(const NetShape& net) {
  return size_t((net.n_params + 3) & ~3) * 4 + size_t(net.n_mats) * 64 * kHStride * 4 + 64 * kDStride * 4 + 16;
}

cudaError_t launch_train_simt(Cache* c, const float* pool, const float* target, int64_t n_pool, int64_t batch,
                              uint64_t a, uint64_t cc, int step, int* n_partials, cudaStream_t st) {
  const size_t smem = train_simt_smem(c->net);
  static std::atomic<int> attr_done[2];
  const int mode = c->cfg.enc_mode;
  {
    const cudaError_t e = mode == 0 ? ensure_smem(k_train_simt<0>, int(smem), &attr_done[0])
                                    : ensure_smem(k_train_simt<1>, int(smem), &attr_done[1]);
    if (e != cudaSuccess) return e;
  }
  const int blocks = int((batch + kTrainRows - 1) / kTrainRows);
  cudaError_t pe = ensure_partials(c, blocks);
  if (pe != cudaSuccess) return pe;
  const float inv3n = float(1.0 / (3.0 * double(batch)));
  if (mode == 0)
    k_train_simt<0><<<blocks, kTrainRows, smem, st>>>(pool, target, n_pool, batch, a, cc, step, c->w, c->net,
                                                      c->cfg.pad_value, c->cfg.loss_mode, c->cfg.loss_eps, inv3n,
                                                      c->partials, c->t, c->cfg.refl_factor);
  else
    k_train_simt<1><<<blocks, kTrainRows, smem, st>>>(pool, target, n_pool, batch, a, cc, step, c->w, c->net,
                                                      c->cfg.pad_value, c->cfg.loss_mode, c->cfg.loss_eps, inv3n,
                                                      c->partials, c->t, c->cfg.refl_factor);
  *n_partials = blocks;
  return cudaGetLastError();
}

// -------------------------------------------------------- reduce + Adam
// Sums the per-CTA weight-gradient partials in a fixed order (deterministic),
// scales them, and applies Adam (Sec. 5; Kingma & Ba 2015) with bias
// correction to the FP32 master weights; writes the 16-bit copy into the
// swizzled weight image when the cache computes in FP16/BF16.
// A block handles 32 consecutive weights (one per lane, coalesced reads);
// its 8 warps each sum every 8th partial, then warp 0 adds the 8 sums in
// warp order.  Block 0's warp 1 also sums the loss slots.
constexpr int kAdamGroups = 8;

// One block: the 32 weights p = blockIdx.x * 32 + lane of one cache.
template <int IMG>  // 0: no image, 1: FP16, 2: BF16
__device__ __forceinline__ void adam_block(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                                           const long long* __restrict__ t_ctr, const float* __restrict__ partials,
                                           int n_partials, const NetShape& net, const ImageShape& img,
                                           uint8_t* __restrict__ wimg, float grad_scale, float lr, float b1, float b2,
                                           float eps, float* __restrict__ loss_out, bool do_loss,
                                           float* __restrict__ ema, uint8_t* __restrict__ wimg_ema, float alpha) {
  __shared__ float red[kAdamGroups][32];
  __shared__ float corr[4];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const size_t stride = partial_stride(net.n_params);
  const int p = blockIdx.x * 32 + lane;
  if (do_loss && grp == 1 && loss_out) {
    float s = 0.0f;
    for (int k = lane; k < n_partials; k += 32) s += partials[size_t(k) * stride + net.n_params];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) *loss_out = s;
  }
  float part = 0.0f;
  if (p < net.n_params) {
    // 16 independent loads in flight per thread (the partials were just
    // written and sit in L2; latency, not bandwidth, bounds this loop)
    const float* src = partials + p;
    int k = grp;
    float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (; k + 15 * kAdamGroups < n_partials; k += 16 * kAdamGroups) {
      float t[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) t[u] = __ldcg(src + size_t(k + u * kAdamGroups) * stride);
#pragma unroll
      for (int u = 0; u < 16; ++u) a[u & 3] += t[u];
    }
    for (; k < n_partials; k += kAdamGroups) a[0] += __ldcg(src + size_t(k) * stride);
    part = (a[0] + a[1]) + (a[2] + a[3]);
  }
  if (threadIdx.x == 0) {  // bias corrections, once per block (after this thread's loads are in flight)
    const long long t = *t_ctr;
    corr[0] = 1.0f - pow_int(b1, t);
    corr[1] = 1.0f - pow_int(b2, t);
    if (ema) {
      corr[2] = 1.0f - pow_int(alpha, t);      // eta_t of Eq. 2
      corr[3] = 1.0f - pow_int(alpha, t - 1);  // eta_{t-1}
    }
  }
  red[grp][lane] = part;
  __syncthreads();
  if (grp != 0 || p >= net.n_params) return;
  float g = 0.0f;
#pragma unroll
  for (int q = 0; q < kAdamGroups; ++q) g += red[q][lane];
  g *= grad_scale;
  const float c1 = corr[0], c2 = corr[1];
  const float mn = fmaf(b1, m[p], (1.0f - b1) * g);
  const float vn = fmaf(b2, v[p], (1.0f - b2) * g * g);
  m[p] = mn;
  v[p] = vn;
  const float wn = w[p] - lr * (mn / c1) / (sqrtf(vn / c2) + eps);
  w[p] = wn;
  // the weight average of Eq. 2 (bias-corrected reading); it never feeds back
  // into training
  float en = 0.0f;
  if (ema) {
    en = ((1.0f - alpha) * wn + alpha * corr[3] * ema[p]) / corr[2];
    ema[p] = en;
  }
  if (IMG) {
    int l = 0;
    while (l + 1 < net.n_mats && p >= net.w_off[l + 1]) ++l;
    const int q = p - net.w_off[l];
    const int o = q / net.dims[l], i = q % net.dims[l];
    const uint32_t off = img_offset(img, l, uint32_t(o), uint32_t(i));
    if (IMG == 1) {
      *reinterpret_cast<__half*>(wimg + off) = __float2half_rn(wn);
      if (ema) *reinterpret_cast<__half*>(wimg_ema + off) = __float2half_rn(en);
    } else {
      *reinterpret_cast<__nv_bfloat16*>(wimg + off) = __float2bfloat16_rn(wn);
      if (ema) *reinterpret_cast<__nv_bfloat16*>(wimg_ema + off) = __float2bfloat16_rn(en);
    }
  }
}

template <int IMG>  // 0: no image, 1: FP16, 2: BF16
__global__ void __launch_bounds__(32 * kAdamGroups) k_adam(float* __restrict__ w, float* __restrict__ m,
                                                           float* __restrict__ v, const long long* __restrict__ t_ctr,
                                                           const float* __restrict__ partials, int n_partials,
                                                           const __grid_constant__ NetShape net,
                                                           const __grid_constant__ ImageShape img,
                                                           uint8_t* __restrict__ wimg, float grad_scale, float lr,
                                                           float b1, float b2, float eps, float* __restrict__ loss_out,
                                                           float* __restrict__ ema, uint8_t* __restrict__ wimg_ema,
                                                           float alpha) {
  pdl_wait();  // the partials and the step counter come from the kernel before
  pdl_launch_dependents();
  adam_block<IMG>(w, m, v, t_ctr, partials, n_partials, net, img, wimg, grad_scale, lr, b1, b2, eps, loss_out,
                  blockIdx.x == 0, ema, wimg_ema, alpha);
}

// All caches of a batched step: blockIdx.y selects the cache.
template <int IMG>
__global__ void __launch_bounds__(32 * kAdamGroups) k_adam_batched(const AdamJob* __restrict__ jobs,
                                                                   const __grid_constant__ NetShape net,
                                                                   const __grid_constant__ ImageShape img, float lr,
                                                                   float b1, float b2, float eps, float alpha) {
  pdl_wait();
  pdl_launch_dependents();
  const AdamJob J = jobs[blockIdx.y];
  adam_block<IMG>(J.w, J.m, J.v, J.t_ctr, J.partials, J.n_partials, net, img, J.wimg, J.grad_scale, lr, b1, b2, eps,
                  J.loss_out, blockIdx.x == 0, J.ema, J.wimg_ema, alpha);
}

cudaError_t launch_adam(Cache* c, int n_partials, float grad_scale, float* loss_out, cudaStream_t st) {
  const int threads = 32 * kAdamGroups;
  const int blocks = (c->net.n_params + 31) / 32;
  const nrc_config& k = c->cfg;
  // Launched with programmatic stream serialisation: its blocks may start
  // before the gradient kernel finishes and wait for it on the device.
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(unsigned(blocks));
  lc.blockDim = dim3(unsigned(threads));
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  const NetShape& net = c->net;
  const ImageShape& img = c->img;
  float* ema = k.ema ? c->ema : nullptr;
  if (fp16_like(k.dtype))
    return cudaLaunchKernelEx(&lc, k_adam<1>, c->w, c->m, c->v, (const long long*)c->t, (const float*)c->partials,
                              n_partials, net, img, c->wimg, grad_scale, k.lr, k.beta1, k.beta2, k.adam_eps, loss_out,
                              ema, c->wimg_ema, k.ema_alpha);
  if (k.dtype == NRC_BF16)
    return cudaLaunchKernelEx(&lc, k_adam<2>, c->w, c->m, c->v, (const long long*)c->t, (const float*)c->partials,
                              n_partials, net, img, c->wimg, grad_scale, k.lr, k.beta1, k.beta2, k.adam_eps, loss_out,
                              ema, c->wimg_ema, k.ema_alpha);
  return cudaLaunchKernelEx(&lc, k_adam<0>, c->w, c->m, c->v, (const long long*)c->t, (const float*)c->partials,
                            n_partials, net, img, c->wimg, grad_scale, k.lr, k.beta1, k.beta2, k.adam_eps, loss_out,
                            ema, c->wimg_ema, k.ema_alpha);
}

cudaError_t launch_adam_batched(const Cache* proto, const AdamJob* jobs, int n_jobs, cudaStream_t st) {
  const nrc_config& k = proto->cfg;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(unsigned((proto->net.n_params + 31) / 32), unsigned(n_jobs));
  lc.blockDim = dim3(32 * kAdamGroups);
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  if (k.dtype == NRC_FP16) return cudaLaunchKernelEx(&lc, k_adam_batched<1>, jobs, proto->net, proto->img, k.lr, k.beta1, k.beta2, k.adam_eps, k.ema_alpha);
  if (k.dtype == NRC_BF16) return cudaLaunchKernelEx(&lc, k_adam_batched<2>, jobs, proto->net, proto->img, k.lr, k.beta1, k.beta2, k.adam_eps, k.ema_alpha);
  return cudaLaunchKernelEx(&lc, k_adam_batched<0>, jobs, proto->net, proto->img, k.lr, k.beta1, k.beta2, k.adam_eps, k.ema_alpha);
}

__global__ void k_step_increment(long long* t) { *t += 1; }

cudaError_t launch_step_increment(Cache* c, cudaStream_t st) {
  k_step_increment<<<1, 1, 0, st>>>(c->t);
  return cudaGetLastError();
}

// ------------------------------------------------------------ weight image
template <int IMG>
__global__ void k_build_image(const float* __restrict__ w, const __grid_constant__ NetShape net,
                              const __grid_constant__ ImageShape img, uint8_t* __restrict__ wimg) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= net.n_params) return;
  int l = 0;
  while (l + 1 < net.n_mats && p >= net.w_off[l + 1]) ++l;
  const int q = p - net.w_off[l];
  const int o = q / net.dims[l], i = q % net.dims[l];
  uint8_t* dst = wimg + img_offset(img, l, uint32_t(o), uint32_t(i));
  if (IMG == 1)
    *reinterpret_cast<__half*>(dst) = __float2half_rn(w[p]);
  else
    *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(w[p]);
}

cudaError_t launch_build_image_of(const Cache* c, const float* w, uint8_t* img, cudaStream_t st) {
  if (c->cfg.dtype == NRC_FP32) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(img, 0, size_t(c->img.off[c->net.n_mats]), st);
  if (e != cudaSuccess) return e;
  const int threads = 256;
  const int blocks = (c->net.n_params + threads - 1) / threads;
  if (fp16_like(c->cfg.dtype))
    k_build_image<1><<<blocks, threads, 0, st>>>(w, c->net, c->img, img);
  else
    k_build_image<2><<<blocks, threads, 0, st>>>(w, c->net, c->img, img);
  return cudaGetLastError();
}

cudaError_t launch_build_image(Cache* c, cudaStream_t st) { return launch_build_image_of(c, c->w, c->wimg, st); }

}  // namespace nrc
