// Plain per-layer FP32 path: the same arithmetic as the fused kernels, but
// every stage is its own kernel and every activation, delta and gradient
// partial round-trips through HBM -- the unfused way of running the network
// (the reference point the paper measures its fused network against, Fig. 5).
#include "nrc_internal.cuh"

namespace nrc {

constexpr int kPR = 64;       // rows per CTA
constexpr int kPS = 65;       // padded shared-memory row stride

// Y[r][o] = sum_i X[r][i] W[o][i] (ReLU optional); X [n][din], W [dout][din]
// (din, dout <= 128).  A CTA computes 64 rows x 64 outputs (blockIdx.y selects
// the output block), the inner dimension in chunks of 64 through shared memory.
template <bool RELU>
__global__ void __launch_bounds__(256) k_plain_dense(const float* __restrict__ X, const float* __restrict__ W,
                                                     float* __restrict__ Y, int64_t n, int din, int dout) {
  __shared__ float Xs[kPR * kPS];
  __shared__ float Ws[64 * kPS];
  const int tid = threadIdx.x;
  const int64_t r0 = int64_t(blockIdx.x) * kPR;
  const int o0 = blockIdx.y * 64;
  const int ty = tid >> 4, tx = tid & 15;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < din; k0 += 64) {
    __syncthreads();
    for (int e = tid; e < kPR * 64; e += 256) {
      const int r = e >> 6, k = e & 63;
      Xs[r * kPS + k] = (r0 + r < n && k0 + k < din) ? X[(r0 + r) * din + k0 + k] : 0.0f;
    }
    for (int e = tid; e < 64 * 64; e += 256) {
      const int o = e >> 6, k = e & 63;
      Ws[o * kPS + k] = (o0 + o < dout && k0 + k < din) ? W[(o0 + o) * din + k0 + k] : 0.0f;
    }
    __syncthreads();
    for (int k = 0; k < 64; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) a[j] = Xs[(ty * 4 + j) * kPS + k];
#pragma unroll
      for (int i = 0; i < 4; ++i) b[i] = Ws[(tx * 4 + i) * kPS + k];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = fmaf(a[j], b[i], acc[j][i]);
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t r = r0 + ty * 4 + j;
    if (r >= n) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int o = o0 + tx * 4 + i;
      if (o < dout) Y[r * dout + o] = RELU ? fmaxf(acc[j][i], 0.0f) : acc[j][i];
    }
  }
}

// Relative L2 loss (Eq. 5): G[r] = dL/dy scaled by 1/(3N); per-CTA loss sums
// go to the loss slot of the CTA's partial.  With rec (reflectance
// factorisation, Sec. 5) the loss sees y times the record's diffuse +
// specular albedo f, and G is dL/d(y f) times f.
__global__ void __launch_bounds__(kPR) k_plain_loss(const float* __restrict__ Yh, const float* __restrict__ T,
                                                    float* __restrict__ G, int64_t n, int loss_mode, float eps,
                                                    float inv3n, float* __restrict__ partials, int n_params,
                                                    const float* __restrict__ rec) {
  __shared__ float red[kPR / 32];
  const int64_t r = int64_t(blockIdx.x) * kPR + threadIdx.x;
  float loss_row = 0.0f;
  if (r < n) {
    float y[3], f[3] = {1.0f, 1.0f, 1.0f};
    for (int ch = 0; ch < 3; ++ch) {
      if (rec) f[ch] = rec[r * kRecFloats + 8 + ch] + rec[r * kRecFloats + 11 + ch];
      y[ch] = Yh[r * 3 + ch] * f[ch];
    }
    const float lum = 0.2126f * y[0] + 0.7152f * y[1] + 0.0722f * y[2];
    for (int ch = 0; ch < 3; ++ch) {
      const float den = (loss_mode == NRC_LOSS_LUMINANCE ? lum * lum : y[ch] * y[ch]) + eps;
      const float inv = 1.0f / den;
      const float diff = y[ch] - T[r * 3 + ch];
      loss_row = fmaf(diff * diff, inv, loss_row);
      G[r * 3 + ch] = 2.0f * diff * inv * inv3n * f[ch];
    }
  }
  float s = loss_row;
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.0f;
    for (int k = 0; k < kPR / 32; ++k) tot += red[k];
    partials[size_t(blockIdx.x) * partial_stride(n_params) + n_params] = tot * inv3n;
  }
}

// Din[r][i] = (sum_o Dout[r][o] W[o][i]) * [H[r][i] > 0]; Dout [n][dout],
// W [dout][din], H and Din [n][din].  blockIdx.y selects 64 of the inputs.
__global__ void __launch_bounds__(256) k_plain_bwd(const float* __restrict__ Dout, const float* __restrict__ W,
                                                   const float* __restrict__ H, float* __restrict__ Din, int64_t n,
                                                   int dout, int din) {
  __shared__ float Ds[kPR * kPS];
  __shared__ float Ws[64 * kPS];
  const int tid = threadIdx.x;
  const int64_t r0 = int64_t(blockIdx.x) * kPR;
  const int i0 = blockIdx.y * 64;
  const int ty = tid >> 4, tx = tid & 15;
  float acc[4][4] = {};
  for (int o0 = 0; o0 < dout; o0 += 64) {
    __syncthreads();
    for (int e = tid; e < kPR * 64; e += 256) {
      const int r = e >> 6, o = e & 63;
      Ds[r * kPS + o] = (r0 + r < n && o0 + o < dout) ? Dout[(r0 + r) * dout + o0 + o] : 0.0f;
    }
    for (int e = tid; e < 64 * 64; e += 256) {
      const int o = e >> 6, i = e & 63;
      Ws[o * kPS + i] = (o0 + o < dout && i0 + i < din) ? W[(o0 + o) * din + i0 + i] : 0.0f;
    }
    __syncthreads();
    for (int o = 0; o < 64; ++o) {
      float a[4], b[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) a[j] = Ds[(ty * 4 + j) * kPS + o];
#pragma unroll
      for (int i = 0; i < 4; ++i) b[i] = Ws[o * kPS + tx * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = fmaf(a[j], b[i], acc[j][i]);
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t r = r0 + ty * 4 + j;
    if (r >= n) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int c = i0 + tx * 4 + i;
      if (c < din) Din[r * din + c] = H[r * din + c] > 0.0f ? acc[j][i] : 0.0f;
    }
  }
}

// Partial k of dW[o][i] = sum over rows of chunk k of D[r][o] H[r][i];
// blockIdx.y selects a 64 x 64 block of dW (output block major).
__global__ void __launch_bounds__(256) k_plain_dw(const float* __restrict__ D, const float* __restrict__ H,
                                                  float* __restrict__ partials, int64_t n, int dout, int din,
                                                  int w_off, int n_params) {
  __shared__ float Ds[kPR * kPS];
  __shared__ float Hs[kPR * kPS];
  const int tid = threadIdx.x;
  const int64_t r0 = int64_t(blockIdx.x) * kPR;
  const int ib = (din + 63) / 64;
  const int o0 = (blockIdx.y / ib) * 64, i0 = (blockIdx.y % ib) * 64;
  for (int e = tid; e < kPR * 64; e += 256) {
    const int r = e >> 6, c = e & 63;
    const bool ok = r0 + r < n;
    Ds[r * kPS + c] = (ok && o0 + c < dout) ? D[(r0 + r) * dout + o0 + c] : 0.0f;
    Hs[r * kPS + c] = (ok && i0 + c < din) ? H[(r0 + r) * din + i0 + c] : 0.0f;
  }
  __syncthreads();
  const int to = tid >> 4, ti = tid & 15;
  float acc[4][4] = {};
  for (int r = 0; r < kPR; ++r) {
    float a[4], b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = Ds[r * kPS + to * 4 + j];
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = Hs[r * kPS + ti * 4 + i];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[j][i] = fmaf(a[j], b[i], acc[j][i]);
  }
  float* P = partials + size_t(blockIdx.x) * partial_stride(n_params) + w_off;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int o = o0 + to * 4 + j;
    if (o >= dout) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int c = i0 + ti * 4 + i;
      if (c < din) P[o * din + c] = acc[j][i];
    }
  }
}

static cudaError_t ensure_plain(Cache* c, size_t bytes) {
  if (bytes <= c->plain_bytes) return cudaSuccess;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  cudaFree(c->plain_buf);
  c->plain_buf = nullptr;
  c->plain_bytes = 0;
  e = dev_alloc(&c->plain_buf, bytes);
  if (e == cudaSuccess) c->plain_bytes = bytes;
  return e;
}

// Reflectance factorisation of query outputs: rgb[r] *= diffuse + specular albedo.
__global__ void __launch_bounds__(kPR) k_plain_factor(const float* __restrict__ rec, int64_t n, float* __restrict__ rgb) {
  const int64_t r = int64_t(blockIdx.x) * kPR + threadIdx.x;
  if (r >= n) return;
  for (int ch = 0; ch < 3; ++ch) rgb[r * 3 + ch] *= rec[r * kRecFloats + 8 + ch] + rec[r * kRecFloats + 11 + ch];
}

static unsigned out_blocks(int d) { return unsigned((d + 63) / 64); }

cudaError_t plain_infer(Cache* c, const float* rec, int64_t n, float* rgb, cudaStream_t st) {
  const size_t act = size_t(n) * size_t(c->net.dims[1] > 64 ? c->net.dims[1] : 64);
  cudaError_t e = ensure_plain(c, act * 2 * 4);
  if (e != cudaSuccess) return e;
  float* A = c->plain_buf;
  float* B = A + act;
  e = launch_encode(rec, n, A, NRC_FP32, c->cfg.enc_mode, c->cfg.pad_value, st);
  c->launches += 1;
  if (e != cudaSuccess) return e;
  const unsigned blocks = unsigned((n + kPR - 1) / kPR);
  const NetShape& s = c->net;
  for (int l = 0; l < s.n_mats; ++l) {
    const float* W = query_weights(c) + s.w_off[l];
    const dim3 grid(blocks, out_blocks(s.dims[l + 1]));
    if (l + 1 < s.n_mats)
      k_plain_dense<true><<<grid, 256, 0, st>>>(A, W, B, n, s.dims[l], s.dims[l + 1]);
    else
      k_plain_dense<false><<<grid, 256, 0, st>>>(A, W, rgb, n, s.dims[l], s.dims[l + 1]);
    c->launches += 1;
    float* t = A;
    A = B;
    B = t;
  }
  if (c->cfg.refl_factor) {
    k_plain_factor<<<blocks, kPR, 0, st>>>(rec, n, rgb);
    c->launches += 1;
  }
  return cudaGetLastError();
}

cudaError_t plain_train(Cache* c, const float* pool, const float* target, int64_t n_pool, int64_t batch, uint64_t a,
                        uint64_t cc, int step, float* loss_out, cudaStream_t st) {
  const NetShape& s = c->net;
  const size_t B = size_t(batch);
  // rec [B][16], tgt [B][3], H_0..H_{L-1} [B][dims[l]] (slots of Wd = max width), Y [B][3], G [B][3],
  // D0/D1 [B][Wd]
  const size_t Wd = size_t(s.dims[1] > 64 ? s.dims[1] : 64);
  const size_t need = B * 16 + B * 4 + size_t(s.n_mats) * B * Wd + B * 4 + B * 4 + 2 * B * Wd;
  cudaError_t e = ensure_plain(c, need * 4);
  if (e != cudaSuccess) return e;
  const unsigned blocks = unsigned((batch + kPR - 1) / kPR);
  e = ensure_partials(c, int(blocks));
  if (e != cudaSuccess) return e;
  float* rec = c->plain_buf;
  float* tgt = rec + B * 16;
  float* H = tgt + B * 4;
  float* Y = H + size_t(s.n_mats) * B * Wd;
  float* G = Y + B * 4;
  float* D0 = G + B * 4;
  float* D1 = D0 + B * Wd;
  e = launch_gather(pool, target, n_pool, batch, a, cc, step, rec, tgt, st);
  if (e != cudaSuccess) return e;
  e = launch_encode(rec, batch, H, NRC_FP32, c->cfg.enc_mode, c->cfg.pad_value, st);
  if (e != cudaSuccess) return e;
  c->launches += 2;
  for (int l = 0; l < s.n_mats; ++l) {
    const float* W = c->w + s.w_off[l];
    float* X = H + size_t(l) * B * Wd;
    const dim3 grid(blocks, out_blocks(s.dims[l + 1]));
    if (l + 1 < s.n_mats)
      k_plain_dense<true><<<grid, 256, 0, st>>>(X, W, X + B * Wd, batch, s.dims[l], s.dims[l + 1]);
    else
      k_plain_dense<false><<<grid, 256, 0, st>>>(X, W, Y, batch, s.dims[l], s.dims[l + 1]);
    c->launches += 1;
  }
  const float inv3n = float(1.0 / (3.0 * double(batch)));
  k_plain_loss<<<blocks, kPR, 0, st>>>(Y, tgt, G, batch, c->cfg.loss_mode, c->cfg.loss_eps, inv3n, c->partials,
                                      s.n_params, c->cfg.refl_factor ? rec : nullptr);
  c->launches += 1;
  const float* Dcur = G;
  float* Dnext = D0;
  for (int l = s.n_mats - 1; l >= 0; --l) {
    const float* Hl = H + size_t(l) * B * Wd;
    k_plain_dw<<<dim3(blocks, out_blocks(s.dims[l + 1]) * out_blocks(s.dims[l])), 256, 0, st>>>(
        Dcur, Hl, c->partials, batch, s.dims[l + 1], s.dims[l], s.w_off[l], s.n_params);
    c->launches += 1;
    if (l == 0) break;
    k_plain_bwd<<<dim3(blocks, out_blocks(s.dims[l])), 256, 0, st>>>(Dcur, c->w + s.w_off[l], Hl, Dnext, batch,
                                                                     s.dims[l + 1], s.dims[l]);
    c->launches += 1;
    Dcur = Dnext;
    Dnext = (Dnext == D0) ? D1 : D0;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // t is incremented by a one-element add so that Adam sees this step's t.
  e = launch_step_increment(c, st);
  if (e != cudaSuccess) return e;
  e = c->cfg.optimizer == NRC_OPT_SHAMPOO ? launch_shampoo(c, int(blocks), 1.0f, loss_out, st)
                                          : launch_adam(c, int(blocks), 1.0f, loss_out, st);
  c->launches += 2;
  return e;
}

}  // namespace nrc
