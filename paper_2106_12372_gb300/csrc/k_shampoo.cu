// Shampoo, the second-order optimiser the paper evaluated beside Adam
// (Sec. 5 "Optimizer"; Gupta et al. 2018, with the exponential statistics,
// root interval and Adam grafting of Anil et al. 2020).  Per weight matrix
// W_l (out x in) with gradient G:
//   m <- b1 m + (1-b1) G,  v <- b2 v + (1-b2) G*G          (Adam's moments)
//   L <- b2 L + (1-b2) G G^T,  R <- b2 R + (1-b2) G^T G
//   every `interval` steps from step 1:
//     P_L = (L/(1-b2^t) + eps I)^(-1/4), P_R likewise, eps = eps_rel tr(.)/n
//   D = P_L m^ P_R,  A = m^ / (sqrt(v^) + adam_eps)
//   W <- W - lr D ||A||_F / ||D||_F                         (layer-wise grafting)
// Three launches follow the gradient kernel: k_shampoo_grad (reduces the
// weight-gradient partials, updates m and v, the per-block ||A||^2),
// k_shampoo_roots (one CTA per statistic: update, and on root steps the
// inverse fourth root by the coupled Newton iteration of Guo & Higham 2006 in
// FP32 shared memory), k_shampoo_update (one CTA per layer: D, grafting, the
// weights, their 16-bit image and the weight average).
#include "nrc_internal.cuh"

namespace nrc {

constexpr int kShN = 64;          // statistics are stored as 64 x 64 (logical size n <= 64)
constexpr int kShThreads = 256;   // 16 x 16 threads, a 4 x 4 block of a 64 x 64 product each
constexpr int kShMaxIter = 40;

// Weight gradient of one 32-weight block: the fixed-order sum of the partials
// (the same reduction as the Adam kernel).  Valid in group 0 for p < n_params.
__device__ __forceinline__ float reduce_grad(const float* __restrict__ partials, int n_partials, int n_params,
                                             int p, bool valid, int grp, int lane, float (*red)[32]) {
  const size_t stride = partial_stride(n_params);
  float part = 0.0f;
  if (valid) {
    const float* src = partials + p;
    float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int k = grp;
    for (; k + 15 * 8 < n_partials; k += 16 * 8) {
      float t[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) t[u] = __ldcg(src + size_t(k + u * 8) * stride);
#pragma unroll
      for (int u = 0; u < 16; ++u) a[u & 3] += t[u];
    }
    for (; k < n_partials; k += 8) a[0] += __ldcg(src + size_t(k) * stride);
    part = (a[0] + a[1]) + (a[2] + a[3]);
  }
  red[grp][lane] = part;
  __syncthreads();
  float g = 0.0f;
  if (grp == 0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) g += red[q][lane];
  }
  return g;
}

// grid: one block of 256 threads (8 groups) per 32 weights.
__global__ void __launch_bounds__(kShThreads) k_shampoo_grad(const float* __restrict__ partials, int n_partials,
                                                             const __grid_constant__ NetShape net, float grad_scale, const long long* __restrict__ t_ctr,
                                                             float* __restrict__ G, float* __restrict__ m,
                                                             float* __restrict__ v, float* __restrict__ anorm,
                                                             float b1, float b2, float adam_eps,
                                                             float* __restrict__ loss_out) {
  pdl_wait();  // the partials and the step counter come from the gradient kernel
  pdl_launch_dependents();
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + lane;
  const bool valid = p < net.n_params;
  if (blockIdx.x == 0 && grp == 1 && loss_out) {
    const size_t stride = partial_stride(net.n_params);
    float s = 0.0f;
    for (int k = lane; k < n_partials; k += 32) s += partials[size_t(k) * stride + net.n_params];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) *loss_out = s;
  }
  const float g = reduce_grad(partials, n_partials, net.n_params, p, valid, grp, lane, red) * grad_scale;
  if (grp != 0) return;
  const long long t = *t_ctr;
  float a2 = 0.0f;
  if (valid) {
    const float mn = fmaf(b1, m[p], (1.0f - b1) * g);
    const float vn = fmaf(b2, v[p], (1.0f - b2) * g * g);
    m[p] = mn;
    v[p] = vn;
    G[p] = g;
    const float A = (mn / (1.0f - pow_int(b1, t))) / (sqrtf(vn / (1.0f - pow_int(b2, t))) + adam_eps);
    a2 = A * A;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a2 += __shfl_down_sync(0xffffffffu, a2, off);
  if (lane == 0) anorm[blockIdx.x] = a2;
}

// C = A B for n x n matrices stored 64 x 64 row-major in shared memory (zero
// outside n x n); thread (ty, tx) computes rows 4ty.., columns 4tx...
__device__ __forceinline__ void sh_matmul(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ C,
                                          int n) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int k = 0; k < n; ++k) {
    float a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = A[(4 * ty + r) * kShN + k];
    const float4 bv = *reinterpret_cast<const float4*>(B + k * kShN + 4 * tx);
    b[0] = bv.x;
    b[1] = bv.y;
    b[2] = bv.z;
    b[3] = bv.w;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
    *reinterpret_cast<float4*>(C + (4 * ty + r) * kShN + 4 * tx) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
}

__device__ __forceinline__ float block_sum(float x, float* scratch) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = x;
  __syncthreads();
  float s = 0.0f;
#pragma unroll
  for (int w = 0; w < kShThreads / 32; ++w) s += scratch[w];
  return s;
}

__device__ __forceinline__ float block_max(float x, float* scratch) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x = fmaxf(x, __shfl_down_sync(0xffffffffu, x, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = x;
  __syncthreads();
  float s = 0.0f;
#pragma unroll
  for (int w = 0; w < kShThreads / 32; ++w) s = fmaxf(s, scratch[w]);
  return s;
}

// grid: 2 * n_mats blocks; block 2l updates L_l (out x out), block 2l+1 R_l
// (in x in), and on root steps writes the inverse fourth root.
__global__ void __launch_bounds__(kShThreads) k_shampoo_roots(const __grid_constant__ NetShape net,
                                                              const float* __restrict__ G, float* __restrict__ stats,
                                                              float* __restrict__ roots,
                                                              const long long* __restrict__ t_ctr, float b2,
                                                              float eps_rel, int interval) {
  extern __shared__ float4 sh_f4[];
  float* S = reinterpret_cast<float*>(sh_f4);  // statistic; later M
  float* Gs = S + kShN * kShN;                 // G_l (out x in), zero padded; later X
  float* T = Gs + kShN * kShN;
  float* U = T + kShN * kShN;
  float* V = U + kShN * kShN;
  __shared__ float scratch[kShThreads / 32];
  const int l = blockIdx.x >> 1, side = blockIdx.x & 1;
  const int n_out = net.dims[l + 1], n_in = net.dims[l];
  const int n = side ? n_in : n_out;
  float* gS = stats + size_t(blockIdx.x) * kShN * kShN;
  const float* gl = G + net.w_off[l];
  for (int e = threadIdx.x; e < kShN * kShN; e += kShThreads) {
    const int r = e / kShN, c = e % kShN;
    Gs[e] = (r < n_out && c < n_in) ? gl[r * n_in + c] : 0.0f;
    S[e] = gS[e];
  }
  __syncthreads();
  // GG^T (side 0) or G^T G (side 1) into T; the statistic's exponential average
  {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    const int kn = side ? n_out : n_in;
    for (int k = 0; k < kn; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        a[r] = side ? Gs[k * kShN + 4 * ty + r] : Gs[(4 * ty + r) * kShN + k];
        b[r] = side ? Gs[k * kShN + 4 * tx + r] : Gs[(4 * tx + r) * kShN + k];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int e = (4 * ty + r) * kShN + 4 * tx + c;
        S[e] = fmaf(b2, S[e], (1.0f - b2) * acc[r][c]);
      }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kShN * kShN; e += kShThreads) gS[e] = S[e];
  const long long t = *t_ctr;
  if ((t - 1) % interval != 0) return;

  // S^ = S / (1 - b2^t) + eps I on the n x n block (zero outside)
  const float inv_c = 1.0f / (1.0f - pow_int(b2, t));
  float tr = 0.0f;
  for (int d = threadIdx.x; d < n; d += kShThreads) tr += S[d * kShN + d];
  tr = block_sum(tr, scratch) * inv_c;
  const float eps = eps_rel * tr / float(n) + 1e-30f;
  float fro2 = 0.0f;
  for (int e = threadIdx.x; e < kShN * kShN; e += kShThreads) {
    const int r = e / kShN, c = e % kShN;
    float x = (r < n && c < n) ? S[e] * inv_c : 0.0f;
    if (r == c && r < n) x += eps;
    S[e] = x;
    fro2 += x * x;
  }
  fro2 = block_sum(fro2, scratch);
  // coupled Newton for S^(-1/4): M_0 = S / c^4, X_0 = I / c with c^4 = ||S||_F >= lambda_max,
  // T = (5 I - M) / 4, X <- X T, M <- T^4 M (all n x n, zero outside)
  const float c4 = fmaxf(sqrtf(fro2), 1e-30f);
  const float c1 = sqrtf(sqrtf(c4));
  float* M = S;
  float* X = Gs;
  for (int e = threadIdx.x; e < kShN * kShN; e += kShThreads) {
    const int r = e / kShN, c = e % kShN;
    M[e] = M[e] / c4;
    X[e] = (r == c && r < n) ? 1.0f / c1 : 0.0f;
  }
  __syncthreads();
  for (int it = 0; it < kShMaxIter; ++it) {
    for (int e = threadIdx.x; e < kShN * kShN; e += kShThreads) {
      const int r = e / kShN, c = e % kShN;
      T[e] = (r == c && r < n) ? (5.0f - M[e]) * 0.25f : -0.25f * M[e];
    }
    __syncthreads();
    sh_matmul(X, T, U, n);  // U = X T
    sh_matmul(T, T, V, n);  // V = T^2
    __syncthreads();
    for (int e = threadIdx.x; e < kShN * kShN; e += kShThreads) X[e] = U[e];
    sh_matmul(V, V, T, n);  // T = T^4 (T is no longer read)
    __syncthreads();
    sh_matmul(T, M, U, n);  // U = T^4 M
    __syncthreads();
    float dev = 0.0f;
    for (int e = threadIdx.x; e < kShN * kShN; e += kShThreads) {
      const int r = e / kShN, c = e % kShN;
      M[e] = U[e];
      if (r < n && c < n) dev = fmaxf(dev, fabsf(U[e] - (r == c ? 1.0f : 0.0f)));
    }
    dev = block_max(dev, scratch);  // (its barriers also order the M update)
    if (dev < 2e-6f) break;
  }
  float* gR = roots + size_t(blockIdx.x) * kShN * kShN;
  for (int e = threadIdx.x; e < kShN * kShN; e += kShThreads) gR[e] = X[e];
}

// grid: n_mats blocks; block l applies the grafted Shampoo step to W_l.
template <int IMG>  // 0: no image, 1: FP16, 2: BF16
__global__ void __launch_bounds__(kShThreads) k_shampoo_update(const __grid_constant__ NetShape net,
                                                               const __grid_constant__ ImageShape img,
                                                               float* __restrict__ w, const float* __restrict__ m,
                                                               const float* __restrict__ roots,
                                                               const float* __restrict__ anorm,
                                                               const long long* __restrict__ t_ctr, float lr, float b1,
                                                               uint8_t* __restrict__ wimg, float* __restrict__ ema,
                                                               uint8_t* __restrict__ wimg_ema, float alpha) {
  extern __shared__ float4 sh_f4[];
  float* PL = reinterpret_cast<float*>(sh_f4);
  float* Mh = PL + kShN * kShN;
  float* PR = Mh + kShN * kShN;
  float* D = PR + kShN * kShN;
  __shared__ float scratch[kShThreads / 32];
  const int l = blockIdx.x;
  const int n_out = net.dims[l + 1], n_in = net.dims[l];
  const long long t = *t_ctr;
  const float inv_b1 = 1.0f / (1.0f - pow_int(b1, t));
  const float* gL = roots + size_t(2 * l) * kShN * kShN;
  const float* gR = roots + size_t(2 * l + 1) * kShN * kShN;
  const float* ml = m + net.w_off[l];
  for (int e = threadIdx.x; e < kShN * kShN; e += kShThreads) {
    const int r = e / kShN, c = e % kShN;
    PL[e] = gL[e];
    PR[e] = gR[e];
    Mh[e] = (r < n_out && c < n_in) ? ml[r * n_in + c] * inv_b1 : 0.0f;
  }
  __syncthreads();
  sh_matmul(PL, Mh, D, kShN);  // P_L m^
  __syncthreads();
  sh_matmul(D, PR, Mh, kShN);  // (P_L m^) P_R
  __syncthreads();
  float d2 = 0.0f;
  for (int e = threadIdx.x; e < n_out * n_in; e += kShThreads) {
    const float x = Mh[(e / n_in) * kShN + e % n_in];
    d2 += x * x;
  }
  d2 = block_sum(d2, scratch);
  float a2 = 0.0f;  // ||A||^2 of this layer, blocks of 32 weights in fixed order
  for (int b = net.w_off[l] / 32; b < net.w_off[l + 1] / 32; ++b) a2 += anorm[b];
  const float scale = d2 > 0.0f ? lr * sqrtf(a2 / d2) : 0.0f;
  float eta_t = 1.0f, eta_p = 0.0f;
  if (ema) {
    eta_t = 1.0f - pow_int(alpha, t);
    eta_p = 1.0f - pow_int(alpha, t - 1);
  }
  for (int e = threadIdx.x; e < n_out * n_in; e += kShThreads) {
    const int o = e / n_in, i = e % n_in;
    const int p = net.w_off[l] + e;
    const float wn = w[p] - scale * Mh[o * kShN + i];
    w[p] = wn;
    float en = 0.0f;
    if (ema) {
      en = ((1.0f - alpha) * wn + alpha * eta_p * ema[p]) / eta_t;
      ema[p] = en;
    }
    if (IMG) {
      const uint32_t off = img.off[l] + sw128_offset(o, i);
      if (IMG == 1) {
        *reinterpret_cast<__half*>(wimg + off) = __float2half_rn(wn);
        if (ema) *reinterpret_cast<__half*>(wimg_ema + off) = __float2half_rn(en);
      } else {
        *reinterpret_cast<__nv_bfloat16*>(wimg + off) = __float2bfloat16_rn(wn);
        if (ema) *reinterpret_cast<__nv_bfloat16*>(wimg_ema + off) = __float2bfloat16_rn(en);
      }
    }
  }
}

cudaError_t launch_shampoo(Cache* c, int n_partials, float grad_scale, float* loss_out, cudaStream_t st) {
  const nrc_config& k = c->cfg;
  const NetShape& net = c->net;
  const int blocks = (net.n_params + 31) / 32;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(unsigned(blocks));
  lc.blockDim = dim3(kShThreads);
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&lc, k_shampoo_grad, (const float*)c->partials, n_partials, net, grad_scale, (const long long*)c->t, c->sh_g, c->m, c->v, c->sh_anorm, k.beta1,
                                     k.beta2, k.adam_eps, loss_out);
  if (e != cudaSuccess) return e;
  static std::atomic<int> attr_done[4];
  const int smem_roots = 5 * kShN * kShN * 4, smem_update = 4 * kShN * kShN * 4;
  e = ensure_smem(k_shampoo_roots, smem_roots, &attr_done[0]);
  if (e == cudaSuccess) e = ensure_smem(k_shampoo_update<0>, smem_update, &attr_done[1]);
  if (e == cudaSuccess) e = ensure_smem(k_shampoo_update<1>, smem_update, &attr_done[2]);
  if (e == cudaSuccess) e = ensure_smem(k_shampoo_update<2>, smem_update, &attr_done[3]);
  if (e != cudaSuccess) return e;
  k_shampoo_roots<<<2 * net.n_mats, kShThreads, smem_roots, st>>>(net, c->sh_g, c->sh_stats, c->sh_roots,
                                                                  (const long long*)c->t, k.beta2, k.shampoo_eps,
                                                                  k.shampoo_interval);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  float* ema = k.ema ? c->ema : nullptr;
  if (fp16_like(k.dtype))
    k_shampoo_update<1><<<net.n_mats, kShThreads, smem_update, st>>>(net, c->img, c->w, c->m, c->sh_roots, c->sh_anorm,
                                                                     (const long long*)c->t, k.lr, k.beta1, c->wimg,
                                                                     ema, c->wimg_ema, k.ema_alpha);
  else if (k.dtype == NRC_BF16)
    k_shampoo_update<2><<<net.n_mats, kShThreads, smem_update, st>>>(net, c->img, c->w, c->m, c->sh_roots, c->sh_anorm,
                                                                     (const long long*)c->t, k.lr, k.beta1, c->wimg,
                                                                     ema, c->wimg_ema, k.ema_alpha);
  else
    k_shampoo_update<0><<<net.n_mats, kShThreads, smem_update, st>>>(net, c->img, c->w, c->m, c->sh_roots, c->sh_anorm,
                                                                     (const long long*)c->t, k.lr, k.beta1, c->wimg,
                                                                     ema, c->wimg_ema, k.ema_alpha);
  return cudaGetLastError();
}

}  // namespace nrc
