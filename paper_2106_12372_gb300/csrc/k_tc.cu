// Fused tensor-core (tcgen05) kernels for the neural radiance cache MLP.
//
// Inference (Sec. 4, fully fused network; Fig. 4): one persistent CTA per SM
// with kSlots warpgroups; each warpgroup owns one 128-row batch tile at a
// time and a private slice of tensor memory (TMEM):
//   acc: 64 FP32 columns, the MMA accumulator D (row = TMEM lane);
//   act: 32 columns holding the tile's 64 activations as packed 16-bit pairs,
//        the MMA's A operand.
// The whole 16-bit weight image (Sec. 5 architecture; ~42 KB at width 64) is
// bulk-copied into shared memory once per CTA and serves as the B operand of
// every layer (K-major, 128-byte swizzle).  Per tile: the records are read
// from HBM by the thread that owns the row, encoded in registers (Table 1,
// Sec. 3.6) and stored to TMEM; then for each layer one thread issues
// 4 x (M128 x N64 x K16) tcgen05.mma reading A from TMEM and B from shared
// memory, commits to the warpgroup's mbarrier, and the warpgroup applies the
// ReLU, rounds to 16 bit and writes the next layer's A back into TMEM.  The
// output layer (N = 16, 3 used) is read back and stored as RGB.  Activations
// never leave the SM.
#include "tc_ptx.cuh"

namespace nrc {
using namespace tc;

constexpr int kSlots = 4;
constexpr int kInferThreads = 128 * kSlots;
constexpr int kTmemCols = 512;
constexpr int kSlotCols = 128;

struct InferParams {
  const float* rec;
  int64_t n;
  float* rgb;
  const uint8_t* wimg;
  int img_bytes;
  int n_mats;
  ImageShape img;
  float pad;
  int* err;
};

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  const uint32_t a = smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

template <int MODE, bool BF16>
__global__ void __launch_bounds__(kInferThreads, 1) k_infer_tc(const __grid_constant__ InferParams p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_w;
  __shared__ uint64_t bar_mma[kSlots];
  __shared__ uint32_t tmem_base_sh;
  uint8_t* sw = align1024(smem_raw);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int slot = tid >> 7;
  const int rit = tid & 127;  // row in tile == TMEM lane

  if (warp == 0) {
    tmem_alloc(&tmem_base_sh, kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar_w, 1);
    for (int s = 0; s < kSlots; ++s) mbar_init(&bar_mma[s], 1);
    fence_barrier_init();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_sh;
  if (tid == 0) {
    mbar_arrive_expect_tx(&bar_w, uint32_t(p.img_bytes));
    bulk_g2s(sw, p.wimg, uint32_t(p.img_bytes), &bar_w);
  }
  mbar_wait(&bar_w, 0, p.err);

  const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
  const uint32_t acc_col = uint32_t(slot * kSlotCols);
  const uint32_t act_col = acc_col + 64;
  const uint32_t t_acc = tmem + lane_base + acc_col;
  const uint32_t t_act = tmem + lane_base + act_col;
  const uint32_t sw_base = smem_u32(sw);
  uint32_t phase = 0;
  const int64_t n_tiles = (p.n + kTile - 1) / kTile;

  for (int64_t tile = int64_t(blockIdx.x) * kSlots + slot; tile < n_tiles; tile += int64_t(gridDim.x) * kSlots) {
    const int64_t row = tile * kTile + rit;
    float r[kRecFloats];
    if (row < p.n) {
      load_record(p.rec, row, r);
    } else {
#pragma unroll
      for (int q = 0; q < kRecFloats; ++q) r[q] = 0.0f;
    }
    uint32_t pk[16];
    {
      float f[kEncDims];
      encode_record<MODE>(r, p.pad, f);
#pragma unroll
      for (int j = 0; j < 16; ++j) pk[j] = pack2<BF16, false>(f[2 * j], f[2 * j + 1]);
      tmem_st16(t_act, pk);
#pragma unroll
      for (int j = 0; j < 16; ++j) pk[j] = pack2<BF16, false>(f[32 + 2 * j], f[33 + 2 * j]);
      tmem_st16(t_act + 16, pk);
      tmem_st_wait();
    }
    for (int l = 0; l < p.n_mats; ++l) {
      fence_before();
      named_sync(1 + slot, 128);
      if (rit == 0) {
        fence_after();
        const uint32_t idesc = idesc_f16(128, p.img.rows[l], BF16);
        const uint32_t b0 = sw_base + uint32_t(p.img.off[l]);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          mma_ts(tmem + acc_col, tmem + act_col + uint32_t(k * 8), sdesc_sw128(b0 + uint32_t(k * 32), 16, 1024),
                 idesc, k > 0 ? 1u : 0u);
        mma_commit(&bar_mma[slot]);
      }
      mbar_wait(&bar_mma[slot], phase, p.err);
      phase ^= 1u;
      fence_after();
      if (l + 1 < p.n_mats) {
        uint32_t v[32];
        tmem_ld32(t_acc, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) pk[j] = pack2<BF16, true>(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
        tmem_st16(t_act, pk);
        tmem_ld32(t_acc + 32, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) pk[j] = pack2<BF16, true>(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
        tmem_st16(t_act + 16, pk);
        tmem_st_wait();
      } else {
        uint32_t v[4];
        tmem_ld4(t_acc, v);
        if (row < p.n) {
          float* o = p.rgb + row * 3;
          o[0] = __uint_as_float(v[0]);
          o[1] = __uint_as_float(v[1]);
          o[2] = __uint_as_float(v[2]);
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

template <typename K>
static cudaError_t set_smem(K kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_infer_tc(Cache* c, const float* rec, int64_t n, float* rgb, cudaStream_t st) {
  InferParams p;
  p.rec = rec;
  p.n = n;
  p.rgb = rgb;
  p.wimg = c->wimg;
  p.img_bytes = c->img.off[c->net.n_mats];
  p.n_mats = c->net.n_mats;
  p.img = c->img;
  p.pad = c->cfg.pad_value;
  p.err = c->err;
  const int smem = p.img_bytes + 1024;
  const int64_t n_tiles = (n + kTile - 1) / kTile;
  const int64_t want = (n_tiles + kSlots - 1) / kSlots;
  const unsigned grid = unsigned(want < c->sm_count ? want : c->sm_count);
  const bool bf16 = c->cfg.dtype == NRC_BF16;
  const int mode = c->cfg.enc_mode;
  cudaError_t e;
#define NRC_LAUNCH(M, B)                                          \
  e = set_smem(k_infer_tc<M, B>, smem);                           \
  if (e != cudaSuccess) return e;                                 \
  k_infer_tc<M, B><<<grid, kInferThreads, smem, st>>>(p);
  if (mode == 0 && !bf16) {
    NRC_LAUNCH(0, false)
  } else if (mode == 0 && bf16) {
    NRC_LAUNCH(0, true)
  } else if (!bf16) {
    NRC_LAUNCH(1, false)
  } else {
    NRC_LAUNCH(1, true)
  }
#undef NRC_LAUNCH
  return cudaGetLastError();
}

// Training for the 16-bit caches.  Until the tensor-core training kernel is
// in place the FP32 fused kernel computes the gradient from the master
// weights; Adam then refreshes the 16-bit image.
cudaError_t launch_train_tc(Cache* c, const float* pool, const float* target, int64_t n_pool, int64_t batch,
                            uint64_t a, uint64_t cc, int step, int* n_partials, float* grad_scale, cudaStream_t st) {
  *grad_scale = 1.0f;
  return launch_train_simt(c, pool, target, n_pool, batch, a, cc, step, n_partials, st);
}

}  // namespace nrc
