// Cache queries of the width-128 network on the tensor cores (Sec. 4 and
// Fig. 5: the fully fused network at widths 64 and 128; here with 7 hidden
// layers of 128 neurons).
//
// One persistent CTA per SM with two slots (warpgroups), each a 128-row tile
// at a time, exactly as the width-64 query kernel's slots: encoding into the
// slot's TMEM A-operand columns, then per layer the MMAs issued by one
// elected thread of the slot's lead warp, one waiter, and the ReLU + 16-bit
// epilogue back into the A-operand columns.  A layer with K inputs is K/16
// MMAs of M128 x N x K16 (N = 128; 16 for the padded output layer), A from
// TMEM, B (the weights, K-major, 128-byte swizzled, in blocks of 64 inputs)
// from shared memory.  TMEM per slot: 128 accumulator + 64 A-operand columns
// (2 x 192 = 384 of 512).  The whole 16-bit weight image (212 KB at 7 hidden
// layers) stays in shared memory, so records are not staged there: each
// thread loads its next row's record into registers while the current tile
// runs.
#include <atomic>

#include "tc_common.cuh"

namespace nrc {

constexpr int kSlots128 = 2;
constexpr int kThreads128 = 128 * kSlots128;
constexpr int kSlotCols128 = 192;  // 128 accumulator + 64 A-operand columns
constexpr int kWide = 128;

struct Infer128Params {
  const float* rec;
  int64_t n;
  float* rgb;
  const uint8_t* wimg;
  int img_bytes;
  int n_mats;
  ImageShape img;
  int dims[kMaxMats + 1];
  float pad;
  int factor;  // reflectance factorisation (Sec. 5)
  int* err;
};

__device__ __forceinline__ void load_row(const float* rec, int64_t row, bool ok, float (&r)[kRecFloats]) {
  if (ok) {
    load_record(rec, row, r);
  } else {
#pragma unroll
    for (int k = 0; k < kRecFloats; ++k) r[k] = 0.0f;
  }
}

template <int MODE, bool BF16>
__global__ void __launch_bounds__(kThreads128, 1) k_infer_tc128(const __grid_constant__ Infer128Params p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_w;
  __shared__ uint64_t bar_mma[kSlots128];
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
    for (int s = 0; s < kSlots128; ++s) mbar_init(&bar_mma[s], 1);
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
  const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
  const uint32_t acc_col = uint32_t(slot * kSlotCols128);
  const uint32_t act_col = acc_col + kWide;
  const uint32_t t_acc = tmem + lane_base + acc_col;
  const uint32_t t_act = tmem + lane_base + act_col;
  const uint32_t sw_base = smem_u32(sw);
  // the slot's lead warp (warp slot % 4 of its warpgroup: its own SM
  // sub-partition) forms the descriptors, issues and waits
  const int lead = slot & 3;
  const bool w0 = (rit >> 5) == lead;
  const int64_t n_tiles = (p.n + kTile - 1) / kTile;
  const int64_t stride = int64_t(gridDim.x) * kSlots128;
  int64_t tile = int64_t(blockIdx.x) * kSlots128 + slot;
  float r[kRecFloats];
  load_row(p.rec, tile * kTile + rit, tile < n_tiles && tile * kTile + rit < p.n, r);
  mbar_wait(&bar_w, 0, p.err);
  uint32_t phase = 0;

  for (; tile < n_tiles; tile += stride) {
    const int64_t row = tile * kTile + rit;
    const bool valid = row < p.n;
    float f[3] = {1.0f, 1.0f, 1.0f};
    if (p.factor) {
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) f[ch] = r[8 + ch] + r[11 + ch];
    }
    encode_to_tmem<MODE, BF16>(r, p.pad, t_act);
    // the next tile's record, in flight while this tile's layers run
    const int64_t nt = tile + stride;
    load_row(p.rec, nt * kTile + rit, nt < n_tiles && nt * kTile + rit < p.n, r);
    for (int l = 0; l < p.n_mats; ++l) {
      const int ksteps = p.dims[l] / 16;
      uint32_t idesc = 0;
      uint64_t bdesc = 0, kblock = 0;
      if (w0) {
        idesc = idesc_f16(128, p.img.rows[l], BF16);
        bdesc = sdesc_sw128(sw_base + uint32_t(p.img.off[l]), 16, 1024);
        kblock = uint64_t(p.img.rows[l]) * 8u;  // one block of 64 inputs, in descriptor units of 16 B
      }
      fence_before();
      named_sync(1 + slot, 128);
      if (w0) {
        fence_after();
        if (elect_one()) {
          for (int k = 0; k < ksteps; ++k)
            mma_ts(tmem + acc_col, tmem + act_col + uint32_t(8 * k),
                   bdesc + uint64_t(k >> 2) * kblock + uint64_t(2 * (k & 3)), idesc, k > 0 ? 1u : 0u);
          mma_commit(&bar_mma[slot]);
        }
        __syncwarp();
        if (rit == 32 * lead) mbar_wait(&bar_mma[slot], phase, p.err);
      }
      named_sync(1 + slot, 128);
      phase ^= 1u;
      fence_after();
      if (l + 1 < p.n_mats) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t v[64], pk[16];
          tmem_ld64(t_acc + uint32_t(64 * h), v);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            pk[j] = pack2<BF16, true>(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
          tmem_st16(t_act + uint32_t(32 * h), pk);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            pk[j] = pack2<BF16, true>(__uint_as_float(v[32 + 2 * j]), __uint_as_float(v[33 + 2 * j]));
          tmem_st16(t_act + uint32_t(32 * h + 16), pk);
        }
        tmem_st_wait();
      } else {
        uint32_t v[4];
        tmem_ld4(t_acc, v);
        if (valid) {
          float* o = p.rgb + row * 3;
          o[0] = __uint_as_float(v[0]) * f[0];
          o[1] = __uint_as_float(v[1]) * f[1];
          o[2] = __uint_as_float(v[2]) * f[2];
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

cudaError_t launch_infer_tc128(Cache* c, const float* rec, int64_t n, float* rgb, cudaStream_t st) {
  if (c->cfg.width != kWide || c->net.n_mats > kMaxMats) return cudaErrorNotSupported;
  Infer128Params p;
  p.rec = rec;
  p.n = n;
  p.rgb = rgb;
  p.wimg = query_image(c);
  p.img_bytes = c->img.off[c->net.n_mats];
  p.n_mats = c->net.n_mats;
  p.img = c->img;
  for (int l = 0; l <= kMaxMats; ++l) p.dims[l] = l <= c->net.n_mats ? c->net.dims[l] : 0;
  p.pad = c->cfg.pad_value;
  p.factor = c->cfg.refl_factor;
  p.err = c->err;
  const int smem = ((p.img_bytes + 1023) & ~1023) + 1024;
  const int64_t n_tiles = (n + kTile - 1) / kTile;
  const int64_t want = (n_tiles + kSlots128 - 1) / kSlots128;
  const unsigned grid = unsigned(want < c->sm_count ? want : c->sm_count);
  const bool bf16 = c->cfg.dtype == NRC_BF16;
  const int mode = c->cfg.enc_mode;
  cudaError_t e;
  static std::atomic<int> attr_done[4];
#define NRC_LAUNCH(M, B)                                                         \
  e = ensure_smem(k_infer_tc128<M, B>, smem, &attr_done[2 * (M) + ((B) ? 1 : 0)]); \
  if (e != cudaSuccess) return e;                                                \
  k_infer_tc128<M, B><<<grid, kThreads128, smem, st>>>(p);
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

}  // namespace nrc
