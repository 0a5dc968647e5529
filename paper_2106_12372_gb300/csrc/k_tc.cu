// Fused tensor-core (tcgen05) kernels for the neural radiance cache MLP.
//
// Inference (Sec. 4, fully fused network; Fig. 4): one persistent CTA per SM
// with kSlots = 5 warpgroups; each warpgroup owns one 128-row batch tile at a
// time and a private slice of tensor memory (TMEM):
//   acc: 64 FP32 columns, the MMA accumulator D (row = TMEM lane);
//   act: 32 columns holding the tile's 64 activations as packed 16-bit pairs,
//        the MMA's A operand.
// The whole 16-bit weight image (Sec. 5 architecture; ~42 KB at width 64) is
// bulk-copied into shared memory once per CTA and serves as the B operand of
// every layer (K-major, 128-byte swizzle).  Per tile: each thread's 64-byte
// record was prefetched into shared memory with cp.async while the previous
// tile ran (double-buffered, 16-byte chunks rotated so that the row reads are
// free of bank conflicts); it is encoded in registers (Table 1, Sec. 3.6) and
// stored to TMEM; then for each layer one thread issues 4 x (M128 x N64 x
// K16) tcgen05.mma reading A from TMEM and B from shared memory, commits to
// the warpgroup's mbarrier, and the warpgroup applies the ReLU, rounds to 16
// bit and writes the next layer's A back into TMEM.  The output layer
// (N = 16, 3 used) is read back and stored as RGB.  Activations never leave
// the SM.
#include <cstring>

#include "tc_common.cuh"

namespace nrc {
using namespace tc;


struct InferParams {
  const float* rec;
  int64_t n;
  float* rgb;
  const uint8_t* wimg;
  int img_bytes;
  int n_mats;
  ImageShape img;
  float pad;
  int factor;  // reflectance factorisation (Sec. 5)
  int* err;
};

struct BatchInferParams {
  const BatchCache* caches;
  const BatchUnit* units;
  int n_units;
  unsigned* counter;      // work-unit counter, zero at launch
  const int* unit_off;    // static ranges: CTA b runs units unit_off[b] .. unit_off[b+1]-1 (null: the counter)
  int img_bytes;
  int n_mats;
  ImageShape img;
  float pad;
  int factor;
  int* err;
};


template <int MODE, bool BF16>
__global__ void __launch_bounds__(kInferThreads, 1) k_infer_tc(const __grid_constant__ InferParams p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_w;
  __shared__ uint64_t bar_mma[kSlots];
  __shared__ uint32_t tmem_base_sh;
  uint8_t* sw = align1024(smem_raw);
  uint8_t* recs = sw + ((p.img_bytes + 1023) & ~1023);  // [kSlots][2][128 rows][64 B]
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

  const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
  SlotTmem st;
  st.tmem = tmem;
  st.acc_col = uint32_t(slot * kSlotCols);
  st.act_col = st.acc_col + 64;
  st.t_acc = tmem + lane_base + st.acc_col;
  st.t_act = tmem + lane_base + st.act_col;
  const uint32_t sw_base = smem_u32(sw);
  const int64_t n_tiles = (p.n + kTile - 1) / kTile;
  const int64_t stride = int64_t(gridDim.x) * kSlots;
  RecStage rs;
  rs.row0 = smem_u32(recs) + uint32_t(slot * 2 * 8192 + rit * 64);
  rs.p = recs + slot * 2 * 8192 + rit * 64;
  rs.rot = uint32_t((rit >> 1) & 3);
  auto prefetch = [&](int64_t t, int b) {
    const int64_t row = t * kTile + rit;
    rs.fetch(p.rec, row, t < n_tiles && row < p.n, b);
  };
  int64_t tile = int64_t(blockIdx.x) * kSlots + slot;
  int buf = 0;
  prefetch(tile, buf);
  mbar_wait(&bar_w, 0, p.err);
  uint32_t phase = 0;

  for (; tile < n_tiles; tile += stride) {
    const int64_t row = tile * kTile + rit;
    prefetch(tile + stride, buf ^ 1);
    cp_async_wait<1>();  // this tile's record has landed (only this thread reads it)
    float r[kRecFloats];
    rs.read(buf, r);
    // the staged record stays in place until the next tile's prefetch, so the
    // output epilogue can read its albedos again there
    const uint8_t* fac_row = p.factor ? rs.p + buf * 8192 : nullptr;
    buf ^= 1;
    encode_to_tmem<MODE, BF16>(r, p.pad, st.t_act);
    tile_layers<BF16>(p.img, p.n_mats, st, sw_base, slot, rit, &bar_mma[slot], phase, p.err,
                      row < p.n ? p.rgb + row * 3 : nullptr, fac_row, rs.rot);
  }
  cp_async_wait<0>();
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// Batched inference over several caches (one persistent launch): the work is
// a list of units, each a run of up to `unit_tiles` 128-row tiles of one
// cache; CTAs take units from a device counter.  A CTA reloads the weight
// image only when its next unit belongs to another cache; within a unit the
// slots take the tiles round-robin exactly as k_infer_tc does, so every row's
// arithmetic is the same as in a single-cache launch.
template <int MODE, bool BF16>
__global__ void __launch_bounds__(kInferThreads, 1) k_infer_batched(const __grid_constant__ BatchInferParams p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_w;
  __shared__ uint64_t bar_mma[kSlots];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int unit_sh;
  uint8_t* sw = align1024(smem_raw);
  uint8_t* recs = sw + ((p.img_bytes + 1023) & ~1023);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int slot = tid >> 7;
  const int rit = tid & 127;
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
  const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
  SlotTmem st;
  st.tmem = tmem;
  st.acc_col = uint32_t(slot * kSlotCols);
  st.act_col = st.acc_col + 64;
  st.t_acc = tmem + lane_base + st.acc_col;
  st.t_act = tmem + lane_base + st.act_col;
  const uint32_t sw_base = smem_u32(sw);
  RecStage rs;
  rs.row0 = smem_u32(recs) + uint32_t(slot * 2 * 8192 + rit * 64);
  rs.p = recs + slot * 2 * 8192 + rit * 64;
  rs.rot = uint32_t((rit >> 1) & 3);
  int cur = -1;
  uint32_t wphase = 0, phase = 0;
  // one unit's tiles, interleaved over the slots; the weight image is loaded
  // when the unit's cache differs from the last one (every slot is done with
  // the previous unit then: the callers synchronise the CTA first)
  auto run_unit = [&](const BatchUnit& U) {
    const BatchCache C = p.caches[U.cache];
    if (U.cache != cur) {
      if (tid == 0) {
        mbar_arrive_expect_tx(&bar_w, uint32_t(p.img_bytes));
        bulk_g2s(sw, C.wimg, uint32_t(p.img_bytes), &bar_w);
      }
      mbar_wait(&bar_w, wphase, p.err);
      wphase ^= 1u;
      cur = U.cache;
    }
    int buf = 0;
    int64_t tile = U.tile_begin + slot;
    auto prefetch = [&](int64_t t, int b) {
      const int64_t row = t * kTile + rit;
      rs.fetch(C.rec, row, t < U.tile_end && row < C.n, b);
    };
    prefetch(tile, buf);
    for (; tile < U.tile_end; tile += kSlots) {
      const int64_t row = tile * kTile + rit;
      prefetch(tile + kSlots, buf ^ 1);
      cp_async_wait<1>();
      float r[kRecFloats];
      rs.read(buf, r);
      const uint8_t* fac_row = p.factor ? rs.p + buf * 8192 : nullptr;
      buf ^= 1;
      encode_to_tmem<MODE, BF16>(r, p.pad, st.t_act);
      tile_layers<BF16>(p.img, p.n_mats, st, sw_base, slot, rit, &bar_mma[slot], phase, p.err,
                        row < C.n ? C.rgb + row * 3 : nullptr, fac_row, rs.rot);
    }
    cp_async_wait<0>();
  };
  if (p.unit_off) {
    // static: this CTA's contiguous range of the tiles, cache after cache
    // (consecutive units of a CTA belong to different caches)
    const int u1 = p.unit_off[blockIdx.x + 1];
    for (int u = p.unit_off[blockIdx.x]; u < u1; ++u) {
      __syncthreads();  // every slot is done with the previous unit (its MMAs completed)
      run_unit(p.units[u]);
    }
  } else {
    while (true) {
      __syncthreads();  // every slot is done with the previous unit (its MMAs completed)
      if (tid == 0) unit_sh = int(atomicAdd(p.counter, 1u));
      __syncthreads();
      const int u = unit_sh;
      if (u >= p.n_units) break;
      run_unit(p.units[u]);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ------------------------------------------------------------ FP8 queries
// The query kernel with E4M3 operands (dtype NRC_FP8): the same slots, record
// staging and TMEM columns as k_infer_tc, with 16 of the 32 activation columns
// used (4 E4M3 values per column) and two K = 32 MMAs per layer.  Scales (all
// powers of two, so undone exactly): weights of matrix l by s_l (from its
// amax, in the image), the encoded inputs by 128, and each row's hidden
// activations by a factor c from that row's amax that puts it in [128, 256);
// the thread keeps 1/(product of its row's scales) to rescale the output.
// Byte offset of matrix l in the E4M3 image: each matrix takes half its bytes
// in the 16-bit image (rows padded to 16, 64 inputs), rounded up to 1 KB.
__host__ __device__ __forceinline__ int img8_offset_of(const ImageShape& img, int l) {
  int off = 0;
  for (int j = 0; j < l; ++j) off += ((img.off[j + 1] - img.off[j]) / 2 + 1023) & ~1023;
  return off;
}

__device__ __forceinline__ uint32_t sw64_offset(uint32_t n, uint32_t k) {
  return (n >> 3) * 512u + (n & 7u) * 64u + ((((k >> 4) ^ (n >> 1)) & 3u) << 4) + (k & 15u);
}

// 2^(7 - floor(log2 a)) as (scale, 1/scale) for a > 0 normal; (1, 1) for a == 0
__device__ __forceinline__ void pow2_scale(float a, float& s, float& inv) {
  const int eb = int((__float_as_uint(a) >> 23) & 0xFFu);
  if (eb == 0) {
    s = inv = 1.0f;
    return;
  }
  const int sb = min(254, max(1, 261 - eb));
  s = __uint_as_float(uint32_t(sb) << 23);
  inv = __uint_as_float(uint32_t(254 - sb) << 23);
}

// One block per matrix: amax -> scale -> E4M3 image (rows padded with zeros).
__global__ void k_build_image_fp8(const float* __restrict__ w, const __grid_constant__ NetShape net,
                                  const __grid_constant__ ImageShape img, uint8_t* __restrict__ img8, int img8_bytes) {
  __shared__ float red[8];
  const int l = blockIdx.x;
  const int n_out = net.dims[l + 1], n_in = net.dims[l];
  const float* wl = w + net.w_off[l];
  float a = 0.0f;
  for (int e = threadIdx.x; e < n_out * n_in; e += blockDim.x) a = fmaxf(a, fabsf(wl[e]));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a = fmaxf(a, __shfl_down_sync(0xffffffffu, a, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  a = 0.0f;
  for (int k = 0; k < int(blockDim.x >> 5); ++k) a = fmaxf(a, red[k]);
  float s, inv;
  pow2_scale(a, s, inv);
  uint8_t* dst = img8 + img8_offset_of(img, l);
  for (int e = threadIdx.x; e < img.rows[l] * n_in; e += blockDim.x) {
    const int o = e / n_in, i = e % n_in;
    const float x = o < n_out ? wl[o * n_in + i] * s : 0.0f;
    dst[sw64_offset(o, i)] = uint8_t(pack_e4m3x2<false>(x, 0.0f) & 0xFFu);
  }
  if (threadIdx.x == 0) reinterpret_cast<float*>(img8 + img8_bytes)[l] = inv;
}

template <int MODE>
__global__ void __launch_bounds__(kInferThreads, 1) k_infer_fp8(const __grid_constant__ InferParams p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_w;
  __shared__ uint64_t bar_mma[kSlots];
  __shared__ uint32_t tmem_base_sh;
  uint8_t* sw = align1024(smem_raw);
  const int img_alloc = (p.img_bytes + kImg8ScaleBytes + 1023) & ~1023;
  uint8_t* recs = sw + img_alloc;
  const float* inv_sw = reinterpret_cast<const float*>(sw + p.img_bytes);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int slot = tid >> 7;
  const int rit = tid & 127;
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
    const uint32_t bytes = uint32_t(p.img_bytes) + uint32_t(kImg8ScaleBytes);
    mbar_arrive_expect_tx(&bar_w, bytes);
    bulk_g2s(sw, p.wimg, bytes, &bar_w);
  }
  const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
  SlotTmem st;
  st.tmem = tmem;
  st.acc_col = uint32_t(slot * kSlotCols);
  st.act_col = st.acc_col + 64;
  st.t_acc = tmem + lane_base + st.acc_col;
  st.t_act = tmem + lane_base + st.act_col;
  const uint32_t sw_base = smem_u32(sw);
  const int64_t n_tiles = (p.n + kTile - 1) / kTile;
  const int64_t stride = int64_t(gridDim.x) * kSlots;
  RecStage rs;
  rs.row0 = smem_u32(recs) + uint32_t(slot * 2 * 8192 + rit * 64);
  rs.p = recs + slot * 2 * 8192 + rit * 64;
  rs.rot = uint32_t((rit >> 1) & 3);
  auto prefetch = [&](int64_t t, int b) {
    const int64_t row = t * kTile + rit;
    rs.fetch(p.rec, row, t < n_tiles && row < p.n, b);
  };
  int64_t tile = int64_t(blockIdx.x) * kSlots + slot;
  int buf = 0;
  prefetch(tile, buf);
  mbar_wait(&bar_w, 0, p.err);
  uint32_t phase = 0;
  for (; tile < n_tiles; tile += stride) {
    const int64_t row = tile * kTile + rit;
    prefetch(tile + stride, buf ^ 1);
    cp_async_wait<1>();
    float r[kRecFloats];
    rs.read(buf, r);
    const uint8_t* fac_row = p.factor ? rs.p + buf * 8192 : nullptr;
    buf ^= 1;
    {  // encoded inputs times 128 (they lie in [-1, 1]) as E4M3
      float f[kEncDims];
      encode_record<MODE>(r, p.pad, f);
      uint32_t pk[16];
#pragma unroll
      for (int j = 0; j < kEncDims; j += 2) mul2(f[j], f[j + 1], 128.0f);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        pk[j] = pack_e4m3x2<false>(f[4 * j], f[4 * j + 1]) | (pack_e4m3x2<false>(f[4 * j + 2], f[4 * j + 3]) << 16);
      tmem_st16(st.t_act, pk);
      tmem_st_wait();
    }
    float inv_row = 1.0f / 128.0f;  // 1 / (the row's accumulated activation scale)
    for (int l = 0; l < p.n_mats; ++l) {
      fence_before();
      named_sync(1 + slot, 128);
      if ((rit >> 5) == (slot & 3)) {
        // the slot's lead warp (warp slot % 4, as in tile_layers) forms the
        // (warp-uniform) descriptor; one elected thread issues
        fence_after();
        const uint32_t idesc = idesc_e4m3(128, p.img.rows[l]);
        const uint64_t bd = sdesc_sw64(sw_base + uint32_t(img8_offset_of(p.img, l)), 512);
        if (elect_one()) {
#pragma unroll
          for (int k = 0; k < 2; ++k)
            mma_ts_f8(st.tmem + st.acc_col, st.tmem + st.act_col + uint32_t(k * 8), bd + uint64_t(2 * k), idesc,
                      k > 0 ? 1u : 0u);
          mma_commit(&bar_mma[slot]);
        }
        __syncwarp();
      }
      if (rit == 32 * (slot & 3)) mbar_wait(&bar_mma[slot], phase, p.err);
      named_sync(1 + slot, 128);
      phase ^= 1u;
      fence_after();
      inv_row *= inv_sw[l];  // the accumulator now carries the row scale times s_l
      if (l + 1 < p.n_mats) {
        uint32_t v[64], pk[16];
        tmem_ld64(st.t_acc, v);
        float x[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) x[j] = __uint_as_float(v[j]);
        // the row's amax (of the ReLU'd values) by a tree of three-input maxima
        float m[22], q[8];
#pragma unroll
        for (int j = 0; j < 21; ++j) m[j] = max3(x[3 * j], x[3 * j + 1], x[3 * j + 2]);
        m[21] = fmaxf(x[63], 0.0f);
#pragma unroll
        for (int j = 0; j < 7; ++j) q[j] = max3(m[3 * j], m[3 * j + 1], m[3 * j + 2]);
        q[7] = m[21];
        const float amax = max3(max3(q[0], q[1], q[2]), max3(q[3], q[4], q[5]), fmaxf(q[6], q[7]));
        float c, inv_c;
        pow2_scale(amax, c, inv_c);
#pragma unroll
        for (int j = 0; j < 64; j += 2) mul2(x[j], x[j + 1], c);
#pragma unroll
        for (int j = 0; j < 16; ++j)
          pk[j] = pack_e4m3x2<true>(x[4 * j], x[4 * j + 1]) | (pack_e4m3x2<true>(x[4 * j + 2], x[4 * j + 3]) << 16);
        tmem_st16(st.t_act, pk);
        tmem_st_wait();
        inv_row *= inv_c;
      } else {
        uint32_t v[4];
        tmem_ld4(st.t_acc, v);
        if (row < p.n) {
          float y0 = __uint_as_float(v[0]) * inv_row, y1 = __uint_as_float(v[1]) * inv_row,
                y2 = __uint_as_float(v[2]) * inv_row;
          if (fac_row) {
            float f[3];
            staged_albedo_sum(fac_row, rs.rot, f);
            y0 *= f[0];
            y1 *= f[1];
            y2 *= f[2];
          }
          float* o = p.rgb + row * 3;
          o[0] = y0;
          o[1] = y1;
          o[2] = y2;
        }
      }
    }
  }
  cp_async_wait<0>();
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// Fault-injection probe: one thread waits, through the kernels' bounded wait,
// on an mbarrier that nothing arrives at; after limit_ns it sets kErrTimeout
// in *err and the kernel returns (the context stays usable).
__global__ void k_wait_probe(int* err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
    mbar_wait(&bar, 0, err, limit_ns);
  }
}

cudaError_t launch_wait_probe(int* err, unsigned long long limit_ns, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(err, limit_ns);
  return cudaGetLastError();
}

cudaError_t launch_infer_tc(Cache* c, const float* rec, int64_t n, float* rgb, cudaStream_t st, const uint8_t* image) {
  InferParams p;
  p.rec = rec;
  p.n = n;
  p.rgb = rgb;
  p.wimg = image ? image : query_image(c);
  p.img_bytes = c->img.off[c->net.n_mats];
  p.n_mats = c->net.n_mats;
  p.img = c->img;
  p.pad = c->cfg.pad_value;
  p.factor = c->cfg.refl_factor;
  p.err = c->err;
  const int smem = ((p.img_bytes + 1023) & ~1023) + kSlots * 2 * 8192 + 1024;
  const int64_t n_tiles = (n + kTile - 1) / kTile;
  const int64_t want = (n_tiles + kSlots - 1) / kSlots;
  const unsigned grid = unsigned(want < c->sm_count ? want : c->sm_count);
  const bool bf16 = c->cfg.dtype == NRC_BF16;
  const int mode = c->cfg.enc_mode;
  cudaError_t e;
  static std::atomic<int> attr_done[4];
#define NRC_LAUNCH(M, B)                                                   \
  e = ensure_smem(k_infer_tc<M, B>, smem, &attr_done[2 * (M) + ((B) ? 1 : 0)]); \
  if (e != cudaSuccess) return e;                                          \
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

cudaError_t launch_infer_batched(const Cache* proto, const BatchCache* caches, const BatchUnit* units, int n_units,
                                 unsigned* counter, int grid, cudaStream_t st, const int* unit_off) {
  BatchInferParams p;
  p.caches = caches;
  p.units = units;
  p.n_units = n_units;
  p.counter = counter;
  p.unit_off = unit_off;
  p.img_bytes = proto->img.off[proto->net.n_mats];
  p.n_mats = proto->net.n_mats;
  p.img = proto->img;
  p.pad = proto->cfg.pad_value;
  p.factor = proto->cfg.refl_factor;
  p.err = proto->err;
  const int smem = ((p.img_bytes + 1023) & ~1023) + kSlots * 2 * 8192 + 1024;
  const bool bf16 = proto->cfg.dtype == NRC_BF16;
  const int mode = proto->cfg.enc_mode;
  cudaError_t e = unit_off ? cudaSuccess : cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  static std::atomic<int> attr_done[4];
#define NRC_LAUNCH(M, B)                                                        \
  e = ensure_smem(k_infer_batched<M, B>, smem, &attr_done[2 * (M) + ((B) ? 1 : 0)]); \
  if (e != cudaSuccess) return e;                                               \
  k_infer_batched<M, B><<<unsigned(grid), kInferThreads, smem, st>>>(p);
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

// ------------------------------------------------------------- training
// Fused training step on the tensor cores (Sec. 4, training the fully fused
// network; Eq. 5; the weight-gradient contraction the paper leaves to a
// split-k GEMM).  Two warpgroups per CTA work on one 128-row batch tile at a
// time: thread (h, r) owns gathered record r (Sec. 3.5 shuffle) and column
// half h (features / neurons 32h .. 32h+31) of every epilogue.
//  forward : H_{l+1} = ReLU(W_l H_l) as in inference; every H_l is also kept
//            in shared memory (16-bit, 128-byte swizzled rows): it is the B
//            operand of the weight gradient and, being post-ReLU, its nonzero
//            entries are the ReLU mask [Z_l > 0] of the backward pass;
//  loss    : relative L2 (Eq. 5) in FP32; g' = 2 (y - t) / den is passed on
//            without the 1/(3N) factor (applied by the Adam kernel) so that
//            16-bit deltas stay in range;
//  backward: per layer two MMAs issued together --
//            dW_l += delta_{l+1}^T H_l  (M = 128 with rows 64..127 a duplicate
//            that is never read, N = 64, K = 128 batch rows; both operands in
//            shared memory, MN-major), accumulated in TMEM across the CTA's
//            tiles; and, for l >= 1, delta_l = (delta_{l+1} W_l) * mask_l
//            (A = delta in TMEM, B = the same weight image read MN-major).
// At the end each CTA writes its dW (FP32) and loss sum to its own partial.
constexpr int kTrainThreads = 256;
constexpr int kTrainMaxMats = 6;  // TMEM: acc 64 + act 32 + 6 x 64 dW columns <= 512

struct TrainParams {
  const TrainJob* jobs;  // per-CTA work of a batched step over several caches; null: one cache (fields below)
  const float* pool;
  const float* target;
  int64_t n_pool;
  int64_t batch;
  uint64_t a, c;
  int step;
  int n_mats;
  ImageShape img;
  int img_bytes;
  int w_off[kMaxMats + 1];
  int n_params;
  float pad;
  int loss_mode;
  float loss_eps;
  int factor;  // reflectance factorisation (Sec. 5)
  float inv3n;
  float* partials;
  long long* t_ctr;
  const uint8_t* wimg;
  int* err;
};


template <int MODE, bool BF16>
__global__ void __launch_bounds__(kTrainThreads, 1) k_train_tc(const __grid_constant__ TrainParams p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_w, bar_mma;
  __shared__ uint32_t tmem_base_sh;
  __shared__ float red[4];
  uint8_t* sw = align1024(smem_raw);                 // weight image
  uint8_t* Hs = sw + ((p.img_bytes + 1023) & ~1023); // n_mats x 16 KB
  uint8_t* Ds = Hs + p.n_mats * 16384;               // 2 x 16 KB (delta of layer l in buffer l % 2)
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int half = tid >> 7;  // column half of this thread
  const int r = tid & 127;    // row in tile == TMEM lane
  if (warp == 0) {
    tmem_alloc(&tmem_base_sh, kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar_w, 1);
    mbar_init(&bar_mma, 1);
    fence_barrier_init();
  }
  fence_before();
  __syncthreads();
  fence_after();
  pdl_launch_dependents();  // the Adam kernel that follows may be scheduled now; it waits for this grid
  const uint32_t tmem = tmem_base_sh;
  bool have_w = false;  // the weights are requested after the first tile's gather and encoding

  const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
  const uint32_t t_acc = tmem + lane_base + uint32_t(32 * half);        // my 32 accumulator columns
  const uint32_t t_act = tmem + lane_base + 64 + uint32_t(16 * half);   // my 16 packed activation columns
  const uint32_t sw_base = smem_u32(sw), hs_base = smem_u32(Hs), ds_base = smem_u32(Ds);
  auto ds_buf = [&](int l) { return Ds + (l & 1) * 16384; };
  const int L = p.n_mats;
  uint32_t phase = 0;
  float loss_acc = 0.0f;
  bool first = true;
  // this CTA's work: tiles tile_begin, tile_begin + tile_step, ... < tile_end of one cache
  TrainJob J;
  if (p.jobs) {
    J = p.jobs[blockIdx.x];
    if (J.seed) lcg_shuffle(J.n_pool, *J.seed, &J.a, &J.c);  // the frame seed lives on the device
  } else {
    J.pool = p.pool;
    J.target = p.target;
    J.n_pool = p.n_pool;
    J.batch = p.batch;
    J.a = p.a;
    J.c = p.c;
    J.seed = nullptr;
    J.step = p.step;
    J.tile_begin = int(blockIdx.x);
    J.tile_end = int((p.batch + kTile - 1) / kTile);
    J.tile_step = int(gridDim.x);
    J.wimg = p.wimg;
    J.partial = p.partials + size_t(blockIdx.x) * partial_stride(p.n_params);
    J.t_ctr = p.t_ctr;
    J.bump_t = blockIdx.x == 0;
    J.inv3n = p.inv3n;
  }

  // One dependent step: make this warpgroup pair's shared-memory and TMEM
  // writes visible, issue the MMAs (one thread), run `overlap` while they
  // execute, wait for them.
  auto mma_stage = [&](auto&& issue, auto&& overlap, bool commit) {
    fence_proxy_async_smem();
    fence_before();
    named_sync(1, kTrainThreads);
    if (warp == 0) {
      // warp 0 forms the (warp-uniform) descriptors together; one elected
      // thread issues
      fence_after();
      const bool lead = elect_one();
      issue(lead);
      if (commit && lead) mma_commit(&bar_mma);
      __syncwarp();
    }
    overlap();
    mbar_wait(&bar_mma, phase, p.err);
    phase ^= 1u;
    fence_after();
  };
  auto mma_sync_issue_wait = [&](auto&& issue) { mma_stage(issue, []() {}, true); };

  // Weight-gradient write-out, overlapped with the backward pass of the CTA's
  // last tile: once dW_l is final and H_l is no longer needed, the threads
  // owning TMEM lanes 0..63 stage dW_l into H_l's buffer (row o at o*64 floats,
  // 16-byte chunk c of each 128-byte half at chunk c ^ (o % 8): conflict-free),
  // and after the next barrier all 256 threads copy it to the CTA's partial
  // with coalesced 16-byte stores.
  float* P = J.partial;
  auto stage_dw = [&](int l) {
    if ((warp & 3) >= 2) return;
    const int o = r;
    const int dout = (l + 1 < L) ? 64 : kOutDims;
    uint32_t v[32];
    tmem_ld32(tmem + lane_base + 128 + uint32_t(l * 64 + 32 * half), v);
    if (o < dout) {
      float* seg = reinterpret_cast<float*>(Hs + l * 16384) + o * 64 + 32 * half;
#pragma unroll
      for (int c = 0; c < 8; ++c)
        *reinterpret_cast<float4*>(seg + ((c ^ (o & 7)) << 2)) =
            make_float4(__uint_as_float(v[4 * c]), __uint_as_float(v[4 * c + 1]), __uint_as_float(v[4 * c + 2]),
                        __uint_as_float(v[4 * c + 3]));
    }
  };
  auto write_dw = [&](int l) {
    const int dout = (l + 1 < L) ? 64 : kOutDims;
    const float* S = reinterpret_cast<const float*>(Hs + l * 16384);
    float4* Pl = reinterpret_cast<float4*>(P + p.w_off[l]);
    for (int e = tid; e < dout * 16; e += kTrainThreads) {
      const int o = e >> 4, c = e & 15;  // 16-byte chunk c of row o: inputs 4c .. 4c+3
      if (NRC_DCHECK(p.w_off[l] + 4 * e + 3 < p.n_params, p.err))
        Pl[e] = *reinterpret_cast<const float4*>(S + o * 64 + (c & 8) * 4 + (((c & 7) ^ (o & 7)) << 2));
    }
  };

  for (int64_t tile = J.tile_begin; tile < J.tile_end; tile += J.tile_step) {
    const int64_t j = tile * kTile + r;
    const bool valid = j < J.batch;
    float rec[kRecFloats], tg[3] = {0.f, 0.f, 0.f}, fac[3] = {1.f, 1.f, 1.f};
    if (valid) {
      const uint64_t i = uint64_t(J.step) * uint64_t(J.batch) + uint64_t(j);
      int64_t src = int64_t((J.a * i + J.c) % uint64_t(J.n_pool));
      if (!NRC_DCHECK(src >= 0 && src < J.n_pool, p.err)) src = 0;
      load_record(J.pool, src, rec);
      if (p.factor) {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) fac[ch] = rec[8 + ch] + rec[11 + ch];
      }
      if (half == 0) {
        tg[0] = __ldg(J.target + src * 3);
        tg[1] = __ldg(J.target + src * 3 + 1);
        tg[2] = __ldg(J.target + src * 3 + 2);
      }
    } else {
#pragma unroll
      for (int q = 0; q < kRecFloats; ++q) rec[q] = 0.0f;
    }
    uint32_t pk[16];
    {
      float f[32];
      encode_record_half<MODE>(rec, p.pad, half, f);
#pragma unroll
      for (int q = 0; q < 16; ++q) pk[q] = pack2<BF16, false>(f[2 * q], f[2 * q + 1]);
    }
    store_half_row_sw128(Hs, r, 4 * half, pk);
    tmem_st16(t_act, pk);
    tmem_st_wait();
    if (!have_w) {
      // Everything above reads only this step's inputs, so it may overlap the
      // previous step's Adam kernel; the weights, the step counter and the
      // partials belong to that step and are touched only after it completes.
      pdl_wait();
      if (tid == 0) {
        if (J.bump_t) *J.t_ctr += 1;  // Adam's step counter for the update that follows
        mbar_arrive_expect_tx(&bar_w, uint32_t(p.img_bytes));
        bulk_g2s(sw, J.wimg, uint32_t(p.img_bytes), &bar_w);
      }
      mbar_wait(&bar_w, 0, p.err);
      have_w = true;
    }

    // ------------------------------------------------------------ forward
    float y[3] = {0.f, 0.f, 0.f};
    for (int l = 0; l < L; ++l) {
      mma_sync_issue_wait([&](bool lead) {
        const uint32_t idesc = idesc_f16(128, p.img.rows[l], BF16);
        const uint64_t bd = sdesc_sw128(sw_base + uint32_t(p.img.off[l]), 16, 1024);
        if (lead) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            mma_ts(tmem + 0, tmem + 64 + uint32_t(k * 8), bd + uint64_t(2 * k), idesc, k > 0 ? 1u : 0u);
        }
      });
      if (l + 1 < L) {
        uint32_t v[32];
        tmem_ld32(t_acc, v);
#pragma unroll
        for (int q = 0; q < 16; ++q) pk[q] = pack2<BF16, true>(__uint_as_float(v[2 * q]), __uint_as_float(v[2 * q + 1]));
        store_half_row_sw128(Hs + (l + 1) * 16384, r, 4 * half, pk);
        tmem_st16(t_act, pk);
        tmem_st_wait();
      } else if (half == 0) {
        uint32_t v[4];
        tmem_ld4(t_acc, v);
        y[0] = __uint_as_float(v[0]);
        y[1] = __uint_as_float(v[1]);
        y[2] = __uint_as_float(v[2]);
      }
    }

    // --------------------------------------------------------------- loss
    // delta_L: 3 gradients, zero-padded to the 16 outputs of the padded layer
#pragma unroll
    for (int q = 0; q < 16; ++q) pk[q] = 0u;
    if (half == 0) {
      // factorisation: the loss sees y * f; the gradient reaching the network is times f
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) y[ch] *= fac[ch];
      const float lum = 0.2126f * y[0] + 0.7152f * y[1] + 0.0722f * y[2];
      float lr = 0.0f, g[3];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float den = (p.loss_mode == NRC_LOSS_LUMINANCE ? lum * lum : y[ch] * y[ch]) + p.loss_eps;
        const float inv = 1.0f / den;
        const float diff = y[ch] - tg[ch];
        lr = fmaf(diff * diff, inv, lr);
        g[ch] = valid ? fminf(fmaxf(2.0f * diff * inv * fac[ch], -60000.0f), 60000.0f) : 0.0f;
      }
      loss_acc += valid ? lr : 0.0f;
      pk[0] = pack2<BF16, false>(g[0], g[1]);
      pk[1] = pack2<BF16, false>(g[2], 0.0f);
    }
    store_half_row_sw128(ds_buf(L), r, 4 * half, pk);
    tmem_st16(t_act, pk);
    tmem_st_wait();

    // ----------------------------------------------------------- backward
    // Stage l issues delta_l = (delta_{l+1} W_l) first and commits it alone:
    // the epilogue waits for these 4 MMAs only, while dW_l (8 MMAs, issued
    // after the commit) finishes in the background.  MMAs complete in issue
    // order, so stage l's wait also covers every earlier stage's dW; dW_l
    // reads delta_{l+1} from buffer (l+1) % 2 while the epilogue writes
    // delta_l into the other one.
    const bool last_tile = tile + J.tile_step >= J.tile_end;
    for (int l = L - 1; l >= 0; --l) {
      const bool first_acc = first;
      mma_stage([&](bool lead) {
        if (l > 0) {
          // delta_l (pre-mask) = delta_{l+1} W_l: K = rows of W_l (64, or 16 for the output layer)
          const int K = p.img.rows[l];
          const uint32_t idd = idesc_f16(128, 64, BF16, false, true);
          const uint64_t bd = sdesc_sw128(sw_base + uint32_t(p.img.off[l]), 1024, 1024);
          if (lead) {
            for (int k = 0; k < K / 16; ++k)
              mma_ts(tmem + 0, tmem + 64 + uint32_t(k * 8), bd + uint64_t(128 * k), idd, k > 0 ? 1u : 0u);
            mma_commit(&bar_mma);
          }
        }
        // dW_l (+)= delta_{l+1}^T H_l over this tile's 128 rows
        const uint32_t idw = idesc_f16(128, 64, BF16, true, true);
        const uint32_t dcol = tmem + 128 + uint32_t(l * 64);
        const uint64_t hd = sdesc_sw128(hs_base + uint32_t(l * 16384), 1024, 1024);
        const uint64_t dd = sdesc_sw128(ds_base + uint32_t(((l + 1) & 1) * 16384), 0, 1024);
        if (lead) {
#pragma unroll
          for (int k = 0; k < 8; ++k)
            mma_ss(dcol, dd + uint64_t(128 * k), hd + uint64_t(128 * k), idw, (first_acc && k == 0) ? 0u : 1u);
          if (l == 0) mma_commit(&bar_mma);  // the last stage waits for dW_0 as well
        }
      }, [&]() {
        if (last_tile) {
          if (l + 2 < L) stage_dw(l + 2);  // dW_{l+2} final since the previous stage's wait
          if (l + 3 < L) write_dw(l + 3);  // staged during the previous stage, before this stage's barrier
        }
      }, false);
      if (l == 0) break;
      uint32_t v[32], h2[16];
      tmem_ld32(t_acc, v);
      load_half_row_sw128(Hs + l * 16384, r, 4 * half, h2);
#pragma unroll
      for (int q = 0; q < 16; ++q)
        pk[q] = masked_delta2<BF16>(__uint_as_float(v[2 * q]), __uint_as_float(v[2 * q + 1]), h2[q]);
      store_half_row_sw128(ds_buf(l), r, 4 * half, pk);
      tmem_st16(t_act, pk);
      tmem_st_wait();
    }
    first = false;
  }

  if (!have_w) pdl_wait();  // (a CTA without a tile still orders its partial after the predecessor)

  // ------------------------------------------- the rest of the CTA's partial
  if (!first) {
    // dW_1 and dW_0 are final after the last backward stage (no epilogue reads
    // H_1 or H_0 any more); dW_2 was staged during that stage
    if (L >= 2) stage_dw(1);
    stage_dw(0);
    __syncthreads();
    if (L >= 3) write_dw(2);
    if (L >= 2) write_dw(1);
    write_dw(0);
  } else {  // a CTA without a tile contributes zeros
    for (int e = tid; e < p.n_params; e += kTrainThreads) P[e] = 0.0f;
  }
  float s = loss_acc;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (half == 0 && (tid & 31) == 0) red[warp] = s;
  fence_before();
  __syncthreads();
  if (tid == 0) P[p.n_params] = ((red[0] + red[1]) + (red[2] + red[3])) * J.inv3n;
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

cudaError_t launch_train_tc(Cache* c, const float* pool, const float* target, int64_t n_pool, int64_t batch,
                            uint64_t a, uint64_t cc, int step, int* n_partials, float* grad_scale, cudaStream_t st) {
  if (c->net.n_mats > kTrainMaxMats) return cudaErrorNotSupported;
  TrainParams p;
  p.jobs = nullptr;
  p.pool = pool;
  p.target = target;
  p.n_pool = n_pool;
  p.batch = batch;
  p.a = a;
  p.c = cc;
  p.step = step;
  p.n_mats = c->net.n_mats;
  p.img = c->img;
  p.img_bytes = c->img.off[c->net.n_mats];
  for (int l = 0; l <= kMaxMats; ++l) p.w_off[l] = c->net.w_off[l];
  p.n_params = c->net.n_params;
  p.pad = c->cfg.pad_value;
  p.loss_mode = c->cfg.loss_mode;
  p.loss_eps = c->cfg.loss_eps;
  p.factor = c->cfg.refl_factor;
  p.inv3n = float(1.0 / (3.0 * double(batch)));
  p.t_ctr = c->t;
  p.wimg = c->wimg;
  p.err = c->err;
  const int64_t n_tiles = (batch + kTile - 1) / kTile;
  const int grid = int(n_tiles < c->sm_count ? n_tiles : c->sm_count);
  cudaError_t e = ensure_partials(c, grid);
  if (e != cudaSuccess) return e;
  p.partials = c->partials;
  const int smem = ((p.img_bytes + 1023) & ~1023) + p.n_mats * 16384 + 2 * 16384 + 1024;
  const bool bf16 = c->cfg.dtype == NRC_BF16;
  const int mode = c->cfg.enc_mode;
  static std::atomic<int> attr_done[4];
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(unsigned(grid));
  lc.blockDim = dim3(kTrainThreads);
  lc.dynamicSmemBytes = size_t(smem);
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
#define NRC_LAUNCH(M, B)                                                   \
  e = ensure_smem(k_train_tc<M, B>, smem, &attr_done[2 * (M) + ((B) ? 1 : 0)]); \
  if (e != cudaSuccess) return e;                                          \
  e = cudaLaunchKernelEx(&lc, k_train_tc<M, B>, p);                        \
  if (e != cudaSuccess) return e;
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
  *n_partials = grid;
  *grad_scale = p.inv3n;
  return cudaGetLastError();
}

// One launch of the training kernel over several caches: CTA b runs jobs[b]
// (device array); proto supplies the shape, dtype, encoding and loss
// settings shared by the caches.
cudaError_t launch_train_batched(const Cache* proto, const TrainJob* jobs, int n_jobs, cudaStream_t st) {
  if (proto->net.n_mats > kTrainMaxMats) return cudaErrorNotSupported;
  TrainParams p;
  memset(&p, 0, sizeof(p));
  p.jobs = jobs;
  p.n_mats = proto->net.n_mats;
  p.img = proto->img;
  p.img_bytes = proto->img.off[proto->net.n_mats];
  for (int l = 0; l <= kMaxMats; ++l) p.w_off[l] = proto->net.w_off[l];
  p.n_params = proto->net.n_params;
  p.pad = proto->cfg.pad_value;
  p.loss_mode = proto->cfg.loss_mode;
  p.loss_eps = proto->cfg.loss_eps;
  p.factor = proto->cfg.refl_factor;
  p.err = proto->err;
  const int smem = ((p.img_bytes + 1023) & ~1023) + p.n_mats * 16384 + 2 * 16384 + 1024;
  const bool bf16 = proto->cfg.dtype == NRC_BF16;
  const int mode = proto->cfg.enc_mode;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(unsigned(n_jobs));
  lc.blockDim = dim3(kTrainThreads);
  lc.dynamicSmemBytes = size_t(smem);
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  cudaError_t e = cudaSuccess;
  static std::atomic<int> attr_done[4];
#define NRC_LAUNCH(M, B)                                                   \
  e = ensure_smem(k_train_tc<M, B>, smem, &attr_done[2 * (M) + ((B) ? 1 : 0)]); \
  if (e != cudaSuccess) return e;                                          \
  e = cudaLaunchKernelEx(&lc, k_train_tc<M, B>, p);                        \
  if (e != cudaSuccess) return e;
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


int img8_offset(const NetShape& net, int l) {
  ImageShape img;
  make_image_shape(net, &img);
  return img8_offset_of(img, l);
}

cudaError_t launch_build_image_fp8(Cache* c, cudaStream_t st) {
  const int bytes = img8_offset(c->net, c->net.n_mats);
  cudaError_t e = cudaMemsetAsync(c->wimg8, 0, size_t(bytes), st);
  if (e != cudaSuccess) return e;
  k_build_image_fp8<<<c->net.n_mats, 256, 0, st>>>(query_weights(c), c->net, c->img, c->wimg8, bytes);
  return cudaGetLastError();
}

cudaError_t launch_infer_fp8(Cache* c, const float* rec, int64_t n, float* rgb, cudaStream_t st) {
  InferParams p;
  p.rec = rec;
  p.n = n;
  p.rgb = rgb;
  p.wimg = c->wimg8;
  p.img_bytes = img8_offset(c->net, c->net.n_mats);
  p.n_mats = c->net.n_mats;
  p.img = c->img;
  p.pad = c->cfg.pad_value;
  p.factor = c->cfg.refl_factor;
  p.err = c->err;
  const int img_alloc = (p.img_bytes + kImg8ScaleBytes + 1023) & ~1023;
  const int smem = img_alloc + kSlots * 2 * 8192 + 1024;
  const int64_t n_tiles = (n + kTile - 1) / kTile;
  const int64_t want = (n_tiles + kSlots - 1) / kSlots;
  const unsigned grid = unsigned(want < c->sm_count ? want : c->sm_count);
  static std::atomic<int> attr_done[2];
  cudaError_t e;
  if (c->cfg.enc_mode == 0) {
    e = ensure_smem(k_infer_fp8<0>, smem, &attr_done[0]);
    if (e != cudaSuccess) return e;
    k_infer_fp8<0><<<grid, kInferThreads, smem, st>>>(p);
  } else {
    e = ensure_smem(k_infer_fp8<1>, smem, &attr_done[1]);
    if (e != cudaSuccess) return e;
    k_infer_fp8<1><<<grid, kInferThreads, smem, st>>>(p);
  }
  return cudaGetLastError();
}
}  // namespace nrc
