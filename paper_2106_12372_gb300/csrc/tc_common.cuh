// Device building blocks shared by the tensor-core query, training and
// frame kernels: the query slots' TMEM columns and layer chain, record
// staging, and the 16-bit swizzled row helpers of the training tiles.
#pragma once

#include "tc_ptx.cuh"

namespace nrc {
using namespace tc;

constexpr int kSlots = kQuerySlots;  // 5 x (64 + 32) = 480 of the 512 TMEM columns
constexpr int kInferThreads = 128 * kSlots;
constexpr int kTmemCols = 512;
constexpr int kSlotCols = 96;

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  const uint32_t a = smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// Encodes a record (Table 1, Sec. 3.6) and stores the 64 packed 16-bit
// inputs into the slot's activation columns (this thread's TMEM lane).
template <int MODE, bool BF16>
__device__ __forceinline__ void encode_to_tmem(const float (&r)[kRecFloats], float pad, uint32_t t_act) {
  uint32_t pk[16];
  float f[kEncDims];
  encode_record<MODE>(r, pad, f);
#pragma unroll
  for (int j = 0; j < 16; ++j) pk[j] = pack2<BF16, false>(f[2 * j], f[2 * j + 1]);
  tmem_st16(t_act, pk);
#pragma unroll
  for (int j = 0; j < 16; ++j) pk[j] = pack2<BF16, false>(f[32 + 2 * j], f[33 + 2 * j]);
  tmem_st16(t_act + 16, pk);
  tmem_st_wait();
}

// Sum of a staged record's diffuse and specular albedo (floats 8..10 and
// 11..13: 16-byte chunks 2 and 3, stored at chunk q ^ rot of the 64-byte row).
__device__ __forceinline__ void staged_albedo_sum(const uint8_t* row, uint32_t rot, float (&f)[3]) {
  const float4 c2 = *reinterpret_cast<const float4*>(row + ((2u ^ rot) << 4));
  const float4 c3 = *reinterpret_cast<const float4*>(row + ((3u ^ rot) << 4));
  f[0] = c2.x + c2.w;
  f[1] = c2.y + c3.x;
  f[2] = c2.z + c3.y;
}

// The layer chain of one tile in one slot (see the file comment): per layer,
// the warpgroup's barrier, 4 MMAs issued by one thread, one waiter, and the
// ReLU + 16-bit epilogue back into the activation columns; the output
// layer's first 3 columns go to out (this thread's row; null if the row is
// past the end).  `last_layer()` runs in every thread of the slot
// just before the output layer's first barrier (the frame kernel publishes
// its next tile index there).
struct SlotTmem {
  uint32_t tmem;     // TMEM base (lane 0) of the CTA
  uint32_t acc_col;  // first accumulator column of the slot
  uint32_t act_col;  // first activation column of the slot
  uint32_t t_acc;    // this warp's lanes, accumulator columns
  uint32_t t_act;    // this warp's lanes, activation columns
};

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

template <bool BF16, class Hook = NoHook>
__device__ __forceinline__ void tile_layers(const ImageShape& img, int n_mats, const SlotTmem& st, uint32_t sw_base,
                                            int slot, int rit, uint64_t* bar, uint32_t& phase, int* err, float* out,
                                            const uint8_t* fac_row, uint32_t rot, Hook last_layer = Hook()) {
  // the slot's lead warp computes the (warp-uniform) descriptors together;
  // one elected thread issues, the warp's lane 0 waits.  The lead is warp
  // slot % 4 of the warpgroup: warp w runs on SM sub-partition w % 4, so the
  // slots' issue and wait work is spread over the four schedulers instead of
  // slowing one of them (and with it every slot's epilogue there).
  const int lead = slot & 3;
  const bool w0 = (rit >> 5) == lead;
  for (int l = 0; l < n_mats; ++l) {
    if (l + 1 == n_mats) last_layer();
    uint32_t idesc = 0;
    uint64_t bdesc = 0;
    if (w0) {
      idesc = idesc_f16(128, img.rows[l], BF16);
      bdesc = sdesc_sw128(sw_base + uint32_t(img.off[l]), 16, 1024);
    }
    fence_before();
    named_sync(1 + slot, 128);
    if (w0) {
      fence_after();
      if (elect_one()) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          mma_ts(st.tmem + st.acc_col, st.tmem + st.act_col + uint32_t(k * 8), bdesc + uint64_t(2 * k), idesc,
                 k > 0 ? 1u : 0u);
        mma_commit(bar);
      }
      __syncwarp();
      // one thread waits for the MMAs; the rest of the warpgroup sleeps at the barrier
      if (rit == 32 * lead) mbar_wait(bar, phase, err);
    }
    named_sync(1 + slot, 128);
    phase ^= 1u;
    fence_after();
    if (l + 1 < n_mats) {
      uint32_t v[64], pk[16];
      tmem_ld64(st.t_acc, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) pk[j] = pack2<BF16, true>(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
      tmem_st16(st.t_act, pk);
#pragma unroll
      for (int j = 0; j < 16; ++j) pk[j] = pack2<BF16, true>(__uint_as_float(v[32 + 2 * j]), __uint_as_float(v[33 + 2 * j]));
      tmem_st16(st.t_act + 16, pk);
      tmem_st_wait();
    } else {
      uint32_t v[4];
      tmem_ld4(st.t_acc, v);
      if (out) {
        float y0 = __uint_as_float(v[0]), y1 = __uint_as_float(v[1]), y2 = __uint_as_float(v[2]);
        if (fac_row) {  // reflectance factorisation: times the record's diffuse + specular albedo
          float f[3];
          staged_albedo_sum(fac_row, rot, f);
          y0 *= f[0];
          y1 *= f[1];
          y2 *= f[2];
        }
        out[0] = y0;
        out[1] = y1;
        out[2] = y2;
      }
    }
  }
}

// A slot's record staging: two 8 KB buffers of 128 rows x 64 B in shared
// memory, filled with cp.async; 16-byte chunk q of row r sits at chunk
// q ^ ((r / 2) % 4) so that the row reads are free of bank conflicts.
struct RecStage {
  uint32_t row0;     // shared address of this thread's row in buffer 0
  const uint8_t* p;  // the same, generic
  uint32_t rot;
  __device__ __forceinline__ void fetch(const float* rec, int64_t row, bool ok, int b) const {
    const float* src = rec + (ok ? row : 0) * kRecFloats;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      cp_async16(row0 + uint32_t(b * 8192) + ((uint32_t(q) ^ rot) << 4), src + 4 * q, ok ? 16u : 0u);
    cp_async_commit();
  }
  __device__ __forceinline__ void read(int b, float (&r)[kRecFloats]) const {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(p + b * 8192 + ((uint32_t(q) ^ rot) << 4));
      r[4 * q] = v.x;
      r[4 * q + 1] = v.y;
      r[4 * q + 2] = v.z;
      r[4 * q + 3] = v.w;
    }
  }
};

// Writes 16-byte chunks c0 .. c0+3 of row r of a 128-byte-swizzled tile.
__device__ __forceinline__ void store_half_row_sw128(uint8_t* base, int r, int c0, const uint32_t (&pk)[16]) {
  uint8_t* row = base + (r >> 3) * 1024 + (r & 7) * 128;
#pragma unroll
  for (int c = 0; c < 4; ++c)
    *reinterpret_cast<uint4*>(row + (((c0 + c) ^ (r & 7)) << 4)) =
        make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
}

__device__ __forceinline__ void load_half_row_sw128(const uint8_t* base, int r, int c0, uint32_t (&pk)[16]) {
  const uint8_t* row = base + (r >> 3) * 1024 + (r & 7) * 128;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint4 v = *reinterpret_cast<const uint4*>(row + (((c0 + c) ^ (r & 7)) << 4));
    pk[4 * c] = v.x;
    pk[4 * c + 1] = v.y;
    pk[4 * c + 2] = v.z;
    pk[4 * c + 3] = v.w;
  }
}

// delta pair from two FP32 pre-activations: rounded to 16 bit, clamped to the
// finite FP16 range, zeroed where the stored post-ReLU activation is zero.
template <bool BF16>
__device__ __forceinline__ uint32_t masked_delta2(float d0, float d1, uint32_t h2) {
  const uint32_t raw = pack2<BF16, false>(d0, d1);
  if (BF16) {
    const __nv_bfloat162 d = *reinterpret_cast<const __nv_bfloat162*>(&raw);
    const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&h2);
    const __nv_bfloat162 r = __hmul2(d, __hgt2(h, __float2bfloat162_rn(0.0f)));
    return *reinterpret_cast<const uint32_t*>(&r);
  } else {
    const __half2 lim = __float2half2_rn(60000.0f);
    const __half2 d = __hmax2(__hmin2(*reinterpret_cast<const __half2*>(&raw), lim), __hneg2(lim));
    const __half2 h = *reinterpret_cast<const __half2*>(&h2);
    const __half2 r = __hmul2(d, __hgt2(h, __float2half2_rn(0.0f)));
    return *reinterpret_cast<const uint32_t*>(&r);
  }
}

}  // namespace nrc
