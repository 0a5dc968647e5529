// One persistent launch per frame: the frame's cache queries and its online
// training steps run side by side on the device (Sec. 3.1-3.5: a frame's
// queries read the weights from before that frame's training, so the two are
// independent; Sec. 4, the fully fused network; Eq. 5; Sec. 5, Adam).
//
// The grid is one CTA per SM (cooperative launch, so every CTA is resident).
// CTAs 0 .. T-1 train, the others answer queries; when the training CTAs have
// run all the steps they answer queries too.  Query tiles are handed out by a
// device counter, so the work balances itself whatever the split.
//
// Query role: exactly the slots of k_infer_tc (five warpgroups, each a 128-row
// tile at a time, activations in TMEM, weights in shared memory).
//
// Training role, per step (Sec. 3.3: the steps of a frame use disjoint
// batches of the shuffled pool, Sec. 3.5):
//  - warps 17-19 (producer) gather the CTA's next tile of records through the
//    shuffle, encode it (Table 1) into a 16-bit swizzled H_0 buffer
//    (double-buffered) and stage its targets (the launch's first tile: the
//    compute warpgroups, one row per thread);
//  - warp 16 (issuer) issues every MMA from one elected thread, with
//    warp-uniform descriptors, after a named-barrier hand-off from the
//    compute warpgroups;
//  - warpgroups 0-3 (compute; thread (q, r) owns row r and columns
//    16q .. 16q+15 of every epilogue) run the epilogues of the layer chain:
//      forward  H_{l+1} = ReLU(W_l H_l)          (4 x M128 N64 K16 per layer;
//               layer 0 reads H_0 from shared memory, the others their A
//               operand from TMEM)
//      loss     relative L2 of Eq. 5, g' = 2 (y - t) / den (1/(3N) applied in Adam)
//      backward delta_l = (delta_{l+1} W_l) * [H_l > 0]   (A = delta in TMEM)
//               dW_l += delta_{l+1}^T H_l       (K = the tile's 128 rows,
//               both operands from shared-memory copies written behind the
//               chain)
//    the weight-gradient MMAs of a stage are issued one stage late, after the
//    next stage's data-gradient MMAs, so that the dependent chain never waits
//    behind them; dW accumulates in TMEM over the CTA's tiles of the step;
//  - then every training CTA writes its dW partial (the layers that became
//    final during the last tile's backward already behind its MMAs), the T
//    CTAs meet at a grid barrier, each reduces a slice of the parameters over
//    the T partials (fixed order), applies Adam (and the weight average of
//    Eq. 2) and writes the 16-bit image of its slice; a second barrier, and
//    every CTA reloads the image for the next step.
// The training writes its weight images into work buffers; the last CTA to
// finish copies them over the cache's images, so that every query of the
// frame, including those of CTAs that trained first, reads the old weights.
//
// Every wait is bounded (mbarrier waits and the grid barrier give up after
// kWaitLimitNs, set the error word and let the kernel run to its end).
#include <algorithm>
#include <cstring>

#include "tc_common.cuh"

namespace nrc {

constexpr int kFrameThreads = kInferThreads;  // 5 warpgroups
constexpr int kFrameCompute = 512;            // training: warpgroups 0-3; warpgroup 4 is the producer
constexpr int kFrameMaxMats = 6;              // TMEM: accumulator 64 + A operand 32 + 6 x 64 dW columns
constexpr int kFrameBufs = 10;                // 16 KB tiles: H_0 x 2, H_1..H_5, delta_L, delta_{L-1}, delta_{L-2}
constexpr int kBarCompute = 6;                // named barrier of the compute warpgroups (1..5: query slots)
constexpr int kBarOps = 7;                    // compute warpgroups -> MMA issuer hand-off
// training TMEM columns: accumulator 0..63, the next MMA's 16-bit A operand
// (activations or deltas) 64..95, dW_l at 96 + 64 l
constexpr uint32_t kActCol = 64;
constexpr uint32_t kDwCol = 96;
constexpr int kIssuerWarp = 16;               // training: warp 16 issues the MMAs, warps 17-19 produce
constexpr int kProducerThreads = kFrameThreads - (kIssuerWarp + 1) * 32;
constexpr int kFrameMaxSteps = 64;            // training steps per frame launch
constexpr int kSumBatch = 12;                 // partial rows loaded in flight per thread in the reduction

struct FrameParams {
  // queries
  const float* rec;
  int64_t n_q;
  float* rgb;
  const uint8_t* qimg;  // the image the queries read (weights before the frame's training)
  // training
  const float* pool;
  const float* target;
  int64_t n_pool;
  int64_t batch;
  uint64_t a, c;  // the frame's shuffle (Sec. 3.5)
  int n_steps;
  int n_train;  // T training CTAs
  float* loss_out;
  float* w;
  float* m;
  float* v;
  long long* t_ctr;
  float* ema;                // null: no weight average
  const uint8_t* img_in;     // image of the weights the first step starts from
  uint8_t* img_work;         // training's image, written by every step
  uint8_t* img_ema_work;     // its weight-average image
  uint8_t* img_out;          // the cache's image (img_work copied here at the end)
  uint8_t* img_ema_out;
  float* partials;           // [T][partial_stride]
  unsigned* sync;            // [0] grid barrier, [1] query tile tickets, [2] retired CTAs, [3] CTAs holding the old image
  TrainView tv;              // the frame's training, as the training role reads it (b unused: blockIdx.x)
  NetShape net;
  ImageShape img;
  int img_bytes;
  float pad;
  int loss_mode;
  float loss_eps;
  int factor;
  float inv3n;
  float lr, b1, b2, eps, alpha;
  int* err;
};

// Two 16-byte chunks c0, c0+1 of row r of a 128-byte-swizzled 128-row tile.
__device__ __forceinline__ void store_q_sw128(uint8_t* base, int r, int c0, const uint32_t (&pk)[8]) {
  uint8_t* row = base + (r >> 3) * 1024 + (r & 7) * 128;
  *reinterpret_cast<uint4*>(row + (((c0) ^ (r & 7)) << 4)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  *reinterpret_cast<uint4*>(row + (((c0 + 1) ^ (r & 7)) << 4)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}
__device__ __forceinline__ void load_q_sw128(const uint8_t* base, int r, int c0, uint32_t (&pk)[8]) {
  const uint8_t* row = base + (r >> 3) * 1024 + (r & 7) * 128;
  const uint4 a = *reinterpret_cast<const uint4*>(row + (((c0) ^ (r & 7)) << 4));
  const uint4 b = *reinterpret_cast<const uint4*>(row + (((c0 + 1) ^ (r & 7)) << 4));
  pk[0] = a.x, pk[1] = a.y, pk[2] = a.z, pk[3] = a.w, pk[4] = b.x, pk[5] = b.y, pk[6] = b.z, pk[7] = b.w;
}

// Barrier of the T training CTAs: the k-th call of the frame waits until the
// counter reaches k * T.  Bounded: gives up after kWaitLimitNs (or at once
// once the error word is set), setting kErrTimeout.
__device__ __forceinline__ void train_grid_barrier(unsigned* ctr, unsigned target, int* err, int tid) {
  named_sync(kBarCompute, kFrameCompute);
  if (tid == 0) {
    // release: the CTA's writes (ordered before this thread by the barrier)
    // happen before the arrival; acquire: the others' before what follows
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
    unsigned long long t0 = 0;
    long long c0 = clock64();
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
      if (v >= target) break;
      if (clock64() - c0 > 8192) {
        if (*reinterpret_cast<volatile int*>(err) != 0) break;
        const unsigned long long now = globaltimer_ns();
        if (t0 == 0) t0 = now;
        if (now - t0 > kWaitLimitNs) {
          atomicOr(err, kErrTimeout);
          break;
        }
        c0 = clock64();
      }
    }
  }
  named_sync(kBarCompute, kFrameCompute);
}

// row r of tile i of a training step (Sec. 3.5: the frame's shuffle of the
// pool; step = the step's index in the shuffled sequence) encoded (Table 1)
// into H_0 buffer par, its targets and factors into aux
template <int MODE, bool BF16>
__device__ __noinline__ void stage_train_row(const float* pool, const float* target, int64_t n_pool, int64_t batch,
                                           int step, int factor, float pad, int* err, uint8_t* Hb, float* aux,
                                           int64_t i, int par, int r, uint64_t sh_a, uint64_t sh_c) {
  const int64_t row = i * kTile + r;
  float rec[kRecFloats], tg[3] = {0.f, 0.f, 0.f}, fac[3] = {1.f, 1.f, 1.f};
  if (row < batch) {
    const uint64_t idx = uint64_t(step) * uint64_t(batch) + uint64_t(row);
    int64_t src = int64_t((sh_a * idx + sh_c) % uint64_t(n_pool));
    if (!NRC_DCHECK(src >= 0 && src < n_pool, err)) src = 0;
    load_record(pool, src, rec);
    tg[0] = __ldg(target + src * 3);
    tg[1] = __ldg(target + src * 3 + 1);
    tg[2] = __ldg(target + src * 3 + 2);
    if (factor) {
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) fac[ch] = rec[8 + ch] + rec[11 + ch];
    }
  } else {
#pragma unroll
    for (int k = 0; k < kRecFloats; ++k) rec[k] = 0.0f;
  }
  float f[kEncDims];
  encode_record<MODE>(rec, pad, f);
  uint8_t* h0 = Hb + par * 16384;
#pragma unroll
  for (int c4 = 0; c4 < 4; ++c4) {
    uint32_t pk[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) pk[k] = pack2<BF16, false>(f[16 * c4 + 2 * k], f[16 * c4 + 2 * k + 1]);
    store_q_sw128(h0, r, 2 * c4, pk);
  }
  float* ax = aux + (par * kTile + r) * 8;
  ax[0] = tg[0], ax[1] = tg[1], ax[2] = tg[2], ax[3] = fac[0], ax[4] = fac[1], ax[5] = fac[2];
}


template <int MODE, bool BF16>
__device__ __forceinline__ void frame_train(const FrameParams& p, const TrainView& tv, const int b, uint8_t* sw,
                                            uint32_t tmem, uint64_t* bar_w,
                                            uint64_t* bar_mma, uint64_t* bar_dw, uint64_t* bar_full,
                                            uint64_t* bar_free, float* red, const float* s_corr) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int T = tv.T;
  const int L = p.net.n_mats;
  const int64_t tiles = (tv.batch + kTile - 1) / kTile;
  uint8_t* Hb = sw + ((p.img_bytes + 1023) & ~1023);
  float* aux = reinterpret_cast<float*>(Hb + kFrameBufs * 16384);  // [2][128][8]: target 3, factor 3
  const uint32_t hb_base = smem_u32(Hb), sw_base = smem_u32(sw);
  // buffer of H_l (H_0 alternates between 0 and 1) and of delta_l
  auto hbuf = [&](int l, int par) { return l == 0 ? par : 1 + l; };
  auto dbuf = [&](int l) { return l == L ? 7 : l == L - 1 ? 8 : l == L - 2 ? 9 : 1 + (l + 2); };

  auto stage_row = [&](int64_t i, int s, int par, int r, uint64_t sh_a, uint64_t sh_c) {
    stage_train_row<MODE, BF16>(tv.pool, tv.target, tv.n_pool, tv.batch, tv.step0 + s, p.factor, p.pad, p.err, Hb, aux, i,
                                par, r, sh_a, sh_c);
  };

  if (warp > kIssuerWarp) {
    // ------------------------------------------------------------ producer
    uint64_t sh_a = tv.a, sh_c = tv.c;
    if (tv.seed) lcg_shuffle(tv.n_pool, *tv.seed, &sh_a, &sh_c);  // the frame seed lives on the device
    // three warps stage each tile's 128 rows (rows pt and pt + 96), then
    // arrive on the tile's full barrier; the launch's first tile is staged
    // by the compute warpgroups (one row per thread) while these stage the
    // second
    const int pt = tid - (kIssuerWarp + 1) * 32;
    int j = 0;
    for (int s = 0; s < p.n_steps; ++s) {
      for (int64_t i = b; i < tiles; i += T, ++j) {
        if (j == 0) continue;
        const int par = j & 1;
        if (j >= 2) mbar_wait(&bar_free[par], uint32_t(((j - 2) >> 1) & 1), p.err);
        for (int r = pt; r < kTile; r += kProducerThreads) stage_row(i, s, par, r, sh_a, sh_c);
        fence_proxy_async_smem();
        mbar_arrive(&bar_full[par]);
      }
    }
    return;
  }

  if (warp == kIssuerWarp) {
    // --------------------------------------------------------------- issuer
    // One elected thread issues every MMA of the training, in the order of
    // the compute warpgroups' epilogues: before each MMA group (except a
    // tile's first layer, which follows its predecessor's last group) the
    // warp waits at kBarOps for the 512 compute threads' arrival (their
    // operands stored, their TMEM reads of the accumulator done).  The warp
    // computes the descriptors together (warp-uniform values), advancing a
    // base descriptor by byte offset / 16 in its start-address field.
    const uint64_t hk = sdesc_sw128(hb_base, 16, 1024);     // H / delta tiles, K-major
    const uint64_t hmn = sdesc_sw128(hb_base, 1024, 1024);  // ... MN-major
    const uint64_t hmn0 = sdesc_sw128(hb_base, 0, 1024);    // ... MN-major, M = 128 reading rows 0..63 twice
    const uint64_t wk = sdesc_sw128(sw_base, 16, 1024);     // weight image, K-major
    const uint64_t wmn = sdesc_sw128(sw_base, 1024, 1024);  // ... MN-major
    const uint32_t idd = idesc_f16(128, 64, BF16, false, true);
    const uint32_t idw = idesc_f16(128, 64, BF16, true, true);
    constexpr uint64_t kBuf = 16384 >> 4;  // one tile buffer in descriptor units
    auto issue_dw = [&](int l, int par, bool first, bool lead) {
      const uint64_t a = hmn0 + uint64_t(dbuf(l + 1)) * kBuf, bb = hmn + uint64_t(hbuf(l, par)) * kBuf;
      const uint32_t dcol = tmem + kDwCol + uint32_t(l * 64);
      if (lead) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
          mma_ss(dcol, a + uint64_t(k * 128), bb + uint64_t(k * 128), idw, (first && k == 0) ? 0u : 1u);
      }
    };
    uint32_t wph = 0;
    int j = 0;
    for (int s = 0; s < p.n_steps; ++s) {
      if (elect_one()) mbar_wait(bar_w, wph, p.err);
      __syncwarp();
      wph ^= 1u;
      // layer 0 of tile jj: reads the producer's H_0 from shared memory
      auto issue_layer0 = [&](int jj) {
        const int pp = jj & 1;
        if (elect_one()) mbar_wait(&bar_full[pp], uint32_t((jj >> 1) & 1), p.err);
        __syncwarp();
        const uint32_t idesc = idesc_f16(128, p.img.rows[0], BF16);
        const uint64_t a = hk + uint64_t(hbuf(0, pp)) * kBuf, bb = wk + uint64_t(p.img.off[0] >> 4);
        fence_after();
        if (elect_one()) {
#pragma unroll
          for (int k = 0; k < 4; ++k) mma_ss(tmem, a + uint64_t(2 * k), bb + uint64_t(2 * k), idesc, k > 0 ? 1u : 0u);
          mma_commit(bar_mma);
        }
        __syncwarp();
      };
      bool first = true;
      // the previous tile's dW_0, issued behind this tile's layer 1 (not with
      // its dW_1 behind layer 0), so that the chain waits for half as many
      // weight-gradient MMAs at each tile boundary
      bool dw0_pending = false, prev_first = false;
      int prev_par = 0;
      for (int64_t i = b; i < tiles; i += T, ++j) {
        const int par = j & 1;
        const bool last_tile = i + T >= tiles;
        if (first) issue_layer0(j);  // later tiles' layer 0 went out ahead of the previous tile's last dW
        for (int l = 1; l < L; ++l) {  // forward: A = the activations the epilogue left in TMEM
          const uint32_t idesc = idesc_f16(128, p.img.rows[l], BF16);
          const uint64_t bb = wk + uint64_t(p.img.off[l] >> 4);
          named_sync(kBarOps, kFrameCompute + 32);
          fence_after();
          const bool lead = elect_one();
          if (lead) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
              mma_ts(tmem, tmem + kActCol + uint32_t(8 * k), bb + uint64_t(2 * k), idesc, k > 0 ? 1u : 0u);
            mma_commit(bar_mma);
          }
          if (l == 1 && dw0_pending) {
            issue_dw(0, prev_par, prev_first, lead);
            if (lead) mma_commit(&bar_free[prev_par]);  // the previous tile's buffers are free
            dw0_pending = false;
          }
          __syncwarp();
        }
        for (int l = L - 1; l >= 1; --l) {  // backward data (A = delta_{l+1} in TMEM) and the deferred dW_{l+1}
          const uint64_t bb = wmn + uint64_t(p.img.off[l] >> 4);
          const int nk = p.img.rows[l] / 16;
          named_sync(kBarOps, kFrameCompute + 32);
          fence_after();
          const bool lead = elect_one();
          if (lead) {
            for (int k = 0; k < nk; ++k) mma_ts(tmem, tmem + kActCol + uint32_t(8 * k), bb + uint64_t(128 * k), idd, k > 0 ? 1u : 0u);
            mma_commit(bar_mma);
          }
          if (l + 1 < L) issue_dw(l + 1, par, first, lead);
          __syncwarp();
        }
        // stage 0: the next tile's layer 0 first (the chain goes on), then
        // dW_1 (deferred); dW_0 follows behind the next tile's layer 1.  The
        // step's last tile issues both now: bar_dw first (the weight
        // gradients issued so far are final: the compute writes dW_2, dW_3
        // behind dW_1 and dW_0), then bar_mma.  bar_free[par], once dW_0 is
        // done, frees this tile's H_0 buffer (producer) and the shared copies
        // the next tile overwrites.
        named_sync(kBarOps, kFrameCompute + 32);
        if (!last_tile) issue_layer0(j + 1);
        fence_after();
        const bool lead = elect_one();
        if (last_tile) {
          if (lead) mma_commit(bar_dw);
          issue_dw(1, par, first, lead);
          issue_dw(0, par, first, lead);
          if (lead) mma_commit(bar_mma);
          if (lead) mma_commit(&bar_free[par]);
        } else {
          issue_dw(1, par, first, lead);
          dw0_pending = true;
          prev_par = par;
          prev_first = first;
        }
        __syncwarp();
        first = false;
      }
    }
    return;
  }

  // -------------------------------------------------------------- compute
  const int q = tid >> 7;    // column quarter
  const int r = tid & 127;   // row == TMEM lane
  const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
  const uint32_t t_acc = tmem + lane_base + uint32_t(16 * q);
  const long long t0 = *tv.t_ctr;
  uint32_t phase = 0;
  int j = 0;
  // one waiter per warp, then the warp's threads order their TMEM reads after it
  auto wait_mma = [&]() {
    if ((tid & 31) == 0) mbar_wait(bar_mma, phase, p.err);
    __syncwarp();
    phase ^= 1u;
    fence_after();
  };
  // operands stored and the accumulator read: the issuer may go on (with
  // the shared-memory copies written so far made visible to the MMAs)
  auto release = [&]() {
    fence_proxy_async_smem();
    fence_before();
    named_arrive(kBarOps, kFrameCompute + 32);
  };
  // the same when the operand went to TMEM only
  auto release_tmem = [&]() {
    fence_before();
    named_arrive(kBarOps, kFrameCompute + 32);
  };
  const uint32_t t_act = tmem + lane_base + kActCol + uint32_t(8 * q);

  // dW_l of this CTA's step to its partial.  Layout (private to this kernel):
  // element (o, i) of matrix l at w_off[l] + ((i / 4) * R_l + o) * 4 + i % 4,
  // R_l = its rows, so that a warp's 32 rows store 32 consecutive 16-byte
  // quads; a quad holds 4 consecutive inputs of one row, as in the weights.
  // TMEM lanes 64..127 hold the same rows as 0..63 (the MMA's M = 128 reads
  // delta's 64 rows twice), so either half of the lanes can write a layer.
  const size_t stride = partial_stride(p.net.n_params);
  float* P = tv.partials + size_t(b) * stride;
  auto write_dw = [&](int l) {
    const int R = p.net.dims[l + 1];
    const int o = r & 63;
    uint32_t v[16];
    tmem_ld16(tmem + lane_base + kDwCol + uint32_t(l * 64 + 16 * q), v);
    if (o < R) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (NRC_DCHECK(p.net.w_off[l] + ((4 * q + c) * R + o) * 4 + 3 < p.net.n_params, p.err))
        *reinterpret_cast<float4*>(P + p.net.w_off[l] + ((4 * q + c) * R + o) * 4) =
            make_float4(__uint_as_float(v[4 * c]), __uint_as_float(v[4 * c + 1]), __uint_as_float(v[4 * c + 2]),
                        __uint_as_float(v[4 * c + 3]));
    }
  };
  const bool lanes_lo = (warp & 3) < 2;  // this warp's TMEM lanes are 0..63
  float w1 = 0.f, m1 = 0.f, v1 = 0.f, e1 = 0.f;  // the Adam state of the thread's parameter

  for (int s = 0; s < p.n_steps; ++s) {
    if (tid == 0) {
      fence_proxy_async_global();
      mbar_arrive_expect_tx(bar_w, uint32_t(p.img_bytes));
      bulk_g2s(sw, s == 0 ? tv.img_in : tv.img_work, uint32_t(p.img_bytes), bar_w);
    }
    if (s == 0) {
      // the launch's first tile, one row per thread: the chain waits for one
      // round of record loads instead of the producer's two
      if (tid < kTile) {
        uint64_t sh_a = tv.a, sh_c = tv.c;
        if (tv.seed) lcg_shuffle(tv.n_pool, *tv.seed, &sh_a, &sh_c);
        stage_row(b, 0, 0, tid, sh_a, sh_c);
        fence_proxy_async_smem();
      }
      named_sync(kBarCompute, kFrameCompute);
      if (tid < kProducerThreads) mbar_arrive(&bar_full[0]);  // the count the producer warps would give
    }
    float loss_acc = 0.0f;
    for (int64_t i = b; i < tiles; i += T, ++j) {
      const int par = j & 1;
      const bool last_tile = i + T >= tiles;
      const bool first_of_step = i == b;

      // ------------------------------------------------------------ forward
      // The previous tile's dW_1 went out behind this tile's layer 0 and its
      // dW_0 behind layer 1: H_1's shared copy (dW_1's operand buffer) waits
      // in registers until layer 1's MMAs are done, and from H_3 on (whose
      // buffer holds dW_0's delta operand) the copies wait for bar_free.
      float y[3] = {0.f, 0.f, 0.f};
      uint32_t pk_h1[8];
      bool freed = first_of_step;
      auto wait_free = [&]() {
        if (!freed) {
          if ((tid & 31) == 0) mbar_wait(&bar_free[(j - 1) & 1], uint32_t(((j - 1) >> 1) & 1), p.err);
          __syncwarp();
          freed = true;
        }
      };
      for (int l = 0; l < L; ++l) {
        wait_mma();
        if (l == 1 && !first_of_step) store_q_sw128(Hb + hbuf(1, par) * 16384, r, 2 * q, pk_h1);
        if (l + 1 < L) {
          uint32_t v[16], pk[8];
          tmem_ld16(t_acc, v);
#pragma unroll
          for (int k = 0; k < 8; ++k) pk[k] = pack2<BF16, true>(__uint_as_float(v[2 * k]), __uint_as_float(v[2 * k + 1]));
          tmem_st8(t_act, pk);  // the next layer's A operand
          tmem_st_wait();
          release_tmem();
          // the copy the weight gradients (and the backward masks) read, behind the next layer's MMAs
          if (l == 0 && !first_of_step) {
#pragma unroll
            for (int k = 0; k < 8; ++k) pk_h1[k] = pk[k];
          } else {
            if (l + 1 >= 3) wait_free();
            store_q_sw128(Hb + hbuf(l + 1, par) * 16384, r, 2 * q, pk);
          }
          fence_proxy_async_smem();
        } else {
          if (l == 1 && !first_of_step) fence_proxy_async_smem();  // two layers: H_1 went out above
          if (q == 0) {
            uint32_t v[4];
            tmem_ld4(t_acc, v);
            y[0] = __uint_as_float(v[0]);
            y[1] = __uint_as_float(v[1]);
            y[2] = __uint_as_float(v[2]);
          }
        }
      }
      wait_free();  // (shallow nets: the delta buffers the backward writes next may be dW_0's operands)

      // --------------------------------------------------------------- loss
      if (q == 0) {
        if ((tid & 31) == 0) mbar_wait(&bar_full[par], uint32_t((j >> 1) & 1), p.err);  // the staged targets
        __syncwarp();
        const float* ax = aux + (par * kTile + r) * 8;
        const bool valid = i * kTile + r < tv.batch;
        const float fac[3] = {ax[3], ax[4], ax[5]};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) y[ch] *= fac[ch];
        const float lum = 0.2126f * y[0] + 0.7152f * y[1] + 0.0722f * y[2];
        float lr = 0.0f, g[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          const float den = (p.loss_mode == NRC_LOSS_LUMINANCE ? lum * lum : y[ch] * y[ch]) + p.loss_eps;
          const float inv = 1.0f / den;
          const float diff = y[ch] - ax[ch];
          lr = fmaf(diff * diff, inv, lr);
          g[ch] = valid ? fminf(fmaxf(2.0f * diff * inv * fac[ch], -60000.0f), 60000.0f) : 0.0f;
        }
        loss_acc += valid ? lr : 0.0f;
        uint32_t pk[8] = {pack2<BF16, false>(g[0], g[1]), pack2<BF16, false>(g[2], 0.0f), 0u, 0u, 0u, 0u, 0u, 0u};
        tmem_st8(t_act, pk);  // A of the output layer's backward MMA (K = 16: act columns 0..7)
        tmem_st_wait();
        release_tmem();
        store_q_sw128(Hb + dbuf(L) * 16384, r, 0, pk);
        fence_proxy_async_smem();
      } else {
        release_tmem();
      }

      // ----------------------------------------------------------- backward
      for (int l = L - 1; l >= 1; --l) {
        wait_mma();
        uint32_t v[16], h2[8], pk[8];
        tmem_ld16(t_acc, v);
        load_q_sw128(Hb + hbuf(l, par) * 16384, r, 2 * q, h2);
#pragma unroll
        for (int k = 0; k < 8; ++k) pk[k] = masked_delta2<BF16>(__uint_as_float(v[2 * k]), __uint_as_float(v[2 * k + 1]), h2[k]);
        if (l > 1) {
          tmem_st8(t_act, pk);  // A of the next data-gradient MMA
          tmem_st_wait();
          release_tmem();
          store_q_sw128(Hb + dbuf(l) * 16384, r, 2 * q, pk);
          fence_proxy_async_smem();
          // the step's last tile: dW_{l+2} completed before this stage's data
          // MMAs (issued one stage late, in order); write it behind the next MMAs
          if (last_tile && l + 2 < L && lanes_lo == ((l & 1) == 0)) write_dw(l + 2);
        } else {
          // delta_1 feeds only dW_0, issued right after this release
          store_q_sw128(Hb + dbuf(l) * 16384, r, 2 * q, pk);
          release();
        }
      }
      if (last_tile) {
        // bar_dw: every weight gradient but dW_1 and dW_0 is final; dW_2 and
        // dW_3 go out while those two run, then the step's last MMAs
        if ((tid & 31) == 0) mbar_wait(bar_dw, uint32_t(s & 1), p.err);
        __syncwarp();
        fence_after();
        for (int l = 2; l < L && l < 4; ++l)
          if (lanes_lo == ((l & 1) == 0)) write_dw(l);
        wait_mma();
      }
    }

    // ------------------------------------------- the CTA's partial of step s
    // dW_{L-1} .. dW_2 went out during the last tile's backward (stages l >= 2
    // wrote dW_{l+2}, then dW_3 and dW_2 at bar_dw); dW_1 and dW_0, final
    // now, one per lane half
    for (int l = 0; l < L && l < 2; ++l)
      if (lanes_lo == ((l & 1) == 0)) write_dw(l);
    {
      float sl = loss_acc;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sl += __shfl_down_sync(0xffffffffu, sl, off);
      if (q == 0 && (tid & 31) == 0) red[warp] = sl;
    }
    // CTA b owns the partial quads [q_lo, q_hi); thread tid finishes element
    // tid % 4 of quad tid / 4.  With one element per thread the thread keeps
    // that parameter's state in registers from step to step: loaded before
    // the first step's barrier, written back by the launch's last step
    const int QT = (p.net.n_params + 3) / 4;
    const int q_lo = int((long long)b * QT / T), q_hi = int((long long)(b + 1) * QT / T);
    const int Qb = q_hi - q_lo;
    auto param_of = [&](int Qp, int e, int& l_out) {
      int l = 0;
      while (l + 1 < L && Qp * 4 >= p.net.w_off[l + 1]) ++l;
      const int R = p.net.dims[l + 1];
      const int loc = Qp - p.net.w_off[l] / 4;
      l_out = l;
      return p.net.w_off[l] + (loc % R) * 64 + 4 * (loc / R) + e;
    };
    int pi = -1, li = 0;
    auto load_state = [&](int Qp, int e) {
      pi = param_of(Qp, e, li);
      if (pi < p.net.n_params) {
        w1 = __ldcg(tv.w + pi);
        m1 = __ldcg(tv.m + pi);
        v1 = __ldcg(tv.v + pi);
        if (tv.ema) e1 = __ldcg(tv.ema + pi);
      }
    };
    const bool one_each = 4 * Qb <= kFrameCompute;
    // the slice's weights, moments (and average) come into shared memory by
    // cp.async while the first step's barrier runs: quad qd of array a at
    // st_state[a][qd]
    float4* st_state = reinterpret_cast<float4*>(Hb + 3 * 16384);  // [4][Qb], Qb <= 128
    if (one_each && s == 0 && tid < 4 * Qb) {
      const int a = tid / Qb, qd = tid % Qb;
      const float* arr = a == 0 ? tv.w : a == 1 ? tv.m : a == 2 ? tv.v : tv.ema;
      if (arr) {
        int l_unused;
        const int p0 = param_of(q_lo + qd, 0, l_unused);
        const bool ok = p0 < p.net.n_params;
        cp_async16(smem_u32(st_state + a * Qb + qd), arr + (ok ? p0 : 0), ok ? 16u : 0u);
      }
    }
    cp_async_commit();
    fence_before();
    named_sync(kBarCompute, kFrameCompute);
    if (tid == 0) P[p.net.n_params] = ((red[0] + red[1]) + (red[2] + red[3])) * tv.inv3n;
    train_grid_barrier(tv.bar, unsigned(2 * s + 1) * unsigned(T), p.err, tid);

    // the step's loss: the T partial sums, by one warp (lane k sums partials
    // k, k + 32, ... in order, then a fixed shuffle tree)
    if (b == 0 && warp == kFrameCompute / 32 - 1 && tv.loss_out) {
      float sl = 0.0f;
      for (int k = tid & 31; k < T; k += 32) sl += __ldcg(tv.partials + size_t(k) * stride + p.net.n_params);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sl += __shfl_down_sync(0xffffffffu, sl, off);
      if ((tid & 31) == 0) tv.loss_out[s] = sl;
    }
    // ------------------------------------------------------ reduce + Adam
    // Thread (ch, qd) sums partials ch*C .. ch*C+C-1 of quad qd in order; the
    // element's thread adds the NC chunk sums in order.  With more than 128
    // quads per CTA a thread sums all T partials of its element.
    const float c1 = s_corr[4 * s], c2 = s_corr[4 * s + 1], eta = s_corr[4 * s + 2], eta_prev = s_corr[4 * s + 3];
    const int NC = one_each && Qb > 0 ? max(1, min(T, kFrameCompute / Qb)) : 1;
    const int C = (T + NC - 1) / NC;
    float4* scratch = reinterpret_cast<float4*>(Hb + 2 * 16384);  // [NC][Qb] <= 8 KB, free between tiles
    if (one_each && tid < NC * Qb) {
      const int ch = tid / Qb, qd = tid % Qb;
      const float* src = tv.partials + size_t(q_lo + qd) * 4;
      const int k_lo = ch * C, k_hi = min(T, k_lo + C);
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int k0 = k_lo; k0 < k_hi; k0 += kSumBatch) {
        float4 t4[kSumBatch];
#pragma unroll
        for (int u = 0; u < kSumBatch; ++u)
          t4[u] = (k0 + u < k_hi && NRC_DCHECK(size_t(q_lo + qd) * 4 + 3 < stride, p.err))
                      ? __ldcg(reinterpret_cast<const float4*>(src + size_t(k0 + u) * stride))
                      : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < kSumBatch; ++u) {
          acc.x += t4[u].x;
          acc.y += t4[u].y;
          acc.z += t4[u].z;
          acc.w += t4[u].w;
        }
      }
      scratch[ch * Qb + qd] = acc;
    }
    cp_async_wait<0>();  // this thread's state quads have landed
    named_sync(kBarCompute, kFrameCompute);
    // the parameters' fp32 state goes to global memory once per launch
    // when each thread keeps its parameter's state in registers
    const bool write_state = !one_each || s + 1 == p.n_steps;
    auto adam1 = [&](float g) {  // the loaded parameter's step (pi < n_params)
      g *= tv.inv3n;
      m1 = fmaf(p.b1, m1, (1.0f - p.b1) * g);
      v1 = fmaf(p.b2, v1, (1.0f - p.b2) * g * g);
      w1 = w1 - p.lr * (m1 / c1) / (sqrtf(v1 / c2) + p.eps);
      if (write_state) {
        tv.w[pi] = w1;
        tv.m[pi] = m1;
        tv.v[pi] = v1;
      }
      const int qq = pi - p.net.w_off[li];
      uint32_t off = uint32_t(p.img.off[li]) + sw128_offset(uint32_t(qq / 64), uint32_t(qq % 64));
      if (!NRC_DCHECK(off + 2 <= uint32_t(p.img_bytes), p.err)) off = 0;
      if (BF16)
        *reinterpret_cast<__nv_bfloat16*>(tv.img_work + off) = __float2bfloat16_rn(w1);
      else
        *reinterpret_cast<__half*>(tv.img_work + off) = __float2half_rn(w1);
      if (tv.ema) {
        // the weight average of Eq. 2 (bias-corrected reading); never read by training
        e1 = ((1.0f - p.alpha) * w1 + p.alpha * eta_prev * e1) / eta;
        if (write_state) tv.ema[pi] = e1;
        if (BF16)
          *reinterpret_cast<__nv_bfloat16*>(tv.img_ema_work + off) = __float2bfloat16_rn(e1);
        else
          *reinterpret_cast<__half*>(tv.img_ema_work + off) = __float2half_rn(e1);
      }
    };
    if (one_each) {
      if (tid < 4 * Qb) {
        pi = param_of(q_lo + tid / 4, tid % 4, li);
        if (s == 0) {
          const float* sst = reinterpret_cast<const float*>(st_state);
          w1 = sst[tid];
          m1 = sst[4 * Qb + tid];
          v1 = sst[8 * Qb + tid];
          if (tv.ema) e1 = sst[12 * Qb + tid];
        }
      }
      if (tid < 4 * Qb && pi < p.net.n_params) {
        const float* sc = reinterpret_cast<const float*>(scratch);
        float g = sc[tid];
        for (int ch = 1; ch < NC; ++ch) g += sc[ch * 4 * Qb + tid];
        adam1(g);
      }
    } else {
      for (int e = tid; e < 4 * Qb; e += kFrameCompute) {
        load_state(q_lo + e / 4, e % 4);
        if (pi >= p.net.n_params) continue;
        float g = 0.0f;
        for (int k = 0; k < T; ++k) g += __ldcg(tv.partials + size_t(k) * stride + size_t(q_lo) * 4 + e);
        adam1(g);
      }
    }
    fence_proxy_async_global();
    if (s + 1 < p.n_steps) train_grid_barrier(tv.bar, unsigned(2 * s + 2) * unsigned(T), p.err, tid);
  }
  if (b == 0 && tid == 0) *tv.t_ctr = t0 + p.n_steps;
}

// The training's weight image (and weight-average image) over the cache's:
// all threads of the CTA.
__device__ __forceinline__ void copy_images(const FrameParams& p) {
  const int n16 = p.img_bytes / 16;
  const uint4* src = reinterpret_cast<const uint4*>(p.img_work);
  uint4* dst = reinterpret_cast<uint4*>(p.img_out);
  for (int k = threadIdx.x; k < n16; k += kFrameThreads) dst[k] = __ldcg(src + k);
  if (p.ema) {
    const uint4* se = reinterpret_cast<const uint4*>(p.img_ema_work);
    uint4* de = reinterpret_cast<uint4*>(p.img_ema_out);
    for (int k = threadIdx.x; k < n16; k += kFrameThreads) de[k] = __ldcg(se + k);
  }
}

template <int MODE, bool BF16>
__global__ void __launch_bounds__(kFrameThreads, 1) k_frame_tc(const __grid_constant__ FrameParams p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_w, bar_mma, bar_dw, bar_full[2], bar_free[2];
  __shared__ uint64_t bar_wq, bar_q[kSlots];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int s_next[kSlots];
  __shared__ float red[16];
  __shared__ int s_last;
  // per step: Adam's bias corrections 1 - b1^t, 1 - b2^t and the weight
  // average's eta_t, eta_{t-1} (Eq. 2), t = the step's counter
  __shared__ float s_corr[4 * kFrameMaxSteps];
  uint8_t* sw = align1024(smem_raw);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const bool trainer = int(blockIdx.x) < p.n_train;
  if (warp == 0) {
    tmem_alloc(&tmem_base_sh, kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar_w, 1);
    mbar_init(&bar_mma, 1);
    mbar_init(&bar_dw, 1);
    mbar_init(&bar_full[0], kProducerThreads);
    mbar_init(&bar_full[1], kProducerThreads);
    mbar_init(&bar_free[0], 1);
    mbar_init(&bar_free[1], 1);
    mbar_init(&bar_wq, 1);
    for (int s = 0; s < kSlots; ++s) mbar_init(&bar_q[s], 1);
    fence_barrier_init();
  }
  if (trainer && tid < p.n_steps) {
    const long long t = *p.t_ctr + tid + 1;
    s_corr[4 * tid] = 1.0f - pow_int(p.b1, t);
    s_corr[4 * tid + 1] = 1.0f - pow_int(p.b2, t);
    s_corr[4 * tid + 2] = 1.0f - pow_int(p.alpha, t);
    s_corr[4 * tid + 3] = 1.0f - pow_int(p.alpha, t - 1);
  }
  if (trainer) {
    // delta_L's rows use 2 of their 8 chunks; the rest (read by dW_{L-1}'s
    // unused half) stays zero
    uint8_t* Hb = sw + ((p.img_bytes + 1023) & ~1023);
    uint4* d = reinterpret_cast<uint4*>(Hb + 7 * 16384);
    for (int k = tid; k < 1024; k += kFrameThreads) d[k] = make_uint4(0u, 0u, 0u, 0u);
    fence_proxy_async_smem();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (trainer)
    frame_train<MODE, BF16>(p, p.tv, int(blockIdx.x), sw, tmem, &bar_w, &bar_mma, &bar_dw, bar_full, bar_free, red,
                            s_corr);

  // ---------------------------------------------------------- query role
  const int64_t n_tiles = (p.n_q + kTile - 1) / kTile;
  fence_before();
  __syncthreads();  // the training role (if any) is done with shared memory and TMEM
  fence_after();
  if (n_tiles > 0) {
    const int slot = tid >> 7;
    const int rit = tid & 127;
    uint8_t* recs = sw + ((p.img_bytes + 1023) & ~1023);
    if (tid == 0) {
      mbar_arrive_expect_tx(&bar_wq, uint32_t(p.img_bytes));
      bulk_g2s(sw, p.qimg, uint32_t(p.img_bytes), &bar_wq);
    }
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
    auto prefetch = [&](int64_t t, int bf) {
      const int64_t row = t * kTile + rit;
      rs.fetch(p.rec, row, t < n_tiles && row < p.n_q, bf);
    };
    // tickets: the first two tiles at once, then one per tile, published in
    // the tile's output layer so that the atomic's latency is hidden
    const int lead_t = 32 * (slot & 3);  // lane 0 of the slot's lead warp (as in tile_layers)
    if (rit == lead_t) s_next[slot] = int(atomicAdd(&p.sync[1], 2u));
    named_sync(1 + slot, 128);
    int64_t cur = s_next[slot];
    int64_t nxt = cur + 1;
    int buf = 0;
    prefetch(cur, buf);
    mbar_wait(&bar_wq, 0, p.err);
    // once every CTA holds the old image (and so every training step is
    // done), the last of them copies the training's images over the cache's
    fence_before();
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      const unsigned old = atomicAdd(&p.sync[3], 1u);
      s_last = old + 1 == gridDim.x && p.n_train > 0 && p.n_steps > 0;
      if (s_last) __threadfence();
    }
    __syncthreads();
    if (s_last) copy_images(p);
    __syncthreads();
    fence_after();
    uint32_t phase = 0;
    // A slot retires when it starts its last tile (its next ticket is past
    // the end, so it draws no more): one count on sync[2].  The slot that
    // retires last over the grid zeroes the counters for the next launch once
    // its tile is done; the launch's end then waits for no atomic.
    const unsigned n_slots_all = gridDim.x * unsigned(kSlots);
    auto reset_counters = [&]() {
      p.sync[0] = 0u;
      p.sync[1] = 0u;
      p.sync[2] = 0u;
      p.sync[3] = 0u;
    };
    if (cur >= n_tiles && rit == lead_t && atomicAdd(&p.sync[2], 1u) + 1u == n_slots_all) reset_counters();
    while (cur < n_tiles) {
      const int64_t row = cur * kTile + rit;
      prefetch(nxt, buf ^ 1);
      int nxt2 = 0;
      unsigned retired = 0u;  // the slot's retire count + 1 (lead thread, last tile)
      if (rit == lead_t) {
        if (nxt < n_tiles) {
          nxt2 = int(atomicAdd(&p.sync[1], 1u));
        } else {
          nxt2 = int(n_tiles);
          retired = atomicAdd(&p.sync[2], 1u) + 1u;
        }
      }
      cp_async_wait<1>();
      float r[kRecFloats];
      rs.read(buf, r);
      const uint8_t* fac_row = p.factor ? rs.p + buf * 8192 : nullptr;
      buf ^= 1;
      encode_to_tmem<MODE, BF16>(r, p.pad, st.t_act);
      tile_layers<BF16>(p.img, p.net.n_mats, st, sw_base, slot, rit, &bar_q[slot], phase, p.err,
                        row < p.n_q ? p.rgb + row * 3 : nullptr, fac_row, rs.rot, [&]() {
                          if (rit == lead_t) s_next[slot] = nxt2;
                        });
      if (retired == n_slots_all) reset_counters();
      cur = nxt;
      nxt = s_next[slot];
    }
    cp_async_wait<0>();
  }

  // ------------------------------------------------------------ retire
  // (with queries the slots retired above)
  fence_before();
  __syncthreads();
  if (tid == 0 && n_tiles == 0) {
    __threadfence();
    const unsigned old = atomicAdd(&p.sync[2], 1u);
    s_last = old + 1 == gridDim.x;
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (n_tiles == 0 && s_last) {
    // every CTA is done: without queries the training's images replace the
    // cache's now; the counters are zero again for the next launch
    if (p.n_train > 0 && p.n_steps > 0) copy_images(p);
    __syncthreads();
    if (tid == 0) {
      p.sync[0] = 0u;
      p.sync[1] = 0u;
      p.sync[2] = 0u;
      p.sync[3] = 0u;
      __threadfence();
    }
  }
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// Batched training with the frame's training role: CTA blockIdx.x trains
// views[blockIdx.x] (one cache of the batch; each cache has its own CTAs,
// partials, barrier counter and weight image, so its result depends only on
// its own partition).  counters[0 .. n_counters-2] are the caches' barrier
// counters, counters[n_counters-1] counts retired CTAs; the last CTA zeroes
// them all for the next launch.  Cooperative launch of at most one CTA per SM.
template <int MODE, bool BF16>
__global__ void __launch_bounds__(kFrameThreads, 1)
    k_train_views(const __grid_constant__ FrameParams p, const TrainView* __restrict__ views, unsigned* counters,
                  int n_counters) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_w, bar_mma, bar_dw, bar_full[2], bar_free[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ float red[16];
  __shared__ int s_last;
  __shared__ float s_corr[4 * kFrameMaxSteps];
  uint8_t* sw = align1024(smem_raw);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const TrainView tv = views[blockIdx.x];
  if (warp == 0) {
    tmem_alloc(&tmem_base_sh, kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar_w, 1);
    mbar_init(&bar_mma, 1);
    mbar_init(&bar_dw, 1);
    mbar_init(&bar_full[0], kProducerThreads);
    mbar_init(&bar_full[1], kProducerThreads);
    mbar_init(&bar_free[0], 1);
    mbar_init(&bar_free[1], 1);
    fence_barrier_init();
  }
  if (tid < p.n_steps) {
    const long long t = *tv.t_ctr + tid + 1;
    s_corr[4 * tid] = 1.0f - pow_int(p.b1, t);
    s_corr[4 * tid + 1] = 1.0f - pow_int(p.b2, t);
    s_corr[4 * tid + 2] = 1.0f - pow_int(p.alpha, t);
    s_corr[4 * tid + 3] = 1.0f - pow_int(p.alpha, t - 1);
  }
  {
    uint8_t* Hb = sw + ((p.img_bytes + 1023) & ~1023);
    uint4* d = reinterpret_cast<uint4*>(Hb + 7 * 16384);
    for (int k = tid; k < 1024; k += kFrameThreads) d[k] = make_uint4(0u, 0u, 0u, 0u);
    fence_proxy_async_smem();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_sh;
  frame_train<MODE, BF16>(p, tv, tv.b, sw, tmem, &bar_w, &bar_mma, &bar_dw, bar_full, bar_free, red, s_corr);
  fence_before();
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned old = atomicAdd(&counters[n_counters - 1], 1u);
    s_last = old + 1 == gridDim.x;
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (s_last) {
    for (int k = tid; k < n_counters; k += kFrameThreads) counters[k] = 0u;
    __threadfence();
  }
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// Shared constants of a batched training launch: the configuration of the
// batch's caches (all equal), n_steps steps, the first cache's error word.
static void train_views_params(const Cache* proto, int n_steps, FrameParams* p) {
  std::memset(p, 0, sizeof(*p));
  p->n_steps = n_steps;
  p->net = proto->net;
  p->img = proto->img;
  p->img_bytes = int(proto->img.off[proto->net.n_mats]);
  p->pad = proto->cfg.pad_value;
  p->loss_mode = proto->cfg.loss_mode;
  p->loss_eps = proto->cfg.loss_eps;
  p->factor = proto->cfg.refl_factor;
  p->lr = proto->cfg.lr;
  p->b1 = proto->cfg.beta1;
  p->b2 = proto->cfg.beta2;
  p->eps = proto->cfg.adam_eps;
  p->alpha = proto->cfg.ema_alpha;
  p->err = proto->err;
}

bool train_views_ok(const Cache* proto) {
  const nrc_config& k = proto->cfg;
  return k.path == NRC_PATH_FUSED && (k.dtype == NRC_FP16 || k.dtype == NRC_BF16) && k.optimizer == NRC_OPT_ADAM &&
         k.width == 64 && proto->net.n_mats <= kFrameMaxMats;
}

cudaError_t launch_train_views(const Cache* proto, const TrainView* views, int n_views, unsigned* counters,
                               int n_counters, int n_steps, cudaStream_t st) {
  if (!train_views_ok(proto) || n_views < 1 || n_views > proto->sm_count || n_steps < 1 || n_steps > kFrameMaxSteps)
    return cudaErrorInvalidValue;
  FrameParams p;
  train_views_params(proto, n_steps, &p);
  const int align = 1024;
  const int img_alloc = (p.img_bytes + 1023) & ~1023;
  const int smem = img_alloc + kFrameBufs * 16384 + 2 * kTile * 8 * 4 + align;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(unsigned(n_views));
  lc.blockDim = dim3(kFrameThreads);
  lc.dynamicSmemBytes = size_t(smem);
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  const bool bf16 = proto->cfg.dtype == NRC_BF16;
  const int mode = proto->cfg.enc_mode;
  cudaError_t e = cudaSuccess;
  static std::atomic<int> attr_done[4];
#define NRC_LAUNCH(M, B)                                                            \
  e = ensure_smem(k_train_views<M, B>, smem, &attr_done[2 * (M) + ((B) ? 1 : 0)]); \
  if (e != cudaSuccess) return e;                                                   \
  e = cudaLaunchKernelEx(&lc, k_train_views<M, B>, p, views, counters, n_counters);  \
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

// Training CTAs of a frame: the split that minimises a model of the frame's
// length.  A query tile costs about kQueryTileSmUs SM-microseconds; a CTA's
// training tile about kTrainTileUs of dependent chain, a step's write-out,
// reduction, Adam and barriers about kStepUs (measured on GB300 at 2.07 GHz
// with %clock64 stamps).  The frame lasts at least the training's chain and
// at least the total SM time over the grid.
constexpr double kQueryTileSmUs = 0.88;
constexpr double kTrainTileUs = 8.8;
constexpr double kStepUs = 7.7;

int frame_split(const Cache* c, int64_t n_q, int64_t batch, int n_steps) {
  const int64_t tiles = (batch + kTile - 1) / kTile;
  const int cap = int(std::min<int64_t>(tiles, c->sm_count));
  if (n_q <= 0) return cap;
  const double qsm = double((n_q + kTile - 1) / kTile) * kQueryTileSmUs;
  int best = 1;
  double best_t = 1e30;
  for (int T = 1; T <= cap; ++T) {
    const double chain = n_steps * (double((tiles + T - 1) / T) * kTrainTileUs + kStepUs);
    const double t = std::max(chain, (qsm + T * chain) / c->sm_count);
    if (t < best_t - 1e-9) {
      best_t = t;
      best = T;
    }
  }
  return best;
}

cudaError_t launch_frame_tc(Cache* c, const float* rec, int64_t n_q, float* rgb, const float* pool, const float* target,
                            int64_t n_pool, int64_t batch, int n_steps, uint64_t a, uint64_t cc, float* loss_out,
                            int n_train, cudaStream_t st) {
  if (c->net.n_mats > kFrameMaxMats || c->cfg.width != 64) return cudaErrorNotSupported;
  const size_t img_bytes = size_t(c->img.off[c->net.n_mats]);
  cudaError_t e = cudaSuccess;
  if (!c->frame_sync) {  // set-up on first use (resumable: each buffer is made once)
    if (!c->wimg_work) {
      e = dev_alloc(&c->wimg_work, img_bytes + 1024);
      if (e == cudaSuccess) e = cudaMemsetAsync(c->wimg_work, 0, img_bytes + 1024, st);
    }
    if (e == cudaSuccess && c->cfg.ema && !c->wimg_ema_work) {
      e = dev_alloc(&c->wimg_ema_work, img_bytes + 1024);
      if (e == cudaSuccess) e = cudaMemsetAsync(c->wimg_ema_work, 0, img_bytes + 1024, st);
    }
    unsigned* sync = nullptr;
    if (e == cudaSuccess) e = dev_alloc(&sync, 64);
    if (e == cudaSuccess) e = cudaMemsetAsync(sync, 0, 64, st);
    if (e != cudaSuccess) {
      cudaFree(sync);
      return e;
    }
    c->frame_sync = sync;
  }
  const int64_t tiles = (batch + kTile - 1) / kTile;
  const int T = (n_steps > 0 && batch > 0) ? int(std::max<int64_t>(1, std::min<int64_t>(n_train, tiles))) : 0;
  if (T > c->sm_count) return cudaErrorInvalidValue;
  e = ensure_partials(c, std::max(T, 1));
  if (e != cudaSuccess) return e;
  FrameParams p;
  std::memset(&p, 0, sizeof(p));
  p.rec = rec;
  p.n_q = n_q;
  p.rgb = rgb;
  p.qimg = query_image(c);
  p.pool = pool;
  p.target = target;
  p.n_pool = n_pool;
  p.batch = batch;
  p.a = a;
  p.c = cc;
  p.n_steps = T > 0 ? n_steps : 0;
  p.n_train = T;
  p.loss_out = loss_out;
  p.w = c->w;
  p.m = c->m;
  p.v = c->v;
  p.t_ctr = c->t;
  p.ema = c->cfg.ema ? c->ema : nullptr;
  p.img_in = c->wimg;
  p.img_work = c->wimg_work;
  p.img_ema_work = c->wimg_ema_work;
  p.img_out = c->wimg;
  p.img_ema_out = c->wimg_ema;
  p.partials = c->partials;
  p.sync = c->frame_sync;
  p.net = c->net;
  p.img = c->img;
  p.img_bytes = int(img_bytes);
  p.pad = c->cfg.pad_value;
  p.loss_mode = c->cfg.loss_mode;
  p.loss_eps = c->cfg.loss_eps;
  p.factor = c->cfg.refl_factor;
  p.inv3n = batch > 0 ? float(1.0 / (3.0 * double(batch))) : 0.0f;
  p.lr = c->cfg.lr;
  p.b1 = c->cfg.beta1;
  p.b2 = c->cfg.beta2;
  p.eps = c->cfg.adam_eps;
  p.alpha = c->cfg.ema_alpha;
  p.err = c->err;
  TrainView& tv = p.tv;
  tv.pool = p.pool;
  tv.target = p.target;
  tv.n_pool = p.n_pool;
  tv.batch = p.batch;
  tv.a = p.a;
  tv.c = p.c;
  tv.seed = nullptr;
  tv.step0 = 0;
  tv.T = p.n_train;
  tv.b = 0;
  tv.w = p.w;
  tv.m = p.m;
  tv.v = p.v;
  tv.ema = p.ema;
  tv.t_ctr = p.t_ctr;
  tv.img_in = p.img_in;
  tv.img_work = p.img_work;
  tv.img_ema_work = p.img_ema_work;
  tv.partials = p.partials;
  tv.bar = p.sync;
  tv.loss_out = p.loss_out;
  tv.inv3n = p.inv3n;
  const int align = 1024;
  const int img_alloc = (p.img_bytes + 1023) & ~1023;
  const int smem_train = img_alloc + kFrameBufs * 16384 + 2 * kTile * 8 * 4 + align;
  const int smem_query = img_alloc + kSlots * 2 * 8192 + align;
  const int smem = std::max(smem_train, smem_query);
  const unsigned grid = n_q > 0 ? unsigned(c->sm_count) : unsigned(T);
  if (grid == 0) return cudaSuccess;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(kFrameThreads);
  lc.dynamicSmemBytes = size_t(smem);
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  const bool bf16 = c->cfg.dtype == NRC_BF16;
  const int mode = c->cfg.enc_mode;
  static std::atomic<int> attr_done[4];
#define NRC_LAUNCH(M, B)                                                         \
  e = ensure_smem(k_frame_tc<M, B>, smem, &attr_done[2 * (M) + ((B) ? 1 : 0)]); \
  if (e != cudaSuccess) return e;                                                \
  e = cudaLaunchKernelEx(&lc, k_frame_tc<M, B>, p);                              \
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

}  // namespace nrc
