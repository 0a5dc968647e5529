// Training-record pipeline around the cache query (Sec. 3.3-3.5; the path
// termination heuristic of Sec. 3.4, Eqs. 3-4), on path vertices of 24 floats
// (layout in include/nrc.h).  Per pixel: the rendering path ends at the first
// vertex x_n (n >= 2) whose area spread a(x_1..x_n) = (sum_i sqrt(|x_{i-1} -
// x_i|^2 / (pdf_i |cos_i|)))^2 exceeds c a_0, a_0 = |x_0 - x_1|^2 / (4 pi
// cos_1); its record is the cache query, and the emitted light along the path
// and the throughput to x_n are kept for the pixel composite.  Per screen tile
// one pixel (at a per-frame offset) is a training path: its suffix restarts the
// spread sum at x_n and ends at the first x_m with a(x_n..x_m) > c a_0, or --
// every 16th tile -- continues from each vertex with probability q only
// (Russian roulette, the bounce weighted by 1/q).  The self-training targets
// transport the cache's value at x_m (0 where the roulette ended the path)
// back to x_0..x_{m-1} (Sec. 3.3).  The termination decisions use
// round-to-nearest FP32 operations in a fixed order, so any implementation of
// the same order takes the same decisions.
#include <cmath>

#include "nrc_internal.cuh"

namespace nrc {

constexpr int kVtx = 24;  // floats per path vertex
constexpr float kFourPi = 12.566370614359172f;

__device__ __forceinline__ float d2_rn(const float* a, const float* b) {
  const float dx = __fsub_rn(a[0], b[0]), dy = __fsub_rn(a[1], b[1]), dz = __fsub_rn(a[2], b[2]);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// A path whose vertices 0 and 1 are staged in shared memory (the rest stays in
// global memory).
struct StagedPath {
  const float* s;
  const float* g;
  __device__ __forceinline__ const float* operator()(int j) const { return j < 2 ? s + j * kVtx : g + j * kVtx; }
};

// spread term of vertex j >= 1: sqrt(|x_{j-1} - x_j|^2 / (pdf_j |cos_j|))
template <class V>
__device__ __forceinline__ float spread_term(const V& v, int j) {
  const float* a = v(j - 1);
  const float* b = v(j);
  return __fsqrt_rn(__fdiv_rn(d2_rn(a, b), __fmul_rn(b[14], b[15])));
}

template <class V>
__device__ __forceinline__ float spread_threshold(const V& v, const float* cam, float c) {
  const float* x0 = v(0);
  const float a0 = __fdiv_rn(d2_rn(x0, cam), __fmul_rn(kFourPi, x0[15]));
  return __fmul_rn(c, a0);
}

// index of the rendering path's terminal vertex
template <class V>
__device__ __forceinline__ int render_end(const V& v, int K, float thr) {
  float acc = 0.0f;
  for (int j = 1; j < K; ++j) {
    acc = __fadd_rn(acc, spread_term(v, j));
    if (__fmul_rn(acc, acc) > thr) return j;
  }
  return K - 1;
}

__device__ __forceinline__ void write_record(float* dst, const float* vj) {
  float4* d = reinterpret_cast<float4*>(dst);
  d[0] = make_float4(vj[0], vj[1], vj[2], vj[3]);
  d[1] = make_float4(vj[4], vj[5], vj[6], vj[7]);
  d[2] = make_float4(vj[8], vj[9], vj[10], vj[11]);
  d[3] = make_float4(vj[12], vj[13], 0.0f, 0.0f);
}

struct PathsArgs {
  const float* vtx;
  int width, height, K;
  float cam[3];
  float c;
  int tile, ox, oy, phase;
  float q;
  int tiles_x, n_tiles;
};

// End of a training path's suffix from x_n (Sec. 3.4/3.5): the first x_m
// past the spread threshold (the sum restarted at x_n), or -- for a
// roulette-only suffix -- where the roulette stops it.
template <class V>
__device__ __forceinline__ int suffix_end(const V& v, int K, float thr, int n, bool unb, float q) {
  if (unb) {
    for (int j = n; j < K; ++j)
      if (j == K - 1 || !(v(j)[22] < q)) return j;
    return K - 1;
  }
  float acc = 0.0f;
  for (int j = n + 1; j < K; ++j) {
    acc = __fadd_rn(acc, spread_term(v, j));
    if (__fmul_rn(acc, acc) > thr) return j;
  }
  return K - 1;
}

// One warp per 32 consecutive pixels.  Vertices 0 and 1 of its pixels (the
// first 192 bytes of each path; the rendering path ends at vertex 1 for most
// pixels) are staged in shared memory with coalesced 16-byte loads, and the
// outputs leave through the same buffer as contiguous stores; vertices past 1
// are read from global memory.
constexpr int kRenderWarps = 4;
constexpr int kStageStride = 2 * kVtx + 1;  // odd: lane t's floats fall in distinct banks
constexpr int kOutStride = kRecFloats + 1;

__global__ void __launch_bounds__(kRenderWarps * 32)
    k_paths_render(const __grid_constant__ PathsArgs a, float* __restrict__ rq, float* __restrict__ emitted,
                   float* __restrict__ throughput, int* __restrict__ tiles, float* __restrict__ tq) {
  __shared__ float stage[kRenderWarps][32 * kStageStride];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t P = int64_t(a.width) * a.height;
  const int64_t p0 = (int64_t(blockIdx.x) * kRenderWarps + warp) * 32;
  if (p0 >= P) return;  // the whole warp
  const int valid = P - p0 < 32 ? int(P - p0) : 32;
  const int64_t path_floats = int64_t(a.K) * kVtx;
  {  // a tile whose training pixel lies outside the image has no training path
    const int64_t g = p0 + lane;
    if (g < a.n_tiles) {
      const int ty = int(g / a.tiles_x), tx = int(g - int64_t(ty) * a.tiles_x);
      if (tx * a.tile + a.ox >= a.width || ty * a.tile + a.oy >= a.height)
        reinterpret_cast<int4*>(tiles)[g] = make_int4(-1, 0, 0, 0);
    }
  }
  float* sm = stage[warp];
  {  // 12 float4 per pixel = vertices 0 and 1; all of a lane's loads in flight at once
    float4 x[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const int i = lane + 32 * k, pix = i / 12, q = i - pix * 12;
      if (i < valid * 12) x[k] = __ldcs(reinterpret_cast<const float4*>(a.vtx + (p0 + pix) * path_floats) + q);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const int i = lane + 32 * k, pix = i / 12, q = i - pix * 12;
      if (i < valid * 12) {
        float* d = sm + pix * kStageStride + q * 4;
        d[0] = x[k].x;
        d[1] = x[k].y;
        d[2] = x[k].z;
        d[3] = x[k].w;
      }
    }
  }
  __syncwarp();
  float rec[14], E[3] = {0.0f, 0.0f, 0.0f}, T[3] = {1.0f, 1.0f, 1.0f};
  if (lane < valid) {
    const StagedPath v{sm + lane * kStageStride, a.vtx + (p0 + lane) * path_floats};
    const float thr = spread_threshold(v, a.cam, a.c);
    const int n = render_end(v, a.K, thr);
    // the training pixel of its tile: the tile's entry and the tail's query record
    const int64_t p = p0 + lane;
    const int py = int(p / a.width), px = int(p - int64_t(py) * a.width);
    if (px >= a.ox && py >= a.oy && (px - a.ox) % a.tile == 0 && (py - a.oy) % a.tile == 0) {
      const int t = ((py - a.oy) / a.tile) * a.tiles_x + (px - a.ox) / a.tile;
      const bool unb = a.phase >= 0 && t % 16 == a.phase;
      const int m = suffix_end(v, a.K, thr, n, unb, a.q);
      reinterpret_cast<int4*>(tiles)[t] = make_int4(int(p), n, m, unb ? 1 : 0);
      write_record(tq + int64_t(t) * kRecFloats, v(m));
    }
    for (int j = 0; j <= n; ++j) {
      const float* vj = v(j);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) E[ch] = fmaf(T[ch], vj[16 + ch], E[ch]);
      if (j < n) {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) T[ch] *= vj[19 + ch];
      }
    }
    const float* vn = v(n);
#pragma unroll
    for (int q = 0; q < 14; ++q) rec[q] = vn[q];
  }
  __syncwarp();
  // outputs: records [32][kOutStride], then emitted [32][3], then throughput [32][3]
  float* so = sm + 32 * kOutStride;
  if (lane < valid) {
#pragma unroll
    for (int q = 0; q < 14; ++q) sm[lane * kOutStride + q] = rec[q];
    sm[lane * kOutStride + 14] = 0.0f;
    sm[lane * kOutStride + 15] = 0.0f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      so[lane * 3 + ch] = E[ch];
      so[96 + lane * 3 + ch] = T[ch];
    }
  }
  __syncwarp();
  for (int i = lane; i < valid * 4; i += 32) {
    const int pix = i >> 2, q = i & 3;
    const float* src = sm + pix * kOutStride + q * 4;
    reinterpret_cast<float4*>(rq + (p0 + pix) * kRecFloats)[q] = make_float4(src[0], src[1], src[2], src[3]);
  }
  for (int i = lane; i < valid * 3; i += 32) {
    emitted[p0 * 3 + i] = so[i];
    throughput[p0 * 3 + i] = so[96 + i];
  }
}

// Exclusive scan of the records per training path (m of them) in tile order,
// in two launches over blocks of kScanTiles tiles: the first writes each
// block's total after the offsets, the second adds the totals of the blocks
// before it to its own block-local scan.  A block loads its tiles coalesced and
// transposes them through shared memory, so that each thread scans
// kScanItems consecutive tiles.  Integer sums: the result is exact.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTiles = kScanThreads * kScanItems;

__device__ __forceinline__ int tile_records(const int* tiles, int t, int n_tiles) {
  if (t >= n_tiles) return 0;
  const int4 info = reinterpret_cast<const int4*>(tiles)[t];
  return info.x >= 0 ? info.z : 0;
}

// inclusive scan of one value per thread over the block; *total gets the sum
__device__ __forceinline__ int64_t block_scan(int64_t x, int64_t* wsum, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  int64_t before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kScanThreads / 32; ++w) {
    const int64_t v = wsum[w];
    before += w < warp ? v : 0;
    all += v;
  }
  *total = all;
  return before + x;
}

__global__ void __launch_bounds__(kScanThreads) k_paths_block_sums(const int* __restrict__ tiles, int n_tiles,
                                                                   int64_t* __restrict__ sums) {
  __shared__ int64_t wsum[kScanThreads / 32];
  const int base = blockIdx.x * kScanTiles;
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) s += tile_records(tiles, base + i * kScanThreads + threadIdx.x, n_tiles);
  int64_t total;
  block_scan(s, wsum, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_paths_scan(const int* __restrict__ tiles, int n_tiles,
                                                             const int64_t* __restrict__ sums,
                                                             int64_t* __restrict__ offsets, int64_t* __restrict__ count) {
  __shared__ int64_t buf[kScanThreads * (kScanItems + 1)];  // element e at e + e / kScanItems
  __shared__ int64_t wsum[kScanThreads / 32];
  __shared__ int64_t base_sh;
  const int tid = threadIdx.x;
  const int base = blockIdx.x * kScanTiles;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int e = i * kScanThreads + tid;
    buf[e + e / kScanItems] = tile_records(tiles, base + e, n_tiles);
  }
  if (tid < 32) {  // the totals of the blocks before this one
    int64_t b = 0;
    for (int k = tid; k < int(blockIdx.x); k += 32) b += sums[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) b += __shfl_down_sync(0xffffffffu, b, off);
    if (tid == 0) base_sh = b;
  }
  __syncthreads();
  int64_t* mine = buf + tid * (kScanItems + 1);
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t x = mine[k];
    mine[k] = s;
    s += x;
  }
  int64_t total;
  const int64_t incl = block_scan(s, wsum, &total);
  const int64_t before = base_sh + incl - s;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) mine[k] += before;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int e = i * kScanThreads + tid, t = base + e;
    if (t < n_tiles) offsets[t] = buf[e + e / kScanItems];
  }
  if (blockIdx.x == gridDim.x - 1 && tid == 0) *count = base_sh + total;
}

// One thread per (training path, vertex j < m): the target of record j is the
// transport recurrence L_k = w_k (Le_{k+1} + L_{k+1}) from the tail down to j,
// each thread taking the same operations in the same order as a serial pass.
__global__ void k_paths_targets(const __grid_constant__ PathsArgs a, const int* __restrict__ tiles,
                                const int64_t* __restrict__ offsets, const float* __restrict__ tail_rgb,
                                float* __restrict__ pool, float* __restrict__ targets, int64_t max_records) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= int64_t(a.n_tiles) * a.K) return;
  const int t = int(i / a.K), j = int(i - int64_t(t) * a.K);
  const int4 info = reinterpret_cast<const int4*>(tiles)[t];
  const int n = info.y, m = info.z;
  if (info.x < 0 || j >= m) return;
  const int64_t r = offsets[t] + j;
  if (r >= max_records) return;
  const float* v = a.vtx + int64_t(info.x) * a.K * kVtx;
  const bool unb = info.w != 0;
  float L[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) L[ch] = unb ? 0.0f : tail_rgb[t * 3 + ch];
  const float inv_q = 1.0f / a.q;
  for (int k = m - 1; k >= j; --k) {
    const float* vk = v + k * kVtx;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float w = vk[19 + ch];
      if (unb && k >= n) w *= inv_q;
      L[ch] = w * (vk[kVtx + 16 + ch] + L[ch]);
    }
  }
  write_record(pool + r * kRecFloats, v + j * kVtx);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) targets[r * 3 + ch] = L[ch];
}

__global__ void k_paths_composite(const float* __restrict__ emitted, const float* __restrict__ throughput,
                                  const float* __restrict__ rgb, int64_t n3, float* __restrict__ image) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n3) image[i] = fmaf(throughput[i], rgb[i], emitted[i]);
}

// the same on 16-byte aligned arrays, four floats per thread
__global__ void k_paths_composite4(const float4* __restrict__ emitted, const float4* __restrict__ throughput,
                                   const float4* __restrict__ rgb, int64_t n4, float4* __restrict__ image) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  const float4 e = __ldcs(emitted + i), t = __ldcs(throughput + i), c = __ldcs(rgb + i);
  __stcs(image + i, make_float4(fmaf(t.x, c.x, e.x), fmaf(t.y, c.y, e.y), fmaf(t.z, c.z, e.z), fmaf(t.w, c.w, e.w)));
}

static nrc_status paths_args(const nrc_paths* ps, const nrc_path_params* pr, PathsArgs* a) {
  if (!ps || !pr || !ps->vertices) return set_error("paths: NULL argument"), NRC_ERR_INVALID_ARG;
  if (ps->width <= 0 || ps->height <= 0 || ps->n_vertices < 2 || ps->n_vertices > 64 ||
      int64_t(ps->width) * ps->height > (int64_t(1) << 30))
    return set_error("paths: width, height > 0, 2 <= n_vertices <= 64"), NRC_ERR_INVALID_ARG;
  if (pr->tile < 1 || pr->tile_ox < 0 || pr->tile_ox >= pr->tile || pr->tile_oy < 0 || pr->tile_oy >= pr->tile ||
      pr->unbiased_phase < -1 || pr->unbiased_phase > 15 || !(pr->rr_survive > 0.0f && pr->rr_survive <= 1.0f) ||
      !(pr->c >= 0.0f))
    return set_error("paths: tile >= 1, offsets in [0, tile), unbiased_phase in [-1, 15], rr_survive in (0, 1]"),
           NRC_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ps->vertices) & 15u) return set_error("paths: vertices must be 16-byte aligned"), NRC_ERR_INVALID_ARG;
  a->vtx = ps->vertices;
  a->width = ps->width;
  a->height = ps->height;
  a->K = ps->n_vertices;
  for (int k = 0; k < 3; ++k) a->cam[k] = ps->camera[k];
  a->c = pr->c;
  a->tile = pr->tile;
  a->ox = pr->tile_ox;
  a->oy = pr->tile_oy;
  a->phase = pr->unbiased_phase;
  a->q = pr->rr_survive;
  a->tiles_x = (ps->width + pr->tile - 1) / pr->tile;
  a->n_tiles = a->tiles_x * ((ps->height + pr->tile - 1) / pr->tile);
  return NRC_OK;
}

}  // namespace nrc

using namespace nrc;

extern "C" {

int64_t nrc_paths_tile_count(int32_t width, int32_t height, int32_t tile) {
  if (width <= 0 || height <= 0 || tile < 1) return 0;
  return int64_t((width + tile - 1) / tile) * ((height + tile - 1) / tile);
}

int64_t nrc_paths_offsets_count(int64_t n_tiles) {
  return n_tiles <= 0 ? 0 : n_tiles + (n_tiles + kScanTiles - 1) / kScanTiles;
}

int32_t nrc_paths_adapt_tile(int32_t tile, int64_t generated, int64_t target) {
  if (tile < 1) tile = 1;
  if (generated <= 0 || target <= 0) return tile;
  const double s = double(tile) * std::sqrt(double(generated) / double(target));
  const int32_t r = int32_t(s + 0.5);
  return r < 1 ? 1 : (r > 256 ? 256 : r);
}

nrc_status nrc_paths_terminate(const nrc_paths* paths, const nrc_path_params* params, float* render_queries,
                               float* render_emitted, float* render_throughput, int32_t* tiles, float* tail_queries,
                               nrc_stream stream) {
  PathsArgs a;
  nrc_status s = paths_args(paths, params, &a);
  if (s != NRC_OK) return s;
  if (!render_queries || !render_emitted || !render_throughput || !tiles || !tail_queries)
    return set_error("nrc_paths_terminate: NULL output"), NRC_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(render_queries) | reinterpret_cast<uintptr_t>(tail_queries) |
       reinterpret_cast<uintptr_t>(tiles)) & 15u)
    return set_error("nrc_paths_terminate: record and tile buffers must be 16-byte aligned"), NRC_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t P = int64_t(a.width) * a.height;
  k_paths_render<<<unsigned((P + kRenderWarps * 32 - 1) / (kRenderWarps * 32)), kRenderWarps * 32, 0, st>>>(
      a, render_queries, render_emitted, render_throughput, tiles, tail_queries);
  return cuda_status(cudaGetLastError(), "nrc_paths_terminate");
}

nrc_status nrc_paths_records(const nrc_paths* paths, const nrc_path_params* params, const int32_t* tiles,
                             const float* tail_rgb, float* pool, float* targets, int64_t max_records,
                             int64_t* offsets, int64_t* count, nrc_stream stream) {
  PathsArgs a;
  nrc_status s = paths_args(paths, params, &a);
  if (s != NRC_OK) return s;
  if (!tiles || !tail_rgb || !offsets || !count || max_records < 0 || (max_records > 0 && (!pool || !targets)))
    return set_error("nrc_paths_records: NULL argument or max_records < 0"), NRC_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(pool) | reinterpret_cast<uintptr_t>(tiles)) & 15u)
    return set_error("nrc_paths_records: pool and tiles must be 16-byte aligned"), NRC_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int blocks = int((int64_t(a.n_tiles) + kScanTiles - 1) / kScanTiles);
  if (blocks == 0) {
    const cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int64_t), st);
    return cuda_status(e, "nrc_paths_records");
  }
  int64_t* sums = offsets + a.n_tiles;
  k_paths_block_sums<<<blocks, kScanThreads, 0, st>>>(tiles, a.n_tiles, sums);
  k_paths_scan<<<blocks, kScanThreads, 0, st>>>(tiles, a.n_tiles, sums, offsets, count);
  const int64_t threads = int64_t(a.n_tiles) * a.K;
  if (threads > 0)
    k_paths_targets<<<unsigned((threads + 255) / 256), 256, 0, st>>>(a, tiles, offsets, tail_rgb, pool, targets,
                                                                     max_records);
  return cuda_status(cudaGetLastError(), "nrc_paths_records");
}

nrc_status nrc_paths_composite(const float* emitted, const float* throughput, const float* rgb, int64_t n,
                               float* image, nrc_stream stream) {
  if (n < 0) return set_error("nrc_paths_composite: n < 0"), NRC_ERR_INVALID_ARG;
  if (n == 0) return NRC_OK;
  if (!emitted || !throughput || !rgb || !image) return set_error("nrc_paths_composite: NULL argument"), NRC_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const bool aligned = ((reinterpret_cast<uintptr_t>(emitted) | reinterpret_cast<uintptr_t>(throughput) |
                        reinterpret_cast<uintptr_t>(rgb) | reinterpret_cast<uintptr_t>(image)) & 15u) == 0;
  if (aligned && (3 * n) % 4 == 0)
    k_paths_composite4<<<unsigned((3 * n / 4 + 255) / 256), 256, 0, st>>>(
        reinterpret_cast<const float4*>(emitted), reinterpret_cast<const float4*>(throughput),
        reinterpret_cast<const float4*>(rgb), 3 * n / 4, reinterpret_cast<float4*>(image));
  else
    k_paths_composite<<<unsigned((3 * n + 255) / 256), 256, 0, st>>>(emitted, throughput, rgb, 3 * n, image);
  return cuda_status(cudaGetLastError(), "nrc_paths_composite");
}

}  // extern "C"
