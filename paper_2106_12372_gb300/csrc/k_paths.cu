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

// spread term of vertex j >= 1: sqrt(|x_{j-1} - x_j|^2 / (pdf_j |cos_j|))
__device__ __forceinline__ float spread_term(const float* v, int j) {
  const float* a = v + (j - 1) * kVtx;
  const float* b = v + j * kVtx;
  return __fsqrt_rn(__fdiv_rn(d2_rn(a, b), __fmul_rn(b[14], b[15])));
}

__device__ __forceinline__ float spread_threshold(const float* v, const float* cam, float c) {
  const float a0 = __fdiv_rn(d2_rn(v, cam), __fmul_rn(kFourPi, v[15]));
  return __fmul_rn(c, a0);
}

// index of the rendering path's terminal vertex
__device__ __forceinline__ int render_end(const float* v, int K, float thr) {
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

__global__ void k_paths_render(const __grid_constant__ PathsArgs a, float* __restrict__ rq, float* __restrict__ emitted,
                               float* __restrict__ throughput) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= int64_t(a.width) * a.height) return;
  const float* v = a.vtx + p * a.K * kVtx;
  const int n = render_end(v, a.K, spread_threshold(v, a.cam, a.c));
  float T[3] = {1.0f, 1.0f, 1.0f}, E[3] = {0.0f, 0.0f, 0.0f};
  for (int j = 0; j <= n; ++j) {
    const float* vj = v + j * kVtx;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) E[ch] = fmaf(T[ch], vj[16 + ch], E[ch]);
    if (j < n) {
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) T[ch] *= vj[19 + ch];
    }
  }
  write_record(rq + p * kRecFloats, v + n * kVtx);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    emitted[p * 3 + ch] = E[ch];
    throughput[p * 3 + ch] = T[ch];
  }
}

// tiles[t] = {pixel (-1: none), n, m, unbiased}; the tail query of a training path
__global__ void k_paths_tiles(const __grid_constant__ PathsArgs a, int* __restrict__ tiles, float* __restrict__ tq) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_tiles) return;
  const int ty = t / a.tiles_x, tx = t % a.tiles_x;
  const int px = tx * a.tile + a.ox, py = ty * a.tile + a.oy;
  int4 info = make_int4(-1, 0, 0, 0);
  if (px < a.width && py < a.height) {
    const int64_t p = int64_t(py) * a.width + px;
    const float* v = a.vtx + p * a.K * kVtx;
    const float thr = spread_threshold(v, a.cam, a.c);
    const int n = render_end(v, a.K, thr);
    const bool unb = a.phase >= 0 && t % 16 == a.phase;
    int m = a.K - 1;
    if (unb) {
      for (int j = n; j < a.K; ++j)
        if (j == a.K - 1 || !(v[j * kVtx + 22] < a.q)) {
          m = j;
          break;
        }
    } else {
      float acc = 0.0f;
      for (int j = n + 1; j < a.K; ++j) {
        acc = __fadd_rn(acc, spread_term(v, j));
        if (__fmul_rn(acc, acc) > thr) {
          m = j;
          break;
        }
      }
    }
    info = make_int4(int(p), n, m, unb ? 1 : 0);
    write_record(tq + int64_t(t) * kRecFloats, v + m * kVtx);
  }
  reinterpret_cast<int4*>(tiles)[t] = info;
}

// Exclusive scan of the records per training path (m of them) in tile order;
// one block, so the order -- and the pool layout -- is fixed.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_paths_scan(const int* __restrict__ tiles, int n_tiles,
                                                             int64_t* __restrict__ offsets, int64_t* __restrict__ count) {
  __shared__ int64_t part[kScanThreads];
  const int per = (n_tiles + kScanThreads - 1) / kScanThreads;
  const int b = threadIdx.x * per, e = min(n_tiles, b + per);
  int64_t s = 0;
  for (int t = b; t < e; ++t) s += tiles[4 * t] >= 0 ? tiles[4 * t + 2] : 0;
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < kScanThreads; off <<= 1) {  // inclusive Hillis-Steele scan of the chunk sums
    const int64_t add = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  int64_t run = part[threadIdx.x] - s;
  for (int t = b; t < e; ++t) {
    offsets[t] = run;
    run += tiles[4 * t] >= 0 ? tiles[4 * t + 2] : 0;
  }
  if (threadIdx.x == kScanThreads - 1) *count = part[kScanThreads - 1];
}

__global__ void k_paths_targets(const __grid_constant__ PathsArgs a, const int* __restrict__ tiles,
                                const int64_t* __restrict__ offsets, const float* __restrict__ tail_rgb,
                                float* __restrict__ pool, float* __restrict__ targets, int64_t max_records) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_tiles) return;
  const int4 info = reinterpret_cast<const int4*>(tiles)[t];
  if (info.x < 0) return;
  const float* v = a.vtx + int64_t(info.x) * a.K * kVtx;
  const int n = info.y, m = info.z;
  const bool unb = info.w != 0;
  float L[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) L[ch] = unb ? 0.0f : tail_rgb[t * 3 + ch];
  const float inv_q = 1.0f / a.q;
  const int64_t base = offsets[t];
  for (int j = m - 1; j >= 0; --j) {
    const float* vj = v + j * kVtx;
    const float* vn = vj + kVtx;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float w = vj[19 + ch];
      if (unb && j >= n) w *= inv_q;
      L[ch] = w * (vn[16 + ch] + L[ch]);
    }
    const int64_t r = base + j;
    if (r < max_records) {
      write_record(pool + r * kRecFloats, vj);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) targets[r * 3 + ch] = L[ch];
    }
  }
}

__global__ void k_paths_composite(const float* __restrict__ emitted, const float* __restrict__ throughput,
                                  const float* __restrict__ rgb, int64_t n3, float* __restrict__ image) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n3) image[i] = fmaf(throughput[i], rgb[i], emitted[i]);
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
  k_paths_render<<<unsigned((P + 255) / 256), 256, 0, st>>>(a, render_queries, render_emitted, render_throughput);
  k_paths_tiles<<<unsigned((a.n_tiles + 255) / 256), 256, 0, st>>>(a, tiles, tail_queries);
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
  k_paths_scan<<<1, kScanThreads, 0, st>>>(tiles, a.n_tiles, offsets, count);
  k_paths_targets<<<unsigned((a.n_tiles + 255) / 256), 256, 0, st>>>(a, tiles, offsets, tail_rgb, pool, targets,
                                                                    max_records);
  return cuda_status(cudaGetLastError(), "nrc_paths_records");
}

nrc_status nrc_paths_composite(const float* emitted, const float* throughput, const float* rgb, int64_t n,
                               float* image, nrc_stream stream) {
  if (n < 0) return set_error("nrc_paths_composite: n < 0"), NRC_ERR_INVALID_ARG;
  if (n == 0) return NRC_OK;
  if (!emitted || !throughput || !rgb || !image) return set_error("nrc_paths_composite: NULL argument"), NRC_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_paths_composite<<<unsigned((3 * n + 255) / 256), 256, 0, st>>>(emitted, throughput, rgb, 3 * n, image);
  return cuda_status(cudaGetLastError(), "nrc_paths_composite");
}

}  // extern "C"
