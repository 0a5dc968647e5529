// Batched caches: many independent caches (each its own weights, Adam state
// and target field) queried in one persistent launch and trained in one
// gradient launch plus one Adam launch per step, with a work-unit size chosen
// by measurement (nrc_batch_autotune).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "batch.cuh"

namespace nrc {

static size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// A pinned slot that no copy in flight still reads.
static uint8_t* ring_slot(Batch* b, int* idx) {
  const int i = b->ring;
  b->ring = (b->ring + 1) % kRing;
  cudaEventSynchronize(b->ev[i]);
  *idx = i;
  return b->pinned + size_t(i) * b->slot_bytes;
}

bool batch_same_cfg(const nrc_config& a, const nrc_config& b) {
  return a.width == b.width && a.hidden_layers == b.hidden_layers && a.dtype == b.dtype && a.enc_mode == b.enc_mode &&
         a.loss_mode == b.loss_mode && a.pad_value == b.pad_value && a.lr == b.lr && a.beta1 == b.beta1 &&
         a.beta2 == b.beta2 && a.adam_eps == b.adam_eps && a.loss_eps == b.loss_eps && a.ema == b.ema &&
         (!a.ema || a.ema_alpha == b.ema_alpha) && a.refl_factor == b.refl_factor;
}

nrc_status batch_check(nrc_cache* const* caches, int n_caches) {
  for (int c = 0; c < n_caches; ++c) {
    if (!caches[c]) return set_error("batched caches: cache %d is NULL", c), NRC_ERR_INVALID_ARG;
    if (caches[c]->cfg.dtype != NRC_FP16 && caches[c]->cfg.dtype != NRC_BF16)
      return set_error("batched caches compute in FP16 or BF16"), NRC_ERR_UNSUPPORTED;
    if (caches[c]->cfg.width != 64 || caches[c]->cfg.path != NRC_PATH_FUSED)
      return set_error("batched caches take the fused width-64 network"), NRC_ERR_UNSUPPORTED;
    if (caches[c]->cfg.optimizer != NRC_OPT_ADAM)
      return set_error("batched caches train with Adam"), NRC_ERR_UNSUPPORTED;
    if (!batch_same_cfg(caches[c]->cfg, caches[0]->cfg))
      return set_error("batched caches: cache %d differs in configuration from cache 0", c), NRC_ERR_INVALID_ARG;
    if (caches[c]->device != caches[0]->device)
      return set_error("batched caches live on different devices"), NRC_ERR_INVALID_ARG;
  }
  return NRC_OK;
}

static size_t slot_size(const Batch* b) {
  return up256(sizeof(BatchCache) * b->max_caches) + up256(sizeof(BatchUnit) * b->max_units) +
         up256(sizeof(TrainJob) * b->max_jobs) + up256(sizeof(AdamJob) * b->max_caches) +
         up256(sizeof(int) * (b->sm_count + 1)) + up256(sizeof(TrainView) * b->max_jobs);
}
// where a ring slot keeps the static query ranges' unit offsets
static size_t uoff_offset(const Batch* b) {
  return up256(sizeof(BatchCache) * b->max_caches) + up256(sizeof(BatchUnit) * b->max_units) +
         up256(sizeof(TrainJob) * b->max_jobs) + up256(sizeof(AdamJob) * b->max_caches);
}
// where a ring slot keeps the training views
static size_t views_offset(const Batch* b) { return slot_size(b) - up256(sizeof(TrainView) * b->max_jobs); }

void batch_free(Batch* b) {
  cudaFree(b->d_caches);
  cudaFree(b->d_units);
  cudaFree(b->d_counter);
  cudaFree(b->d_jobs);
  cudaFree(b->d_adam);
  cudaFree(b->d_views);
  cudaFree(b->d_uoff);
  cudaFree(b->d_tcounters);
  cudaFree(b->d_partials);
  cudaFreeHost(b->pinned);
  for (int i = 0; i < kRing; ++i)
    if (b->ev[i]) cudaEventDestroy(b->ev[i]);
  b->d_caches = nullptr;
  b->d_units = nullptr;
  b->d_counter = nullptr;
  b->d_jobs = nullptr;
  b->d_adam = nullptr;
  b->d_partials = nullptr;
  b->pinned = nullptr;
  for (int i = 0; i < kRing; ++i) b->ev[i] = nullptr;
}

nrc_status batch_init(Batch* b, const nrc_cache* proto, int max_caches) {
  b->sm_count = proto->sm_count;
  b->max_caches = max_caches;
  b->max_jobs = b->sm_count;
  b->max_units = 1 << 16;
  b->stride = partial_stride(proto->net.n_params);
  b->slot_bytes = slot_size(b);
  cudaError_t e = dev_alloc(&b->d_caches, sizeof(BatchCache) * max_caches);
  if (e == cudaSuccess) e = dev_alloc(&b->d_units, sizeof(BatchUnit) * b->max_units);
  if (e == cudaSuccess) e = dev_alloc(&b->d_counter, sizeof(unsigned));
  if (e == cudaSuccess) e = dev_alloc(&b->d_jobs, sizeof(TrainJob) * b->max_jobs);
  if (e == cudaSuccess) e = dev_alloc(&b->d_adam, sizeof(AdamJob) * max_caches);
  if (e == cudaSuccess) e = dev_alloc(&b->d_views, sizeof(TrainView) * b->max_jobs);
  if (e == cudaSuccess) e = dev_alloc(&b->d_uoff, sizeof(int) * (b->sm_count + 1));
  if (e == cudaSuccess) e = dev_alloc(&b->d_tcounters, sizeof(unsigned) * (max_caches + 1));
  if (e == cudaSuccess) e = cudaMemset(b->d_tcounters, 0, sizeof(unsigned) * (max_caches + 1));
  if (e == cudaSuccess) e = dev_alloc(&b->d_partials, size_t(b->max_jobs) * b->stride * 4);
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&b->pinned), b->slot_bytes * kRing, cudaHostAllocDefault);
  for (int i = 0; i < kRing && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    nrc_status s = cuda_status(e, "batched caches: allocation");
    batch_free(b);
    return s;
  }
  return NRC_OK;
}

// Room for n_jobs training CTAs.  Growing waits for the work in flight on st
// (the only stream these buffers are used on) and for the pinned ring.
static nrc_status reserve_jobs(Batch* b, int n_jobs, cudaStream_t st) {
  if (n_jobs <= b->max_jobs) return NRC_OK;
  cudaError_t e = cudaStreamSynchronize(st);
  for (int i = 0; i < kRing && e == cudaSuccess; ++i) e = cudaEventSynchronize(b->ev[i]);
  if (e != cudaSuccess) return cuda_status(e, "batched training: growing the job buffers");
  cudaFree(b->d_jobs);
  cudaFree(b->d_views);
  cudaFree(b->d_partials);
  cudaFreeHost(b->pinned);
  b->d_jobs = nullptr;
  b->d_views = nullptr;
  b->d_partials = nullptr;
  b->pinned = nullptr;
  b->h_jobs.clear();
  b->h_views.clear();
  b->max_jobs = n_jobs;
  b->slot_bytes = slot_size(b);
  e = dev_alloc(&b->d_jobs, sizeof(TrainJob) * b->max_jobs);
  if (e == cudaSuccess) e = dev_alloc(&b->d_views, sizeof(TrainView) * b->max_jobs);
  if (e == cudaSuccess) e = dev_alloc(&b->d_partials, size_t(b->max_jobs) * b->stride * 4);
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&b->pinned), b->slot_bytes * kRing, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    b->max_jobs = 0;
    return cuda_status(e, "batched training: growing the job buffers");
  }
  return NRC_OK;
}

nrc_status batch_infer(Batch* b, nrc_cache* const* caches, int nc, const float* const* records, const int64_t* n,
                       float* const* rgb, cudaStream_t st) {
  if (!records || !n || !rgb) return set_error("batched query: NULL argument"), NRC_ERR_INVALID_ARG;
  if (nc > b->max_caches) return set_error("batched query: %d caches, capacity %d", nc, b->max_caches), NRC_ERR_INVALID_ARG;
  std::vector<BatchCache> hc(static_cast<size_t>(nc));
  std::vector<BatchUnit> hu;
  for (int c = 0; c < nc; ++c) {
    if (n[c] < 0) return set_error("batched query: n[%d] < 0", c), NRC_ERR_INVALID_ARG;
    if (n[c] > 0 && (!records[c] || !rgb[c] || (reinterpret_cast<uintptr_t>(records[c]) & 15u)))
      return set_error("batched query: buffers of cache %d NULL or misaligned", c), NRC_ERR_INVALID_ARG;
    if (n[c] > (int64_t(1) << 38)) return set_error("batched query: n[%d] too large", c), NRC_ERR_INVALID_ARG;
    hc[c] = BatchCache{query_image(caches[c]), records[c], rgb[c], n[c]};
    const int64_t tiles = (n[c] + kTile - 1) / kTile;
    if (b->unit_tiles > 0)
      for (int64_t t = 0; t < tiles; t += b->unit_tiles)
        hu.push_back(BatchUnit{c, int(t), int(std::min<int64_t>(tiles, t + b->unit_tiles))});
  }
  // static ranges (unit_tiles 0): CTA g takes tiles [g T / G, (g + 1) T / G)
  // of all the caches' tiles in order, cut where a cache ends
  std::vector<int> hoff;
  int grid_static = 0;
  if (b->unit_tiles == 0) {
    int64_t total = 0;
    std::vector<int64_t> first(static_cast<size_t>(nc) + 1, 0);
    for (int c = 0; c < nc; ++c) {
      first[size_t(c)] = total;
      total += (n[c] + kTile - 1) / kTile;
    }
    first[size_t(nc)] = total;
    grid_static = int(std::min<int64_t>(b->sm_count, (total + kQuerySlots - 1) / kQuerySlots));
    int c = 0;
    for (int g = 0; g < grid_static; ++g) {
      hoff.push_back(int(hu.size()));
      const int64_t lo = total * g / grid_static, hi = total * (g + 1) / grid_static;
      int64_t t = lo;
      while (t < hi) {
        while (first[size_t(c) + 1] <= t) ++c;
        const int64_t end = std::min(hi, first[size_t(c) + 1]);
        hu.push_back(BatchUnit{c, int(t - first[size_t(c)]), int(end - first[size_t(c)])});
        t = end;
      }
    }
    hoff.push_back(int(hu.size()));
  }
  if (hu.empty()) return NRC_OK;
  if (int(hu.size()) > b->max_units) return set_error("batched query: too many work units"), NRC_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  const bool same = hc.size() == b->h_caches.size() && hu.size() == b->h_units.size() && hoff == b->h_uoff &&
                    !std::memcmp(hc.data(), b->h_caches.data(), sizeof(BatchCache) * hc.size()) &&
                    !std::memcmp(hu.data(), b->h_units.data(), sizeof(BatchUnit) * hu.size());
  if (!same) {  // descriptors are uploaded only when they change (a replayed graph reuses them)
    int slot;
    uint8_t* h = ring_slot(b, &slot);
    std::memcpy(h, hc.data(), sizeof(BatchCache) * nc);
    uint8_t* hu_p = h + up256(sizeof(BatchCache) * b->max_caches);
    std::memcpy(hu_p, hu.data(), sizeof(BatchUnit) * hu.size());
    e = cudaMemcpyAsync(b->d_caches, h, sizeof(BatchCache) * nc, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_units, hu_p, sizeof(BatchUnit) * hu.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !hoff.empty()) {
      int* ho = reinterpret_cast<int*>(h + uoff_offset(b));
      std::memcpy(ho, hoff.data(), sizeof(int) * hoff.size());
      e = cudaMemcpyAsync(b->d_uoff, ho, sizeof(int) * hoff.size(), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->ev[slot], st);
    if (e != cudaSuccess) return cuda_status(e, "batched query: descriptor upload");
    b->h_caches = hc;
    b->h_units = hu;
    b->h_uoff = hoff;
  }
  const int grid = b->unit_tiles == 0 ? grid_static : std::min<int>(b->sm_count, int(hu.size()));
  e = launch_infer_batched(caches[0], b->d_caches, b->d_units, int(hu.size()), b->d_counter, grid, st,
                           b->unit_tiles == 0 ? b->d_uoff : nullptr);
  for (int c = 0; c < nc; ++c) caches[c]->launches += 1;
  return cuda_status(e, "batched query");
}

nrc_status batch_train_step(Batch* b, nrc_cache* const* caches, int nc, const float* const* pool,
                            const float* const* target, const int64_t* n_pool, const int64_t* batch,
                            const uint64_t* frame_seed, int32_t step, float* const* loss_out, cudaStream_t st,
                            const uint64_t* seed_dev) {
  if (!pool || !target || !n_pool || !batch || (!frame_seed && !seed_dev) || step < 0)
    return set_error("batched training: NULL argument or negative step"), NRC_ERR_INVALID_ARG;
  if (seed_dev && (reinterpret_cast<uintptr_t>(seed_dev) & 7u))
    return set_error("batched training: frame seeds must be 8-byte aligned"), NRC_ERR_INVALID_ARG;
  if (nc > b->max_caches) return set_error("batched training: %d caches, capacity %d", nc, b->max_caches), NRC_ERR_INVALID_ARG;
  std::vector<int64_t> tiles(size_t(nc), 0);
  int64_t total = 0;
  for (int c = 0; c < nc; ++c) {
    if (batch[c] < 0 || batch[c] > kMaxBatch) return set_error("batched training: batch[%d] out of range", c), NRC_ERR_INVALID_ARG;
    if (batch[c] == 0) continue;
    if (n_pool[c] >= (int64_t(1) << 31) || (int64_t(step) + 1) * batch[c] > n_pool[c])
      return set_error("batched training: (step+1)*batch[%d] exceeds n_pool or n_pool too large", c), NRC_ERR_INVALID_ARG;
    if (!pool[c] || !target[c] || (reinterpret_cast<uintptr_t>(pool[c]) & 15u))
      return set_error("batched training: buffers of cache %d NULL or misaligned", c), NRC_ERR_INVALID_ARG;
    tiles[c] = (batch[c] + kTile - 1) / kTile;
    total += tiles[c];
  }
  if (total == 0) return NRC_OK;
  std::vector<int> k(size_t(nc), 0);
  int used = 0;
  if (b->train_tiles > 0) {  // each cache's CTA count from its own batch alone
    for (int c = 0; c < nc; ++c) {
      k[c] = int((tiles[c] + b->train_tiles - 1) / b->train_tiles);
      used += k[c];
    }
    nrc_status s = reserve_jobs(b, used, st);
    if (s != NRC_OK) return s;
  } else {
    // CTAs per cache so that the largest number of tiles any CTA trains is as
    // small as it can be with at most one CTA per SM in all: the smallest m
    // with sum_c ceil(tiles_c / m) <= budget, then k_c = ceil(tiles_c / m)
    const int budget = std::max(nc, b->sm_count);
    nrc_status s = reserve_jobs(b, budget, st);
    if (s != NRC_OK) return s;
    auto ctas_for = [&](int64_t m) {
      int64_t sum = 0;
      for (int c = 0; c < nc; ++c) sum += (tiles[c] + m - 1) / m;
      return sum;
    };
    int64_t lo = 1, hi = *std::max_element(tiles.begin(), tiles.end());
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (ctas_for(mid) <= budget)
        hi = mid;
      else
        lo = mid + 1;
    }
    for (int c = 0; c < nc; ++c) {
      k[c] = int((tiles[c] + lo - 1) / lo);
      used += k[c];
    }
  }
  if (train_views_ok(caches[0]) && *std::max_element(k.begin(), k.end()) <= b->sm_count) {
    // the frame kernel's training role: CTA q of cache c trains tiles q,
    // q + k[c], ... of its batch and takes slice q of its parameters in the
    // reduction and Adam.  One cooperative launch per run of whole caches
    // whose CTAs fit one per SM, so a cache's arithmetic never depends on
    // the others.  (Views zero-initialised, compared byte for byte with the
    // last upload.)
    std::vector<TrainView> hv(static_cast<size_t>(used));
    int jv = 0;
    for (int c = 0; c < nc; ++c) {
      if (!tiles[c]) continue;
      nrc_cache* cc = caches[c];
      uint64_t a = 0, ic = 0;
      if (!seed_dev) lcg_params(n_pool[c], frame_seed[c], &a, &ic);
      const int j0 = jv;
      for (int q = 0; q < k[c]; ++q, ++jv) {
        TrainView& V = hv[size_t(jv)];
        V.pool = pool[c];
        V.target = target[c];
        V.n_pool = n_pool[c];
        V.batch = batch[c];
        V.a = a;
        V.c = ic;
        V.seed = seed_dev ? seed_dev + c : nullptr;
        V.step0 = step;
        V.T = k[c];
        V.b = q;
        V.w = cc->w;
        V.m = cc->m;
        V.v = cc->v;
        V.ema = cc->cfg.ema ? cc->ema : nullptr;
        V.t_ctr = cc->t;
        V.img_in = cc->wimg;
        V.img_work = cc->wimg;
        V.img_ema_work = cc->cfg.ema ? cc->wimg_ema : nullptr;
        V.partials = b->d_partials + size_t(j0) * b->stride;
        V.bar = b->d_tcounters + c;
        V.loss_out = loss_out ? loss_out[c] : nullptr;
        V.inv3n = float(1.0 / (3.0 * double(batch[c])));
      }
    }
    cudaError_t e = cudaSuccess;
    if (hv.size() != b->h_views.size() || std::memcmp(hv.data(), b->h_views.data(), sizeof(TrainView) * hv.size())) {
      int slot;
      uint8_t* h = ring_slot(b, &slot) + views_offset(b);
      std::memcpy(h, hv.data(), sizeof(TrainView) * hv.size());
      e = cudaMemcpyAsync(b->d_views, h, sizeof(TrainView) * hv.size(), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaEventRecord(b->ev[slot], st);
      if (e != cudaSuccess) return cuda_status(e, "batched training");
      b->h_views.swap(hv);
    }
    int first = 0, run = 0;
    for (int c = 0; c <= nc && e == cudaSuccess; ++c) {
      if (c == nc || run + k[c] > b->sm_count) {
        if (run > 0) e = launch_train_views(caches[0], b->d_views + first, run, b->d_tcounters, nc + 1, 1, st);
        first += run;
        run = 0;
      }
      if (c < nc) run += k[c];
    }
    for (int c = 0; c < nc; ++c) caches[c]->launches += 1;
    return cuda_status(e, "batched training");
  }
  // descriptors in zero-initialised vectors (padding included), so that an
  // unchanged call compares equal to the last upload byte for byte
  std::vector<TrainJob> hj(static_cast<size_t>(used));
  std::vector<AdamJob> ha;
  ha.reserve(size_t(nc));
  int j = 0, n_adam = 0;
  for (int c = 0; c < nc; ++c) {
    if (!tiles[c]) continue;
    nrc_cache* cc = caches[c];
    uint64_t a = 0, ic = 0;
    if (!seed_dev) lcg_params(n_pool[c], frame_seed[c], &a, &ic);
    const int j0 = j;
    for (int q = 0; q < k[c]; ++q, ++j) {
      TrainJob& J = hj[size_t(j)];
      J.pool = pool[c];
      J.target = target[c];
      J.n_pool = n_pool[c];
      J.batch = batch[c];
      J.a = a;
      J.c = ic;
      J.seed = seed_dev ? seed_dev + c : nullptr;
      J.step = step;
      J.tile_begin = int(tiles[c] * q / k[c]);
      J.tile_end = int(tiles[c] * (q + 1) / k[c]);
      J.tile_step = 1;
      J.wimg = cc->wimg;
      J.partial = b->d_partials + size_t(j) * b->stride;
      J.t_ctr = cc->t;
      J.bump_t = q == 0;
      J.inv3n = float(1.0 / (3.0 * double(batch[c])));
    }
    ha.emplace_back();  // value-initialised: padding zero
    AdamJob& A = ha.back();
    A.w = cc->w;
    A.m = cc->m;
    A.v = cc->v;
    A.ema = cc->cfg.ema ? cc->ema : nullptr;
    A.wimg_ema = cc->wimg_ema;
    A.t_ctr = cc->t;
    A.partials = b->d_partials + size_t(j0) * b->stride;
    A.n_partials = k[c];
    A.wimg = cc->wimg;
    A.grad_scale = float(1.0 / (3.0 * double(batch[c])));
    A.loss_out = loss_out ? loss_out[c] : nullptr;
    ++n_adam;
  }
  cudaError_t e = cudaSuccess;
  const bool same = hj.size() == b->h_jobs.size() && ha.size() == b->h_adam.size() &&
                    !std::memcmp(hj.data(), b->h_jobs.data(), sizeof(TrainJob) * hj.size()) &&
                    !std::memcmp(ha.data(), b->h_adam.data(), sizeof(AdamJob) * ha.size());
  if (!same) {
    int slot;
    uint8_t* h = ring_slot(b, &slot);
    std::memcpy(h, hj.data(), sizeof(TrainJob) * hj.size());
    std::memcpy(h + up256(sizeof(TrainJob) * b->max_jobs), ha.data(), sizeof(AdamJob) * ha.size());
    e = cudaMemcpyAsync(b->d_jobs, h, sizeof(TrainJob) * j, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_adam, h + up256(sizeof(TrainJob) * b->max_jobs), sizeof(AdamJob) * n_adam,
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev[slot], st);
    if (e != cudaSuccess) return cuda_status(e, "batched training");
    b->h_jobs.swap(hj);
    b->h_adam.swap(ha);
  }
  if (e == cudaSuccess) e = launch_train_batched(caches[0], b->d_jobs, j, st);
  if (e == cudaSuccess) e = launch_adam_batched(caches[0], b->d_adam, n_adam, st);
  for (int c = 0; c < nc; ++c) caches[c]->launches += 2;
  return cuda_status(e, "batched training");
}

}  // namespace nrc

struct nrc_batch : nrc::Batch {};

using namespace nrc;

extern "C" {

nrc_status nrc_batch_create(nrc_cache* const* caches, int32_t n_caches, nrc_batch** out) {
  if (!out || !caches || n_caches <= 0) return set_error("nrc_batch_create: no caches"), NRC_ERR_INVALID_ARG;
  *out = nullptr;
  nrc_status s = batch_check(caches, n_caches);
  if (s != NRC_OK) return s;
  nrc_batch* b = new (std::nothrow) nrc_batch();
  if (!b) return set_error("host allocation failed"), NRC_ERR_OOM;
  b->caches.assign(caches, caches + n_caches);
  s = batch_init(b, caches[0], n_caches);
  if (s != NRC_OK) {
    delete b;
    return s;
  }
  *out = b;
  return NRC_OK;
}

nrc_status nrc_batch_destroy(nrc_batch* b) {
  if (!b) return NRC_OK;
  cudaError_t e = cudaDeviceSynchronize();
  batch_free(b);
  delete b;
  return cuda_status(e, "nrc_batch_destroy");
}

nrc_status nrc_batch_set_unit_tiles(nrc_batch* b, int32_t unit_tiles) {
  if (!b || unit_tiles < 0 || unit_tiles > 4096) return set_error("unit_tiles must be in [0, 4096]"), NRC_ERR_INVALID_ARG;
  b->unit_tiles = unit_tiles;
  return NRC_OK;
}

nrc_status nrc_batch_set_train_tiles(nrc_batch* b, int32_t train_tiles) {
  if (!b || train_tiles < 0 || train_tiles > 4096) return set_error("train_tiles must be in [0, 4096]"), NRC_ERR_INVALID_ARG;
  b->train_tiles = train_tiles;
  return NRC_OK;
}

nrc_status nrc_batch_infer(nrc_batch* b, const float* const* records, const int64_t* n, float* const* rgb,
                           nrc_stream stream) {
  if (!b) return set_error("nrc_batch_infer: batch is NULL"), NRC_ERR_INVALID_ARG;
  return batch_infer(b, b->caches.data(), int(b->caches.size()), records, n, rgb,
                     reinterpret_cast<cudaStream_t>(stream));
}

nrc_status nrc_batch_train_step(nrc_batch* b, const float* const* pool, const float* const* target,
                                const int64_t* n_pool, const int64_t* batch, const uint64_t* frame_seed,
                                int32_t step, float* const* loss_out, nrc_stream stream) {
  if (!b) return set_error("nrc_batch_train_step: batch is NULL"), NRC_ERR_INVALID_ARG;
  return batch_train_step(b, b->caches.data(), int(b->caches.size()), pool, target, n_pool, batch, frame_seed, step,
                          loss_out, reinterpret_cast<cudaStream_t>(stream));
}

nrc_status nrc_batch_train_step_dev(nrc_batch* b, const float* const* pool, const float* const* target,
                                    const int64_t* n_pool, const int64_t* batch, const uint64_t* frame_seed_dev,
                                    int32_t step, float* const* loss_out, nrc_stream stream) {
  if (!b) return set_error("nrc_batch_train_step_dev: batch is NULL"), NRC_ERR_INVALID_ARG;
  if (!frame_seed_dev) return set_error("nrc_batch_train_step_dev: frame_seed_dev is NULL"), NRC_ERR_INVALID_ARG;
  return batch_train_step(b, b->caches.data(), int(b->caches.size()), pool, target, n_pool, batch, nullptr, step,
                          loss_out, reinterpret_cast<cudaStream_t>(stream), frame_seed_dev);
}

nrc_status nrc_batch_autotune(nrc_batch* b, const float* const* records, const int64_t* n, float* const* rgb,
                              nrc_stream stream, int32_t* chosen) {
  if (!b) return set_error("batch is NULL"), NRC_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int cand[] = {0, 5, 10, 20, 40, 80, 160};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_u = b->unit_tiles;
  for (int u : cand) {
    b->unit_tiles = u;
    float t_min = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, st);
      nrc_status s = nrc_batch_infer(b, records, n, rgb, stream);
      if (s != NRC_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return s;
      }
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) t_min = std::min(t_min, ms);  // the first run of each size includes the descriptor upload
    }
    if (t_min < best) {
      best = t_min;
      best_u = u;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->unit_tiles = best_u;
  if (chosen) *chosen = best_u;
  return cuda_status(cudaGetLastError(), "nrc_batch_autotune");
}

}  // extern "C"
