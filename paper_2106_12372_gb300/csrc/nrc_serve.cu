// Serving runtime: frames from several viewports, each with its own cache,
// batched continuously onto one GPU.
//
// A viewport is admitted when its resident memory -- cache state (weights,
// Adam moments, weight image), its training-record pool with targets, and
// n_slots frame buffers (query records in, RGB out, per-step losses) -- fits
// the server's memory budget; it is refused with NRC_ERR_BUSY otherwise and
// may retry after another viewport closes.  A frame is submitted into one of
// its viewport's slots (refused while that slot's previous frame is still in
// flight).  The scheduler thread keeps at most max_inflight batches queued on
// the server's stream; whenever one finishes it forms the next batch from
// the pending frames in arrival order, at most one frame per viewport (a
// viewport's frame k+1 queries the weights frame k trained, so its frames
// stay in order), and issues one persistent query launch over all of them
// followed by train_steps batched training steps.  Frames that arrive while
// a batch runs join the next one.  A host function on the stream marks the
// batch's frames done; nrc_server_poll hands their timings to the caller.
//
// Each viewport's training uses a CTA count set by its own batch size
// (nrc_batch_set_train_tiles), so a frame's results do not depend on which
// other frames share its launches.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "batch.cuh"

namespace nrc {

constexpr int kMaxSlots = 8;

static int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

static size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

struct Viewport {
  bool open = false;
  nrc_cache* cache = nullptr;
  int64_t max_queries = 0;
  int64_t n_pool = 0;
  int n_slots = 0;
  size_t bytes = 0;  // charged to the budget
  void* block = nullptr;
  float* records[kMaxSlots] = {};
  float* rgb[kMaxSlots] = {};
  float* losses[kMaxSlots] = {};
  float* pool = nullptr;
  float* target = nullptr;
  bool slot_busy[kMaxSlots] = {};
  int queued = 0;  // frames pending or in flight
};

struct Frame {
  int vp;
  int slot;
  int64_t n;
  uint64_t seed;
  int64_t arrival_ns;
  int64_t submit_ns;
  int64_t tag;
};

struct Server;

struct Launched {
  Server* s;
  std::vector<Frame> frames;
  int64_t launch_ns;
  bool failed;
};

struct Server {
  nrc_server_config cfg;
  nrc_config cache_cfg;
  int device = 0;
  cudaStream_t st = nullptr;
  std::vector<Viewport> vps;
  size_t used = 0;
  std::deque<Frame> pending;
  std::deque<nrc_frame_done> done;
  int inflight = 0;
  bool stop = false;
  bool paused = false;  // nrc_server_pause: submitted frames wait, no batch is issued
  std::mutex mu;
  std::condition_variable cv;
  std::thread thr;
  Batch batch;
  bool batch_ready = false;
  nrc_status async_status = NRC_OK;
  std::string async_msg;
  int64_t frames_done = 0, batches = 0, queries_done = 0;
};

static size_t cache_bytes(const nrc_cache* c) {
  const size_t np = size_t(c->net.n_params);
  return up256(np * 4) * 3 + 256 + up256(size_t(c->img.off[c->net.n_mats]) + 1024) + 256;
}

static void CUDART_CB on_batch_done(void* p) {
  Launched* L = static_cast<Launched*>(p);
  Server* s = L->s;
  const int64_t t = now_ns();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (const Frame& f : L->frames) {
      nrc_frame_done d;
      d.viewport = f.vp;
      d.slot = f.slot;
      d.tag = f.tag;
      d.n_queries = f.n;
      d.arrival_ns = f.arrival_ns;
      d.submit_ns = f.submit_ns;
      d.launch_ns = L->launch_ns;
      d.done_ns = t;
      d.batch_frames = int32_t(L->frames.size());
      d.failed = L->failed ? 1 : 0;
      s->done.push_back(d);
      Viewport& v = s->vps[size_t(f.vp)];
      v.slot_busy[f.slot] = false;
      v.queued -= 1;
      s->queries_done += f.n;
    }
    s->frames_done += int64_t(L->frames.size());
    s->inflight -= 1;
  }
  s->cv.notify_all();
  delete L;
}

// Issues one batch: the query launch, then the training steps.
static nrc_status issue(Server* s, const std::vector<Frame>& fr) {
  const int nb = int(fr.size());
  std::vector<nrc_cache*> caches(static_cast<size_t>(nb));
  std::vector<const float*> rec(static_cast<size_t>(nb)), pool(static_cast<size_t>(nb)),
      tgt(static_cast<size_t>(nb));
  std::vector<float*> rgb(static_cast<size_t>(nb)), loss(static_cast<size_t>(nb));
  std::vector<int64_t> n(static_cast<size_t>(nb)), n_pool(static_cast<size_t>(nb)), bs(static_cast<size_t>(nb));
  std::vector<uint64_t> seed(static_cast<size_t>(nb));
  for (int i = 0; i < nb; ++i) {
    const Viewport& v = s->vps[size_t(fr[i].vp)];
    caches[i] = v.cache;
    rec[i] = v.records[fr[i].slot];
    rgb[i] = v.rgb[fr[i].slot];
    n[i] = fr[i].n;
    pool[i] = v.pool;
    tgt[i] = v.target;
    n_pool[i] = v.n_pool;
    bs[i] = s->cfg.train_batch;
    seed[i] = fr[i].seed;
  }
  nrc_status r = batch_infer(&s->batch, caches.data(), nb, rec.data(), n.data(), rgb.data(), s->st);
  for (int k = 0; k < s->cfg.train_steps && r == NRC_OK; ++k) {
    for (int i = 0; i < nb; ++i) loss[i] = s->vps[size_t(fr[i].vp)].losses[fr[i].slot] + k;
    r = batch_train_step(&s->batch, caches.data(), nb, pool.data(), tgt.data(), n_pool.data(), bs.data(),
                         seed.data(), k, loss.data(), s->st);
  }
  return r;
}

static void scheduler(Server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Frame> fr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [s] {
        return s->stop || (!s->paused && !s->pending.empty() && s->inflight < s->cfg.max_inflight);
      });
      if (s->stop) return;
      std::vector<char> taken(s->vps.size(), 0);
      for (auto it = s->pending.begin(); it != s->pending.end();) {
        if (!taken[size_t(it->vp)]) {
          taken[size_t(it->vp)] = 1;
          fr.push_back(*it);
          it = s->pending.erase(it);
        } else {
          ++it;
        }
      }
      s->inflight += 1;
      s->batches += 1;
    }
    Launched* L = new Launched{s, fr, now_ns(), false};
    nrc_status r = issue(s, fr);
    if (r != NRC_OK) {
      std::lock_guard<std::mutex> lk(s->mu);
      L->failed = true;
      if (s->async_status == NRC_OK) {
        s->async_status = r;
        s->async_msg = nrc_last_error_string();
      }
    }
    cudaError_t e = cudaLaunchHostFunc(s->st, on_batch_done, L);
    if (e != cudaSuccess) {  // complete the frames here so that nobody waits for them
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->async_status == NRC_OK) {
          s->async_status = NRC_ERR_CUDA;
          s->async_msg = std::string("nrc_server: cudaLaunchHostFunc: ") + cudaGetErrorString(e);
        }
      }
      L->failed = true;
      cudaStreamSynchronize(s->st);
      on_batch_done(L);
    }
  }
}

}  // namespace nrc

struct nrc_server : nrc::Server {};

using namespace nrc;

static nrc_status report_async(nrc_server* s) {
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->async_status != NRC_OK) set_error("%s", s->async_msg.c_str());
  return s->async_status;
}

extern "C" {

void nrc_server_default_config(nrc_server_config* c) {
  if (!c) return;
  c->memory_budget = uint64_t(16) << 30;
  c->max_viewports = 16;
  c->max_inflight = 2;
  c->train_steps = 4;
  c->train_batch = 16384;
  c->train_tiles = 4;
  c->unit_tiles = 0;
}

int64_t nrc_now_ns(void) { return now_ns(); }

nrc_status nrc_server_create(const nrc_server_config* cfg, const nrc_config* cache_cfg, nrc_server** out) {
  if (!out || !cfg || !cache_cfg) return set_error("nrc_server_create: NULL argument"), NRC_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->max_viewports < 1 || cfg->max_viewports > 4096 || cfg->max_inflight < 1 || cfg->max_inflight > 64 ||
      cfg->train_steps < 0 || cfg->train_steps > 64 || cfg->train_batch < 0 || cfg->train_batch > 65536 ||
      cfg->train_tiles < 1 || cfg->train_tiles > 4096 || cfg->unit_tiles < 0 || cfg->unit_tiles > 4096)
    return set_error("nrc_server_create: configuration out of range"), NRC_ERR_INVALID_ARG;
  if (cache_cfg->dtype != NRC_FP16 && cache_cfg->dtype != NRC_BF16)
    return set_error("nrc_server_create: served caches compute in FP16 or BF16"), NRC_ERR_UNSUPPORTED;
  if (cache_cfg->width != 64 || cache_cfg->path != NRC_PATH_FUSED)
    return set_error("nrc_server_create: served caches take the fused width-64 network"), NRC_ERR_UNSUPPORTED;
  nrc_server* s = new (std::nothrow) nrc_server();
  if (!s) return set_error("host allocation failed"), NRC_ERR_OOM;
  s->cfg = *cfg;
  s->cache_cfg = *cache_cfg;
  s->vps.resize(size_t(cfg->max_viewports));
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    nrc_status r = cuda_status(e, "nrc_server_create");
    delete s;
    return r;
  }
  // a prototype cache fixes the shape every viewport's cache must have
  nrc_cache* proto = nullptr;
  nrc_status r = nrc_create(cache_cfg, reinterpret_cast<nrc_stream>(s->st), &proto);
  if (r == NRC_OK) {
    r = batch_init(&s->batch, proto, cfg->max_viewports);
    s->batch.unit_tiles = cfg->unit_tiles;
    s->batch.train_tiles = cfg->train_tiles;
    s->batch_ready = r == NRC_OK;
    nrc_destroy(proto);
  }
  if (r != NRC_OK) {
    if (s->batch_ready) batch_free(&s->batch);
    cudaStreamDestroy(s->st);
    delete s;
    return r;
  }
  s->thr = std::thread(scheduler, static_cast<Server*>(s));
  *out = s;
  return NRC_OK;
}

nrc_status nrc_server_pause(nrc_server* s, int32_t paused) {
  if (!s) return set_error("server is NULL"), NRC_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->paused = paused != 0;
  }
  s->cv.notify_all();
  return NRC_OK;
}

nrc_status nrc_server_drain(nrc_server* s) {
  if (!s) return set_error("server is NULL"), NRC_ERR_INVALID_ARG;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->paused = false;  // held frames are released
    s->cv.notify_all();
    s->cv.wait(lk, [s] { return s->pending.empty() && s->inflight == 0; });
  }
  cudaError_t e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return cuda_status(e, "nrc_server_drain");
  return report_async(s);
}

nrc_status nrc_server_destroy(nrc_server* s) {
  if (!s) return NRC_OK;
  nrc_status r = nrc_server_drain(s);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->thr.joinable()) s->thr.join();
  for (Viewport& v : s->vps)
    if (v.open) {
      nrc_destroy(v.cache);
      cudaFree(v.block);
    }
  if (s->batch_ready) batch_free(&s->batch);
  cudaStreamDestroy(s->st);
  delete s;
  return r;
}

nrc_status nrc_server_open_viewport(nrc_server* s, const nrc_config* cache_cfg, int64_t max_queries, int64_t n_pool,
                                    int32_t n_slots, int32_t* id_out) {
  if (!s || !cache_cfg || !id_out) return set_error("nrc_server_open_viewport: NULL argument"), NRC_ERR_INVALID_ARG;
  *id_out = -1;
  if (max_queries < 0 || max_queries > (int64_t(1) << 34) || n_slots < 1 || n_slots > kMaxSlots || n_pool < 0 ||
      n_pool >= (int64_t(1) << 31) || int64_t(s->cfg.train_steps) * s->cfg.train_batch > n_pool)
    return set_error("nrc_server_open_viewport: sizes out of range (n_slots 1..%d; n_pool >= train_steps x "
                     "train_batch)", kMaxSlots),
           NRC_ERR_INVALID_ARG;
  // the memory this viewport keeps resident
  const size_t rec_b = up256(size_t(max_queries) * 64), rgb_b = up256(size_t(max_queries) * 12);
  const size_t loss_b = up256(size_t(std::max(1, s->cfg.train_steps)) * 4);
  const size_t pool_b = up256(size_t(n_pool) * 64), tgt_b = up256(size_t(n_pool) * 12);
  const size_t block_b = size_t(n_slots) * (rec_b + rgb_b + loss_b) + pool_b + tgt_b;
  int id = -1;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t i = 0; i < s->vps.size(); ++i)
      if (!s->vps[i].open && !s->vps[i].cache) {
        id = int(i);
        break;
      }
    if (id < 0) return set_error("nrc_server_open_viewport: all %d viewports in use", s->cfg.max_viewports), NRC_ERR_BUSY;
    s->vps[size_t(id)].cache = reinterpret_cast<nrc_cache*>(1);  // reserved while being set up
  }
  auto release = [&](nrc_cache* c, void* blk, size_t charged) {
    if (c) nrc_destroy(c);
    if (blk) cudaFree(blk);
    std::lock_guard<std::mutex> lk(s->mu);
    s->used -= charged;
    s->vps[size_t(id)].cache = nullptr;
  };
  nrc_cache* c = nullptr;
  nrc_status r = nrc_create(cache_cfg, reinterpret_cast<nrc_stream>(s->st), &c);
  if (r == NRC_OK && !batch_same_cfg(c->cfg, s->cache_cfg))
    r = (set_error("nrc_server_open_viewport: the cache configuration differs from the server's (only the seed may "
                   "differ)"),
         NRC_ERR_INVALID_ARG);
  if (r != NRC_OK) {
    release(c, nullptr, 0);
    return r;
  }
  const size_t need = block_b + cache_bytes(c);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->used + need > s->cfg.memory_budget) {
      const size_t used = s->used;
      s->vps[size_t(id)].cache = nullptr;
      nrc_destroy(c);
      return set_error("nrc_server_open_viewport: %zu bytes in use + %zu requested exceed the budget of %llu", used,
                       need, (unsigned long long)s->cfg.memory_budget),
             NRC_ERR_BUSY;
    }
    s->used += need;
  }
  void* blk = nullptr;
  cudaError_t e = dev_alloc(&blk, block_b);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release(c, nullptr, need);
    return set_error("nrc_server_open_viewport: device allocation of %zu bytes failed", block_b), NRC_ERR_OOM;
  }
  Viewport v;
  v.open = true;
  v.cache = c;
  v.max_queries = max_queries;
  v.n_pool = n_pool;
  v.n_slots = n_slots;
  v.bytes = need;
  v.block = blk;
  uint8_t* p = static_cast<uint8_t*>(blk);
  for (int k = 0; k < n_slots; ++k) {
    v.records[k] = reinterpret_cast<float*>(p);
    p += rec_b;
    v.rgb[k] = reinterpret_cast<float*>(p);
    p += rgb_b;
    v.losses[k] = reinterpret_cast<float*>(p);
    p += loss_b;
  }
  v.pool = reinterpret_cast<float*>(p);
  p += pool_b;
  v.target = reinterpret_cast<float*>(p);
  e = cudaMemsetAsync(blk, 0, block_b, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) {
    release(c, blk, need);
    return cuda_status(e, "nrc_server_open_viewport");
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->vps[size_t(id)] = v;
  }
  *id_out = id;
  return NRC_OK;
}

nrc_status nrc_server_close_viewport(nrc_server* s, int32_t id) {
  if (!s || id < 0 || id >= int(s->vps.size())) return set_error("nrc_server_close_viewport: bad viewport"), NRC_ERR_INVALID_ARG;
  Viewport v;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->vps[size_t(id)].open) return set_error("nrc_server_close_viewport: viewport %d is not open", id), NRC_ERR_INVALID_ARG;
    s->paused = false;  // its held frames are released
    s->cv.notify_all();
    s->cv.wait(lk, [s, id] { return s->vps[size_t(id)].queued == 0; });
    v = s->vps[size_t(id)];
    s->vps[size_t(id)].open = false;
  }
  cudaError_t e = cudaStreamSynchronize(s->st);
  nrc_destroy(v.cache);
  cudaFree(v.block);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->used -= v.bytes;
    s->vps[size_t(id)] = Viewport();
  }
  return cuda_status(e, "nrc_server_close_viewport");
}

nrc_status nrc_server_viewport_buffers(nrc_server* s, int32_t id, int32_t slot, float** records, float** rgb,
                                       float** losses) {
  if (!s || id < 0 || id >= int(s->vps.size())) return set_error("nrc_server_viewport_buffers: bad viewport"), NRC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  const Viewport& v = s->vps[size_t(id)];
  if (!v.open || slot < 0 || slot >= v.n_slots)
    return set_error("nrc_server_viewport_buffers: viewport %d not open or slot %d out of range", id, slot), NRC_ERR_INVALID_ARG;
  if (records) *records = v.records[slot];
  if (rgb) *rgb = v.rgb[slot];
  if (losses) *losses = v.losses[slot];
  return NRC_OK;
}

nrc_status nrc_server_viewport_pool(nrc_server* s, int32_t id, float** pool, float** target, nrc_cache** cache) {
  if (!s || id < 0 || id >= int(s->vps.size())) return set_error("nrc_server_viewport_pool: bad viewport"), NRC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  const Viewport& v = s->vps[size_t(id)];
  if (!v.open) return set_error("nrc_server_viewport_pool: viewport %d is not open", id), NRC_ERR_INVALID_ARG;
  if (pool) *pool = v.pool;
  if (target) *target = v.target;
  if (cache) *cache = v.cache;
  return NRC_OK;
}

nrc_status nrc_server_submit(nrc_server* s, int32_t id, int32_t slot, int64_t n_queries, uint64_t frame_seed,
                             int64_t arrival_ns, int64_t tag) {
  if (!s || id < 0 || id >= int(s->vps.size())) return set_error("nrc_server_submit: bad viewport"), NRC_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    Viewport& v = s->vps[size_t(id)];
    if (!v.open || slot < 0 || slot >= v.n_slots || n_queries < 0 || n_queries > v.max_queries)
      return set_error("nrc_server_submit: viewport %d not open, slot %d or n_queries %lld out of range", id, slot,
                       (long long)n_queries),
             NRC_ERR_INVALID_ARG;
    if (v.slot_busy[slot]) return set_error("nrc_server_submit: slot %d of viewport %d is in flight", slot, id), NRC_ERR_BUSY;
    v.slot_busy[slot] = true;
    v.queued += 1;
    s->pending.push_back(Frame{id, slot, n_queries, frame_seed, arrival_ns, now_ns(), tag});
  }
  s->cv.notify_all();
  return NRC_OK;
}

nrc_status nrc_server_poll(nrc_server* s, nrc_frame_done* out, int32_t max_out, int32_t timeout_ms, int32_t* n_out) {
  if (!s || !n_out || (max_out > 0 && !out) || max_out < 0) return set_error("nrc_server_poll: bad argument"), NRC_ERR_INVALID_ARG;
  *n_out = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (timeout_ms > 0 && s->done.empty())
    s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [s] { return !s->done.empty(); });
  int k = 0;
  while (k < max_out && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *n_out = k;
  if (s->async_status != NRC_OK) {
    set_error("%s", s->async_msg.c_str());
    return s->async_status;
  }
  return NRC_OK;
}

nrc_status nrc_server_query(nrc_server* s, nrc_server_info* out) {
  if (!s || !out) return set_error("nrc_server_query: NULL argument"), NRC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->memory_used = s->used;
  out->memory_budget = s->cfg.memory_budget;
  out->frames_done = s->frames_done;
  out->batches = s->batches;
  out->queries_done = s->queries_done;
  out->pending = int64_t(s->pending.size());
  int open = 0;
  for (const Viewport& v : s->vps) open += v.open ? 1 : 0;
  out->viewports = open;
  out->inflight = s->inflight;
  return NRC_OK;
}

}  // extern "C"
