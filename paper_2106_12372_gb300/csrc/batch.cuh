// Internal interface of the batched-cache launches, shared by the nrc_batch
// C API and the serving runtime (which batches a different subset of its
// viewports' caches on every launch).
#pragma once

#include <vector>

#include "nrc_internal.cuh"

namespace nrc {

constexpr int kRing = 8;  // pinned descriptor slots in flight

struct Batch {
  std::vector<nrc_cache*> caches;  // the caches of the nrc_batch C object (unused by the server)
  int unit_tiles = 0;              // 128-row tiles per query work unit; 0: one contiguous range per CTA
  int train_tiles = 0;             // >0: a cache's training CTAs = ceil(its tiles / train_tiles)
  int max_caches = 0;
  int max_units = 0;
  int max_jobs = 0;
  // device descriptors
  BatchCache* d_caches = nullptr;
  BatchUnit* d_units = nullptr;
  unsigned* d_counter = nullptr;
  TrainJob* d_jobs = nullptr;
  AdamJob* d_adam = nullptr;
  TrainView* d_views = nullptr;   // training CTAs of the frame-kernel path (sm_count entries)
  int* d_uoff = nullptr;           // static query ranges: first unit of each CTA (sm_count + 1 entries)
  unsigned* d_tcounters = nullptr;  // its per-cache barrier counters + retire counter (max_caches + 1)
  float* d_partials = nullptr;
  // host: last uploaded query descriptors, pinned staging ring
  std::vector<BatchCache> h_caches;
  std::vector<BatchUnit> h_units;
  std::vector<int> h_uoff;
  // host: last uploaded training descriptors (zero-padded, compared bytewise)
  std::vector<TrainJob> h_jobs;
  std::vector<AdamJob> h_adam;
  std::vector<TrainView> h_views;
  uint8_t* pinned = nullptr;
  size_t slot_bytes = 0;
  cudaEvent_t ev[kRing] = {};
  int ring = 0;
  int sm_count = 0;
  size_t stride = 0;  // floats per weight-gradient partial
};

// Configurations that can share launches (equal in all but the seed and path).
bool batch_same_cfg(const nrc_config& a, const nrc_config& b);
// Checks that the caches can share launches (same shape, dtype and
// hyper-parameters, one device, 16-bit tensor-core path).
nrc_status batch_check(nrc_cache* const* caches, int n_caches);
// Allocates descriptors for up to max_caches caches and sm_count training CTAs.
nrc_status batch_init(Batch* b, const nrc_cache* proto, int max_caches);
void batch_free(Batch* b);

// One persistent query launch over caches[0..nc): work units of unit_tiles
// tiles, taken by CTAs from an atomic counter.  n[c] == 0 skips cache c.
nrc_status batch_infer(Batch* b, nrc_cache* const* caches, int nc, const float* const* records, const int64_t* n,
                       float* const* rgb, cudaStream_t st);
// One training step of every cache with batch[c] > 0: one gradient launch,
// one Adam launch.  CTAs are shared out in proportion to the caches' tiles
// (train_tiles == 0) or set per cache from its own batch (train_tiles > 0,
// which makes each cache's result independent of the other caches).  The
// frame seeds come from the host array frame_seed, or, when seed_dev is not
// null, from the device array seed_dev[c] (read by the gradient kernel).
// The descriptors are uploaded only when they differ from the last upload,
// so with device seeds repeated calls launch kernels only.
nrc_status batch_train_step(Batch* b, nrc_cache* const* caches, int nc, const float* const* pool,
                            const float* const* target, const int64_t* n_pool, const int64_t* batch,
                            const uint64_t* frame_seed, int32_t step, float* const* loss_out, cudaStream_t st,
                            const uint64_t* seed_dev = nullptr);

}  // namespace nrc
