// api.cu -- the C ABI (include/shk.h): build, query, (de)serialisation and the
// batched leaf search.  Host code only orchestrates; every step of the
// construction runs in the kernels of this library.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace shk {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

shk_status fail(shk_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

// Working memory of builds and queries comes from one memory pool per device
// that the library owns.  Its release threshold is unlimited: memory freed at
// the end of a call stays mapped for the next one, so repeated builds do not
// map and unmap device memory at every synchronisation (10^8 keys: the radix
// partition phase 3.4 -> 2.1 ms).  shk_release_memory returns it.  The
// device's default pool, which the caller may use, is left as it is.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];

static cudaError_t pool_of_current(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t created;
      e = cudaMemPoolCreate(&created, &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = ~0ull;
      e = cudaMemPoolSetAttribute(created, cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) {
        cudaMemPoolDestroy(created);
        return e;
      }
      g_pool[dev] = created;
    }
    pool = g_pool[dev];
  }
  *out = pool;
  return cudaSuccess;
}

cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool;
  const cudaError_t e = pool_of_current(&pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// High watermark of the current device's pool (reset: the watermark restarts
// from the bytes in use now).
static uint64_t pool_used_high(bool reset) {
  cudaMemPool_t pool;
  if (pool_of_current(&pool) != cudaSuccess) return 0;
  uint64_t v = 0;
  if (reset) {
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v);
    return 0;
  }
  cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v);
  return v;
}

__global__ void k_set_deadline(unsigned long long* at, uint64_t budget_ns) {
  *at = global_ns() + budget_ns;
}

shk_status init_ctx(Ctx& c) {
  SHK_CUDA(cudaGetDevice(&c.device));
  SHK_CUDA(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device));
  return SHK_OK;
}

static shk_status device_errors(uint32_t e) {
  if (e & kErrCancelled) return fail(SHK_ECANCELLED, "the build was cancelled");
  if (e & kErrTimeout) return fail(SHK_ETIMEOUT, "the build's time budget (deadline_ms) ran out");
  if (e & kErrDup) return fail(SHK_EDUPKEY, "two keys have the same 128-bit fingerprint");
  if (e & kErrBucketOverflow) return fail(SHK_EINVAL, "a bucket holds more than 8192 keys");
  if (e & kErrLeafSize) return fail(SHK_EINVAL, "a leaf has 0 or more than 64 keys");
  if (e & kErrSeedCap) return fail(SHK_ESEEDCAP, "a seed search reached 2^40");
  if (e & kErrRibbon) return fail(SHK_ESEEDCAP, "a retrieval shard was unsolvable for 256 seeds");
  if (e & kErrOrient) return fail(SHK_ECUDA, "internal: orientation of a leaf failed");
  return SHK_OK;
}

// Phase timer on the build stream (profile = 1).
struct PhaseTimer {
  bool on;
  cudaStream_t st;
  cudaEvent_t ev[12];
  int n = 0;
  PhaseTimer(bool enabled, cudaStream_t s) : on(enabled), st(s) {}
  ~PhaseTimer() {
    for (int i = 0; i < n; i++) cudaEventDestroy(ev[i]);
  }
  int mark() {
    if (!on || n >= 12) return -1;
    cudaEventCreate(&ev[n]);
    cudaEventRecord(ev[n], st);
    return n++;
  }
  double ms(int a, int b) const {
    if (!on || a < 0 || b < 0) return 0.0;
    float t = 0;
    cudaEventElapsedTime(&t, ev[a], ev[b]);
    return t;
  }
};


shk_status blocks_per_sm(const void* kernel, int threads, size_t smem, int* out) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
  int dev = 0;
  SHK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(dev, kernel, threads, smem);
  auto it = cache.find(key);
  if (it == cache.end()) {
    int n = 0;
    SHK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem));
    it = cache.emplace(key, n).first;
  }
  *out = it->second;
  return SHK_OK;
}

shk_status raise_smem_limit(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  SHK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[{dev, kernel}];
  if (bytes > cur) {
    SHK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
  }
  return SHK_OK;
}

__global__ void k_u64_to_u32(const uint64_t* in, uint64_t n, uint32_t* out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (uint32_t)in[i];
}

__global__ void k_leaf_descs(const uint32_t* off, uint32_t n_leaves, LeafDesc* d) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_leaves) return;
  LeafDesc v;
  v.key_off = off[i];
  v.m = off[i + 1] - off[i];
  v.code_idx = kNoCode;
  v.bucket = 0;
  d[i] = v;
}

template <class T>
static shk_status d2h(Ctx& c, T* host, const T* dev, size_t count = 1) {
  SHK_CUDA(cudaMemcpyAsync(host, dev, count * sizeof(T), cudaMemcpyDeviceToHost, c.stream));
  return SHK_OK;
}

static void layout(shk_mphf* m) {
  const uint64_t* h = m->hdr;
  const uint64_t B = h[4], rice_bits = h[8], lK = h[9], khb = h[10], lO = h[11], ohb = h[12],
                 rib = h[13], ns = h[7];
  uint64_t p = kHeaderWords;
  m->off_rice = p;
  p += (rice_bits + 63) / 64;
  m->off_kl = p;
  p += ((B + 1) * lK + 63) / 64;
  m->off_kh = p;
  p += (khb + 63) / 64;
  m->off_ol = p;
  p += ((B + 1) * lO + 63) / 64;
  m->off_oh = p;
  p += (ohb + 63) / 64;
  m->off_seed = p;
  p += (ns + 7) / 8;
  m->off_rib = p;
  p += (rib + 63) / 64;
  m->words = p;
}

static void free_mphf(shk_mphf* m) {
  if (!m) return;
  if (m->d_blob) cudaFree(m->d_blob);
  if (m->d_K) cudaFree(m->d_K);
  if (m->d_O) cudaFree(m->d_O);
  if (m->d_shard_off) cudaFree(m->d_shard_off);
  if (m->d_qnode) cudaFree(m->d_qnode);
  if (m->d_qbase) cudaFree(m->d_qbase);
  delete m;
}

// Keys to the device (a copy when they are host buffers).
static shk_status stage_keys(Ctx& c, const shk_keys* keys, const void** data, const uint64_t** offs) {
  *data = keys->data;
  *offs = keys->str_offsets;
  const uint64_t N = keys->n_keys;
  if (keys->on_device || N == 0) return SHK_OK;
  if (keys->kind == SHK_KEYS_U64 || keys->kind == SHK_KEYS_FP128) {
    const size_t bytes = N * (keys->kind == SHK_KEYS_U64 ? 8 : 16);
    uint8_t* d;
    SHK_TRY(c.arena.alloc(&d, bytes));
    SHK_CUDA(cudaMemcpyAsync(d, keys->data, bytes, cudaMemcpyHostToDevice, c.stream));
    *data = d;
  } else {
    const uint64_t total = keys->str_offsets[N];
    uint8_t* d;
    uint64_t* o;
    SHK_TRY(c.arena.alloc(&d, total + 8));
    SHK_TRY(c.arena.alloc(&o, N + 1));
    SHK_CUDA(cudaMemcpyAsync(d, keys->data, total, cudaMemcpyHostToDevice, c.stream));
    SHK_CUDA(cudaMemcpyAsync(o, keys->str_offsets, (N + 1) * 8, cudaMemcpyHostToDevice, c.stream));
    *data = d;
    *offs = o;
  }
  return SHK_OK;
}

static shk_status check_keys(const shk_keys* keys) {
  if (!keys) return fail(SHK_EINVAL, "keys is NULL");
  if (keys->kind != SHK_KEYS_U64 && keys->kind != SHK_KEYS_STR && keys->kind != SHK_KEYS_FP128)
    return fail(SHK_EINVAL, "unknown key kind");
  if (keys->n_keys && !keys->data) return fail(SHK_EINVAL, "key data is NULL");
  if (keys->kind == SHK_KEYS_STR && keys->n_keys && !keys->str_offsets)
    return fail(SHK_EINVAL, "string keys need str_offsets");
  return SHK_OK;
}

shk_status build_controlled(const shk_keys* keys, const shk_build_opts* o, cudaStream_t st,
                            shk_mphf** out, const volatile uint32_t* abort) {
  SHK_TRY(check_keys(keys));
  const uint64_t N = keys->n_keys;
  const uint32_t n = o->leaf_size, b = o->bucket_size;
  if (n < 2 || n > kMaxLeaf) return fail(SHK_EINVAL, "leaf_size must be in [2, 64]");
  if (b < n || b > kMaxBucketSize) return fail(SHK_EINVAL, "bucket_size must be in [leaf_size, 4096]");
  if (N >= (1ull << 32)) return fail(SHK_EINVAL, "at most 2^32 - 1 keys");
  if (o->sched > SHK_SCHED_SINGLE_LAUNCH) return fail(SHK_EINVAL, "unknown schedule");
  if (o->leaf_mode > SHK_LEAF_ROTATION) return fail(SHK_EINVAL, "unknown leaf mode");
  const uint32_t rf = o->leaf_mode;
  const uint32_t rw = ribbon_width(n);  // retrieval row width
  const uint32_t S = o->shard_buckets ? o->shard_buckets : default_shard_buckets(b, rw);
  const uint32_t eps = o->eps_num ? o->eps_num : default_eps_num(rw);
  Ctx c(st);
  SHK_TRY(init_ctx(c));
  // leaf kernel configuration: the autotuner's choice for this leaf size,
  // unless the caller fixes it
  LeafCfg cfg;
  if (rf) {
    cfg = {8u, 8u, 2u, o->chunk_passes ? o->chunk_passes : 2u};
  } else if (o->seeds_per_lane) {
    cfg = {o->seeds_per_lane, o->warps_per_block ? o->warps_per_block : 8u,
           o->key_unroll ? o->key_unroll : 2u, o->chunk_passes ? o->chunk_passes : 8u};
    if (!leaf_cfg_valid(cfg)) return fail(SHK_EINVAL, "unsupported leaf kernel configuration");
  } else {
    SHK_TRY(tuned_leaf_cfg(c, n, &cfg));
    if (o->chunk_passes) cfg.passes = o->chunk_passes;
  }
  PhaseTimer pt(o->profile != 0, st);
  pool_used_high(true);
  // leaf-search control: [0], [1] device start / end of the leaf search,
  // [2] deadline (device time)
  unsigned long long* ctl;
  SHK_TRY(c.arena.alloc(&ctl, 4));
  SHK_CUDA(cudaMemsetAsync(ctl, 0xFF, 8, st));
  SHK_CUDA(cudaMemsetAsync(ctl + 1, 0, 24, st));
  if (o->deadline_ms) {
    k_set_deadline<<<1, 1, 0, st>>>(ctl + 2, (uint64_t)o->deadline_ms * 1000000ull);
    c.launches++;
    SHK_CUDA(cudaGetLastError());
  }
  const int t0 = pt.mark();
  const uint64_t B = N ? (N + b - 1) / b : 0;
  const uint32_t N32 = (uint32_t)N;

  const void* kdata;
  const uint64_t* koffs;
  SHK_TRY(stage_keys(c, keys, &kdata, &koffs));

  // a1: fingerprints, buckets, histogram
  ulonglong2* fp;
  uint32_t *counts, *err;
  SHK_TRY(c.arena.alloc(&fp, N));
  SHK_TRY(c.arena.alloc(&counts, B, true));
  SHK_TRY(c.arena.alloc(&err, 1, true));
  SHK_TRY(launch_fingerprint(c, keys->kind, kdata, koffs, N32, B, fp, counts));
  const int t1 = pt.mark();

  // bucket offsets; tree shape of every bucket, prefix sums, one host sync
  // for the sizes
  uint32_t *K, *nleaf, *ncode, *nsplit, *leaf_base, *code_base, *split_base, *maxb;
  SHK_TRY(c.arena.alloc(&K, B + 1));
  SHK_TRY((exclusive_scan<uint32_t, uint32_t>(c, counts, B, K)));
  const int t1a = pt.mark();
  SHK_TRY(c.arena.alloc(&nleaf, B));
  SHK_TRY(c.arena.alloc(&ncode, B));
  SHK_TRY(c.arena.alloc(&nsplit, B));
  SHK_TRY(c.arena.alloc(&maxb, 1, true));
  SHK_TRY(launch_tree_count(c, K, B, n, nleaf, ncode, nsplit, maxb));
  SHK_TRY(c.arena.alloc(&leaf_base, B + 1));
  SHK_TRY(c.arena.alloc(&code_base, B + 1));
  SHK_TRY(c.arena.alloc(&split_base, B + 1));
  SHK_TRY((exclusive_scan<uint32_t, uint32_t>(c, nleaf, B, leaf_base)));
  SHK_TRY((exclusive_scan<uint32_t, uint32_t>(c, ncode, B, code_base)));
  SHK_TRY((exclusive_scan<uint32_t, uint32_t>(c, nsplit, B, split_base)));
  uint32_t h_maxb = 0, h_L = 0, h_C = 0, h_splits = 0, h_err = 0, h_total = 0;
  SHK_TRY(d2h(c, &h_total, K + B));
  SHK_TRY(d2h(c, &h_maxb, maxb));
  SHK_TRY(d2h(c, &h_L, leaf_base + B));
  SHK_TRY(d2h(c, &h_C, code_base + B));
  SHK_TRY(d2h(c, &h_splits, split_base + B));
  std::vector<uint32_t> h_leaf_base;
  if (o->sched == SHK_SCHED_PER_BUCKET && B) {
    h_leaf_base.resize(B + 1);
    SHK_TRY(d2h(c, h_leaf_base.data(), leaf_base, B + 1));
  }
  SHK_CUDA(cudaStreamSynchronize(st));
  if (h_maxb > kMaxBucketKeys) return fail(SHK_EINVAL, "a bucket holds more than 8192 keys");
  if (h_total != N) return fail(SHK_ECUDA, "bucket histogram does not add up to the key count");

  // a2: partition into buckets (the in-bucket sort opens the splitting kernel)
  ulonglong2* sfp;
  SHK_TRY(c.arena.alloc(&sfp, N));
  const int t1b = pt.mark();
  SHK_TRY(launch_scatter(c, fp, N32, B, K, sfp));
  const int t2 = pt.mark();

  // a3: splitting trees
  uint64_t *codes, *llo, *lhi;
  uint8_t* code_k;
  LeafDesc* leaves;
  SHK_TRY(c.arena.alloc(&codes, h_C));
  SHK_TRY(c.arena.alloc(&code_k, h_C));
  SHK_TRY(c.arena.alloc(&leaves, h_L));
  SHK_TRY(c.arena.alloc(&llo, N));
  SHK_TRY(c.arena.alloc(&lhi, N));
  SHK_TRY(launch_split(c, sfp, K, B, n, h_maxb, code_base, leaf_base, codes, code_k, leaves, llo,
                       lhi, err));
  const int t3 = pt.mark();

  // a4 + a5: leaf seeds
  unsigned long long *best, *counters;
  SHK_TRY(c.arena.alloc(&best, h_L));
  // executed, sum(seed+1), sum((seed+1) m), hash evaluations, seeds tested,
  // rotation-filter steps (double)
  SHK_TRY(c.arena.alloc(&counters, 6, true));
  if (h_L) SHK_CUDA(cudaMemsetAsync(best, 0xFF, (size_t)h_L * 8, st));
  LeafSearchArgs a{leaves, h_L, llo, 0, best, err, counters, cfg,
                   LeafCtl{ctl, o->deadline_ms ? ctl + 2 : nullptr, abort}};
  uint64_t leaf_launches = 0;
  if (o->sched == SHK_SCHED_PERSISTENT) {
    SHK_TRY(rf ? launch_leaf_rf_persistent(c, a) : launch_leaf_persistent(c, a));
    leaf_launches = h_L ? 1 : 0;
  } else if (o->sched == SHK_SCHED_SINGLE_LAUNCH) {
    SHK_TRY(rf ? launch_leaf_rf_range(c, a, 0, h_L) : launch_leaf_range(c, a, 0, h_L));
    leaf_launches = h_L ? 1 : 0;
  } else {
    for (uint64_t i = 0; i < B; i++) {
      if (h_leaf_base[i + 1] > h_leaf_base[i]) {
        SHK_TRY(rf ? launch_leaf_rf_range(c, a, h_leaf_base[i], h_leaf_base[i + 1])
                   : launch_leaf_range(c, a, h_leaf_base[i], h_leaf_base[i + 1]));
        leaf_launches++;
      }
    }
  }
  const int t4 = pt.mark();

  // a6: orientation (also stores leaf seeds into their code slots)
  uint8_t* f;
  SHK_TRY(c.arena.alloc(&f, N, true));
  SHK_TRY(launch_orient(c, leaves, h_L, llo, best, codes, f, nullptr, err, rf));
  SHK_TRY(launch_leaf_sums(c, leaves, h_L, best, counters + 1, rf, llo, (double*)(counters + 5)));
  const int t5 = pt.mark();

  // a7 sizes: Rice bits per bucket, shard slots
  uint64_t *bucket_bits, *O, *slots, *shard_off;
  SHK_TRY(c.arena.alloc(&bucket_bits, B));
  SHK_TRY(c.arena.alloc(&O, B + 1));
  SHK_TRY(launch_rice_bits(c, codes, code_k, code_base, B, bucket_bits));
  SHK_TRY((exclusive_scan<uint64_t, uint64_t>(c, bucket_bits, B, O)));
  const uint64_t num_shards = (B + S - 1) / S;
  uint32_t* max_sk;
  SHK_TRY(c.arena.alloc(&slots, num_shards));
  SHK_TRY(c.arena.alloc(&shard_off, num_shards + 1));
  SHK_TRY(c.arena.alloc(&max_sk, 1, true));
  SHK_TRY(launch_shard_slots(c, K, B, S, eps, rw, num_shards, slots));
  SHK_TRY((exclusive_scan<uint64_t, uint64_t>(c, slots, num_shards, shard_off)));
  SHK_TRY(launch_max_shard_keys(c, K, B, S, num_shards, max_sk));
  uint64_t h_rice_bits = 0, h_rib_bits = 0;
  uint32_t h_max_sk = 0;
  unsigned long long h_cnt[6] = {0, 0, 0, 0, 0, 0}, h_ctl[2] = {0, 0};
  SHK_TRY(d2h(c, &h_rice_bits, O + B));
  SHK_TRY(d2h(c, &h_rib_bits, shard_off + num_shards));
  SHK_TRY(d2h(c, &h_max_sk, max_sk));
  SHK_TRY(d2h(c, h_cnt, counters, 6));
  SHK_TRY(d2h(c, h_ctl, ctl, 2));
  SHK_TRY(d2h(c, &h_err, err));
  SHK_CUDA(cudaStreamSynchronize(st));
  SHK_TRY(device_errors(h_err));

  // the encoded object
  shk_mphf* m = new shk_mphf();
  m->device = c.device;
  const uint32_t lK = ef_low_bits(N, B + 1), lO = ef_low_bits(h_rice_bits, B + 1);
  const uint64_t hdr[kHeaderWords] = {kMagic, N, n, b, B, S, eps, num_shards, h_rice_bits, lK,
                                      (N >> lK) + B + 1, lO, (h_rice_bits >> lO) + B + 1,
                                      h_rib_bits, rf, rw};
  memcpy(m->hdr, hdr, sizeof hdr);
  layout(m);
  shk_status rs = SHK_OK;
  auto cuda_ok = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rs == SHK_OK) rs = fail(SHK_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaSuccess;
  };
  if (cuda_ok(cudaMalloc(&m->d_blob, m->words * 8), "cudaMalloc") &&
      cuda_ok(cudaMalloc(&m->d_K, (B + 1) * 4), "cudaMalloc") &&
      cuda_ok(cudaMalloc(&m->d_O, (B + 1) * 8), "cudaMalloc") &&
      cuda_ok(cudaMalloc(&m->d_shard_off, (num_shards + 1) * 8), "cudaMalloc") &&
      cuda_ok(cudaMemsetAsync(m->d_blob, 0, m->words * 8, st), "cudaMemsetAsync") &&
      cuda_ok(cudaMemcpyAsync(m->d_blob, hdr, sizeof hdr, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync")) {
    if (B == 0) {
      // N = 0: K = O = (0); both Elias-Fano sequences are a single set bit
      cuda_ok(cudaMemsetAsync(K, 0, 4, st), "cudaMemsetAsync");
      cuda_ok(cudaMemsetAsync(O, 0, 8, st), "cudaMemsetAsync");
    }
    rs = launch_rice_write(c, codes, code_k, code_base, B, O, m->d_blob + m->off_rice);
    if (rs == SHK_OK) rs = launch_ef_write_u32(c, K, B + 1, lK, m->d_blob + m->off_kl, m->d_blob + m->off_kh);
    if (rs == SHK_OK) rs = launch_ef_write_u64(c, O, B + 1, lO, m->d_blob + m->off_ol, m->d_blob + m->off_oh);
  }
  const int t6 = pt.mark();
  if (rs == SHK_OK)
    rs = launch_ribbon(c, llo, lhi, f, K, B, S, eps, rw, num_shards, shard_off,
                       (uint32_t)shard_slots(h_max_sk, eps, rw), h_rib_bits, N, m->d_blob + m->off_rib,
                       (uint8_t*)(m->d_blob + m->off_seed), err);
  const int t7 = pt.mark();
  if (rs == SHK_OK) {
    cuda_ok(cudaMemcpyAsync(m->d_K, K, (B + 1) * 4, cudaMemcpyDeviceToDevice, st), "cudaMemcpyAsync");
    cuda_ok(cudaMemcpyAsync(m->d_O, O, (B + 1) * 8, cudaMemcpyDeviceToDevice, st), "cudaMemcpyAsync");
    if (num_shards)
      cuda_ok(cudaMemcpyAsync(m->d_shard_off, shard_off, (num_shards + 1) * 8, cudaMemcpyDeviceToDevice, st),
              "cudaMemcpyAsync");
    else
      cuda_ok(cudaMemsetAsync(m->d_shard_off, 0, 8, st), "cudaMemsetAsync");
    cuda_ok(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    cuda_ok(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (rs == SHK_OK) rs = device_errors(h_err);
  }
  if (rs != SHK_OK) {
    cudaStreamSynchronize(st);
    free_mphf(m);
    return rs;
  }
  shk_stats& s = m->stats;
  s.n_keys = N;
  s.n_buckets = B;
  s.n_leaves = h_L;
  s.n_search_leaves = h_L;
  s.n_split_nodes = h_splits;
  s.leaf_seeds_executed = h_cnt[0];
  s.leaf_seeds_min = h_cnt[1];
  s.leaf_key_evals = h_cnt[2];
  s.leaf_hash_evals = h_cnt[3];
  s.leaf_seeds_tested = h_cnt[4];
  memcpy(&s.leaf_rf_cells, &h_cnt[5], sizeof(double));
  s.leaf_t0_ns = h_L ? h_ctl[0] : 0;
  s.leaf_t1_ns = h_ctl[1];
  s.device_bytes_peak = pool_used_high(false) + m->words * 8 + (B + 1) * 12 + (num_shards + 1) * 8;
  s.kernel_launches = c.launches;
  s.leaf_launches = leaf_launches;
  s.size_bits = m->words * 64;
  s.ms_fingerprint = pt.ms(t0, t1);
  s.ms_partition = pt.ms(t1, t1a) + pt.ms(t1b, t2);
  s.ms_split = pt.ms(t2, t3);
  s.ms_leaf = pt.ms(t3, t4);
  s.ms_orient = pt.ms(t4, t5);
  s.ms_encode = pt.ms(t5, t6);
  s.ms_ribbon = pt.ms(t6, t7);
  s.ms_total = pt.ms(t0, t7);
  s.leaf_cfg[0] = cfg.seeds_per_lane;
  s.leaf_cfg[1] = cfg.warps;
  s.leaf_cfg[2] = cfg.unroll;
  s.leaf_cfg[3] = cfg.passes;
  *out = m;
  return SHK_OK;
}

}  // namespace shk

using namespace shk;

extern "C" const char* shk_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* shk_version(void) { return "SHKRS002"; }

extern "C" void shk_release_memory(void) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (cudaMemPool_t p : g_pool)
    if (p) cudaMemPoolTrimTo(p, 0);
}

extern "C" shk_status shk_build(const shk_keys* keys, const shk_build_opts* opts, void* cuda_stream,
                                shk_mphf** out) {
  if (!out || !opts) return fail(SHK_EINVAL, "NULL argument");
  *out = nullptr;
  g_last_error.clear();
  shk_status st =
      no_throw([&] { return build_controlled(keys, opts, (cudaStream_t)cuda_stream, out, nullptr); });
  if (st != SHK_OK) cudaStreamSynchronize((cudaStream_t)cuda_stream);
  return st;
}

extern "C" shk_status shk_build_stats(const shk_mphf* m, shk_stats* out) {
  if (!m || !out) return fail(SHK_EINVAL, "NULL argument");
  *out = m->stats;
  return SHK_OK;
}

extern "C" uint64_t shk_size_bits(const shk_mphf* m) { return m ? m->words * 64 : 0; }

extern "C" void shk_free(shk_mphf* m) { free_mphf(m); }

extern "C" shk_status shk_serialize(const shk_mphf* m, uint8_t* buf, size_t cap, size_t* len) {
  if (!m || !len) return fail(SHK_EINVAL, "NULL argument");
  *len = m->words * 8;
  if (!buf) return SHK_OK;
  if (cap < *len) return fail(SHK_EINVAL, "buffer too small");
  SHK_CUDA(cudaMemcpy(buf, m->d_blob, *len, cudaMemcpyDeviceToHost));
  return SHK_OK;
}

static shk_status deserialize_impl(const uint8_t* buf, size_t len, shk_mphf** out) {
  if (!buf || !out) return fail(SHK_EINVAL, "NULL argument");
  *out = nullptr;
  if (len < kHeaderWords * 8 || len % 8) return fail(SHK_EFORMAT, "bad length");
  shk_mphf* m = new shk_mphf();
  memcpy(m->hdr, buf, sizeof m->hdr);
  const uint64_t* h = m->hdr;
  const uint64_t N = h[1], n = h[2], b = h[3], B = h[4], S = h[5];
  bool ok = h[0] == kMagic && n >= 2 && n <= kMaxLeaf && b >= n && b <= kMaxBucketSize &&
            N < (1ull << 32) && B == (N ? (N + b - 1) / b : 0) && S >= 1 &&
            h[7] == (B + S - 1) / S && h[9] < 64 && h[11] < 64 && h[9] == ef_low_bits(N, B + 1) &&
            h[10] == (N >> h[9]) + B + 1 && h[11] == ef_low_bits(h[8], B + 1) &&
            h[12] == (h[8] >> h[11]) + B + 1 && h[8] < (1ull << 48) && h[13] < (1ull << 48) &&
            h[14] <= 1 && h[15] == ribbon_width((uint32_t)n);
  if (ok) {
    layout(m);
    ok = m->words * 8 == len;
  }
  if (!ok) {
    delete m;
    return fail(SHK_EFORMAT, "not a well-formed SHKRS002 object");
  }
  Ctx c(nullptr);
  shk_status st = init_ctx(c);
  m->device = c.device;
  auto run = [&]() -> shk_status {
    SHK_CUDA(cudaMalloc(&m->d_blob, m->words * 8));
    SHK_CUDA(cudaMalloc(&m->d_K, (B + 1) * 4));
    SHK_CUDA(cudaMalloc(&m->d_O, (B + 1) * 8));
    SHK_CUDA(cudaMalloc(&m->d_shard_off, (h[7] + 1) * 8));
    SHK_CUDA(cudaMemcpy(m->d_blob, buf, len, cudaMemcpyHostToDevice));
    uint64_t* K64;
    SHK_TRY(c.arena.alloc(&K64, B + 1));
    SHK_TRY(launch_ef_decode(c, m->d_blob + m->off_kl, m->d_blob + m->off_kh, h[10], (uint32_t)h[9],
                             B + 1, K64));
    k_u64_to_u32<<<(unsigned)((B + 1 + 255) / 256), 256, 0, c.stream>>>(K64, B + 1, m->d_K);
    SHK_TRY(launch_ef_decode(c, m->d_blob + m->off_ol, m->d_blob + m->off_oh, h[12], (uint32_t)h[11],
                             B + 1, m->d_O));
    uint32_t* bad;
    uint32_t h_bad = 0;
    SHK_TRY(c.arena.alloc(&bad, 1, true));
    SHK_TRY(launch_validate_index(c, m->d_K, m->d_O, B, N, h[8], bad));
    SHK_CUDA(cudaMemcpyAsync(&h_bad, bad, 4, cudaMemcpyDeviceToHost, c.stream));
    SHK_CUDA(cudaStreamSynchronize(c.stream));
    if (h_bad) return fail(SHK_EFORMAT, "inconsistent bucket index");
    uint64_t* slots;
    SHK_TRY(c.arena.alloc(&slots, h[7]));
    SHK_TRY(launch_shard_slots(c, m->d_K, B, (uint32_t)S, (uint32_t)h[6], (uint32_t)h[15], h[7], slots));
    SHK_TRY((exclusive_scan<uint64_t, uint64_t>(c, slots, h[7], m->d_shard_off)));
    SHK_CUDA(cudaStreamSynchronize(c.stream));
    return SHK_OK;
  };
  if (st == SHK_OK) st = run();
  if (st != SHK_OK) {
    free_mphf(m);
    return st;
  }
  m->stats.n_keys = N;
  m->stats.n_buckets = B;
  m->stats.size_bits = m->words * 64;
  *out = m;
  return SHK_OK;
}

// The query index of m: built once, by the first query, on that query's stream
// (a cache of decoded codes; the object stays logically unchanged).  Published
// only after the build finished, so a concurrent query on another stream sees
// either no index or a complete one.
static shk_status ensure_qindex(Ctx& c, shk_mphf* m) {
  std::lock_guard<std::mutex> lk(m->qmu);
  const uint64_t B = m->hdr[4];
  if (m->d_qnode || B == 0) return SHK_OK;
  const uint32_t n = (uint32_t)m->hdr[2];
  uint32_t *nleaf, *ncode, *nsplit, *maxb;
  SHK_TRY(c.arena.alloc(&nleaf, B));
  SHK_TRY(c.arena.alloc(&ncode, B));
  SHK_TRY(c.arena.alloc(&nsplit, B));
  SHK_TRY(c.arena.alloc(&maxb, 1, true));
  SHK_TRY(launch_tree_count(c, m->d_K, B, n, nleaf, ncode, nsplit, maxb));
  uint32_t* qbase = nullptr;
  QNode* nodes = nullptr;
  auto cleanup = [&](shk_status st) {
    cudaStreamSynchronize(c.stream);
    if (qbase) cudaFree(qbase);
    if (nodes) cudaFree(nodes);
    return st;
  };
  if (cudaMalloc(&qbase, (B + 1) * 4) != cudaSuccess) return cleanup(fail(SHK_ENOMEM, "query index"));
  shk_status st = exclusive_scan<uint32_t, uint32_t>(c, ncode, B, qbase);
  if (st != SHK_OK) return cleanup(st);
  uint32_t total = 0;
  st = d2h(c, &total, qbase + B);
  if (st != SHK_OK || cudaStreamSynchronize(c.stream) != cudaSuccess)
    return cleanup(st != SHK_OK ? st : fail(SHK_ECUDA, "query index"));
  if (cudaMalloc(&nodes, (size_t)(total ? total : 1) * sizeof(QNode)) != cudaSuccess)
    return cleanup(fail(SHK_ENOMEM, "query index"));
  st = launch_qindex_build(c, m, qbase, nodes);
  if (st != SHK_OK || cudaStreamSynchronize(c.stream) != cudaSuccess)
    return cleanup(st != SHK_OK ? st : fail(SHK_ECUDA, "query index"));
  m->d_qbase = qbase;
  m->d_qnode = nodes;
  return SHK_OK;
}

static shk_status query_impl(const shk_mphf* m, const shk_keys* keys, uint64_t* ranks_out,
                                int out_on_device, void* cuda_stream) {
  if (!m || !ranks_out) return fail(SHK_EINVAL, "NULL argument");
  SHK_TRY(check_keys(keys));
  const uint64_t nq = keys->n_keys;
  if (nq && m->hdr[1] == 0) return fail(SHK_EINVAL, "query on an empty MPHF");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Ctx c(st);
  SHK_TRY(init_ctx(c));
  auto run = [&]() -> shk_status {
    const void* kdata;
    const uint64_t* koffs;
    SHK_TRY(stage_keys(c, keys, &kdata, &koffs));
    uint64_t *lo, *hi, *ranks = ranks_out;
    SHK_TRY(c.arena.alloc(&lo, nq));
    SHK_TRY(c.arena.alloc(&hi, nq));
    if (!out_on_device) SHK_TRY(c.arena.alloc(&ranks, nq));
    SHK_TRY(launch_fingerprint_only(c, keys->kind, kdata, koffs, nq, lo, hi));
    if (nq) SHK_TRY(ensure_qindex(c, const_cast<shk_mphf*>(m)));
    SHK_TRY(launch_query(c, m, lo, hi, nq, ranks));
    if (!out_on_device && nq)
      SHK_CUDA(cudaMemcpyAsync(ranks_out, ranks, nq * 8, cudaMemcpyDeviceToHost, st));
    SHK_CUDA(cudaStreamSynchronize(st));
    return SHK_OK;
  };
  shk_status s = run();
  if (s != SHK_OK) cudaStreamSynchronize(st);
  return s;
}

// The batched leaf search runs as one captured CUDA graph (descriptor kernel,
// state clears, the persistent search, orientation).  The instantiated graph
// and its working buffers are cached per host thread and replayed while the
// call's pointers, sizes and kernel configuration stay the same; a replay
// reads the buffers' current contents.
struct LeafGraph {
  bool valid = false;
  const uint64_t* keys = nullptr;
  const uint32_t* off = nullptr;
  uint32_t n = 0;
  uint64_t seed_start = 0;
  uint64_t* seeds = nullptr;
  uint64_t* fmask = nullptr;
  cudaStream_t stream = nullptr;
  int device = -1;
  LeafCfg cfg{};
  cudaGraphExec_t exec = nullptr;
  LeafDesc* d = nullptr;
  uint32_t* state = nullptr;             // work-distribution state
  unsigned long long* flags = nullptr;   // [0] seed counter, [1] error word
  uint64_t replays = 0;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (d) cudaFree(d);
    if (state) cudaFree(state);
    if (flags) cudaFree(flags);
    exec = nullptr;
    d = nullptr;
    state = nullptr;
    flags = nullptr;
    valid = false;
  }
};
static thread_local LeafGraph g_leaf_graph;
static thread_local cudaStream_t g_capture_stream[64];

static shk_status leaf_search_impl(const uint64_t* leaf_keys, const uint32_t* leaf_off,
                                      uint32_t n_leaves, uint64_t seed_start, uint64_t* seeds_out,
                                      uint64_t* f_out, void* cuda_stream) {
  if (n_leaves && (!leaf_keys || !leaf_off || !seeds_out)) return fail(SHK_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Ctx c(st);
  SHK_TRY(init_ctx(c));
  if (n_leaves == 0) return SHK_OK;
  if (c.device < 0 || c.device >= 64) return fail(SHK_EINVAL, "device ordinal out of range");
  // the legacy default stream cannot be captured: use a blocking stream of
  // the library, which is ordered with it
  cudaStream_t run_st = st;
  if (st == nullptr) {
    if (!g_capture_stream[c.device]) SHK_CUDA(cudaStreamCreate(&g_capture_stream[c.device]));
    run_st = g_capture_stream[c.device];
  }
  LeafCfg cfg;
  SHK_TRY(tuned_leaf_cfg(c, kMaxLeaf, &cfg));
  LeafGraph& g = g_leaf_graph;
  const bool hit = g.valid && g.keys == leaf_keys && g.off == leaf_off && g.n == n_leaves &&
                   g.seed_start == seed_start && g.seeds == seeds_out && g.fmask == f_out &&
                   g.stream == run_st && g.device == c.device &&
                   memcmp(&g.cfg, &cfg, sizeof cfg) == 0;
  const uint32_t L = n_leaves;
  const size_t state_words = (size_t)L + (L + 31) / 32 + 1;
  if (!hit) {
    g.release();
    SHK_CUDA(cudaMalloc(&g.d, (size_t)L * sizeof(LeafDesc)));
    SHK_CUDA(cudaMalloc(&g.state, state_words * sizeof(uint32_t)));
    // 64-bit atomics need 8-byte alignment: the flags get their own allocation
    SHK_CUDA(cudaMalloc(&g.flags, 2 * sizeof(unsigned long long)));
    unsigned long long* counter = g.flags;
    uint32_t* err = (uint32_t*)(g.flags + 1);
    Ctx cc(run_st);
    cc.num_sms = c.num_sms;
    cc.device = c.device;
    SHK_CUDA(cudaStreamBeginCapture(run_st, cudaStreamCaptureModeThreadLocal));
    auto capture = [&]() -> shk_status {
      SHK_CUDA(cudaMemsetAsync(g.flags, 0, 2 * sizeof(unsigned long long), run_st));
      k_leaf_descs<<<(L + 255) / 256, 256, 0, run_st>>>(leaf_off, L, g.d);
      SHK_CUDA(cudaGetLastError());
      SHK_CUDA(cudaMemsetAsync(seeds_out, 0xFF, (size_t)L * 8, run_st));
      LeafSearchArgs a{g.d, L, leaf_keys, seed_start, (unsigned long long*)seeds_out, err, counter, cfg};
      SHK_TRY(launch_leaf_persistent_state(cc, a, g.state));
      SHK_TRY(launch_orient(cc, g.d, L, leaf_keys, (unsigned long long*)seeds_out, nullptr, nullptr,
                            f_out, err));
      return SHK_OK;
    };
    const shk_status cs = capture();
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(run_st, &graph);
    if (cs != SHK_OK) {
      if (graph) cudaGraphDestroy(graph);
      g.release();
      return cs;
    }
    if (ee != cudaSuccess) {
      g.release();
      return fail(SHK_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ee));
    }
    const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      g.release();
      return fail(SHK_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
    }
    g.keys = leaf_keys;
    g.off = leaf_off;
    g.n = L;
    g.seed_start = seed_start;
    g.seeds = seeds_out;
    g.fmask = f_out;
    g.stream = run_st;
    g.device = c.device;
    g.cfg = cfg;
    g.valid = true;
  }
  uint32_t h_err = 0;
  auto run = [&]() -> shk_status {
    SHK_CUDA(cudaGraphLaunch(g.exec, run_st));
    g.replays++;
    SHK_CUDA(cudaMemcpyAsync(&h_err, (const uint32_t*)(g.flags + 1), 4, cudaMemcpyDeviceToHost, run_st));
    SHK_CUDA(cudaStreamSynchronize(run_st));
    return device_errors(h_err);
  };
  const shk_status s = run();
  if (s != SHK_OK) cudaStreamSynchronize(run_st);
  return s;
}

extern "C" uint64_t shk_leaf_graph_replays(void) { return g_leaf_graph.replays; }

static shk_status leaf_search_rf_impl(const uint64_t* leaf_keys, const uint32_t* leaf_off,
                                         uint32_t n_leaves, uint64_t* values_out, uint64_t* f_out,
                                         void* cuda_stream) {
  if (n_leaves && (!leaf_keys || !leaf_off || !values_out)) return fail(SHK_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Ctx c(st);
  SHK_TRY(init_ctx(c));
  if (n_leaves == 0) return SHK_OK;
  auto run = [&]() -> shk_status {
    LeafDesc* d;
    uint32_t* err;
    unsigned long long* counters;
    SHK_TRY(c.arena.alloc(&d, n_leaves));
    SHK_TRY(c.arena.alloc(&err, 1, true));
    SHK_TRY(c.arena.alloc(&counters, 1, true));
    k_leaf_descs<<<(n_leaves + 255) / 256, 256, 0, st>>>(leaf_off, n_leaves, d);
    c.launches++;
    SHK_CUDA(cudaGetLastError());
    SHK_CUDA(cudaMemsetAsync(values_out, 0xFF, (size_t)n_leaves * 8, st));
    LeafSearchArgs a{d, n_leaves, leaf_keys, 0, (unsigned long long*)values_out, err, counters,
                     LeafCfg{8, 8, 2, 2}};
    SHK_TRY(launch_leaf_rf_persistent(c, a));
    SHK_TRY(launch_orient(c, d, n_leaves, leaf_keys, (unsigned long long*)values_out, nullptr,
                          nullptr, f_out, err, SHK_LEAF_ROTATION));
    uint32_t h_err = 0;
    SHK_CUDA(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, st));
    SHK_CUDA(cudaStreamSynchronize(st));
    return device_errors(h_err);
  };
  const shk_status s = run();
  if (s != SHK_OK) cudaStreamSynchronize(st);
  return s;
}

static shk_status leaf_tune_impl(uint32_t leaf_size, uint32_t* cfg_out, double* evals_per_s,
                                    int probe_all, double* all_evals_per_s) {
  if (leaf_size < 2 || leaf_size > kMaxLeaf || !cfg_out) return fail(SHK_EINVAL, "bad argument");
  Ctx c(nullptr);
  SHK_TRY(init_ctx(c));
  LeafCfg cfg;
  SHK_TRY(tuned_leaf_cfg(c, leaf_size, &cfg));
  cfg_out[0] = cfg.seeds_per_lane;
  cfg_out[1] = cfg.warps;
  cfg_out[2] = cfg.unroll;
  cfg_out[3] = cfg.passes;
  if (evals_per_s) SHK_TRY(probe_leaf_cfg(c, cfg, leaf_size, evals_per_s, 3));
  if (probe_all && all_evals_per_s)
    for (int i = 0; i < leaf_cfg_count(); i++) SHK_TRY(probe_leaf_cfg(c, leaf_cfg_at(i), leaf_size, &all_evals_per_s[i], 3));
  return SHK_OK;
}

extern "C" uint32_t shk_leaf_configs(uint32_t* cfgs, uint32_t cap) {
  const uint32_t n = (uint32_t)leaf_cfg_count();
  for (uint32_t i = 0; i < n && i < cap; i++) {
    const LeafCfg c = leaf_cfg_at((int)i);
    cfgs[4 * i] = c.seeds_per_lane;
    cfgs[4 * i + 1] = c.warps;
    cfgs[4 * i + 2] = c.unroll;
    cfgs[4 * i + 3] = c.passes;
  }
  return n;
}

// C entry points over the implementations above; no host exception escapes.
extern "C" shk_status shk_deserialize(const uint8_t* buf, size_t len, shk_mphf** out) {
  return no_throw([&] { return deserialize_impl(buf, len, out); });
}

extern "C" shk_status shk_query(const shk_mphf* m, const shk_keys* keys, uint64_t* ranks_out,
                                int out_on_device, void* cuda_stream) {
  return no_throw([&] { return query_impl(m, keys, ranks_out, out_on_device, cuda_stream); });
}

extern "C" shk_status shk_leaf_search(const uint64_t* leaf_keys, const uint32_t* leaf_off,
                                      uint32_t n_leaves, uint64_t seed_start, uint64_t* seeds_out,
                                      uint64_t* f_out, void* cuda_stream) {
  return no_throw([&] {
    return leaf_search_impl(leaf_keys, leaf_off, n_leaves, seed_start, seeds_out, f_out, cuda_stream);
  });
}

extern "C" shk_status shk_leaf_search_rf(const uint64_t* leaf_keys, const uint32_t* leaf_off,
                                         uint32_t n_leaves, uint64_t* values_out, uint64_t* f_out,
                                         void* cuda_stream) {
  return no_throw([&] {
    return leaf_search_rf_impl(leaf_keys, leaf_off, n_leaves, values_out, f_out, cuda_stream);
  });
}

extern "C" shk_status shk_leaf_tune(uint32_t leaf_size, uint32_t* cfg_out, double* evals_per_s,
                                    int probe_all, double* all_evals_per_s) {
  return no_throw([&] { return leaf_tune_impl(leaf_size, cfg_out, evals_per_s, probe_all, all_evals_per_s); });
}
