// server.cu -- serving: a request loop over MPHF builds of different sizes.
//
// Requests are queued first in, first out.  A pool of worker threads, each
// with its own CUDA stream, admits the request at the head of the queue as
// soon as a worker is free and the request's estimated device footprint fits
// in what the budget leaves; a request larger than the whole budget runs alone.
// Builds of different requests run concurrently on their streams, so their
// kernels overlap on the GPU, and new requests are admitted while others run.
// Each build is exactly shk_build on the request's keys and options.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"

namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t id = 0;
  int32_t kind = 0;
  std::vector<uint8_t> data;      // host copy of host keys
  std::vector<uint64_t> offsets;  // string keys
  void* d_data = nullptr;         // device copy of device keys (library pool)
  uint64_t* d_offsets = nullptr;
  uint64_t n_keys = 0;
  shk_build_opts opts{};
  shk_request_info info{};
  shk_mphf* result = nullptr;
  volatile uint32_t* abort = nullptr;  // the running worker's flag
  bool cancelled = false;
};

// offsets[i] -= base on the device
__global__ void k_rebase(uint64_t* o, uint64_t n, uint64_t base) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] -= base;
}

// Device bytes a build holds while it runs: keys staged on the device, three
// 16-byte fingerprint copies (hashed, partitioned once and twice), the leaf
// order copy (lo, hi), orientation bytes, per-leaf arrays (up to ~30 bytes a
// key at the smallest leaves), per-bucket arrays, the encoded result, a fixed
// allowance; and with 128-bit retrieval rows the solver's scratch: its
// persistent warps' rows and bands, sized for a shard of 1.25 times the
// average shard's keys plus 512.
uint64_t footprint(uint64_t n_keys, const shk_build_opts& o, uint64_t key_bytes) {
  const uint64_t b = o.bucket_size ? o.bucket_size : 1;
  const uint64_t buckets = n_keys / b + 1;
  uint64_t bytes = key_bytes + n_keys * 96 + buckets * 96 + (8ull << 20);
  const uint32_t rw = shk::ribbon_width(o.leaf_size);
  if (rw == 128 && n_keys) {
    const uint64_t S = o.shard_buckets ? o.shard_buckets : shk::default_shard_buckets((uint32_t)b, rw);
    const uint64_t shards = (buckets + S - 1) / S;
    const uint32_t eps = o.eps_num ? o.eps_num : shk::default_eps_num(rw);
    uint64_t keys = n_keys / shards + n_keys / shards / 4 + 512;
    if (keys > n_keys) keys = n_keys;
    uint64_t scratch = 0;
    if (shk::ribbon128_scratch_bytes(shards, shk::shard_slots(keys, eps, rw), &scratch) == SHK_OK) bytes += scratch;
  }
  return bytes;
}

}  // namespace

struct shk_server {
  int device = 0;
  uint64_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> all;
  std::vector<std::thread> threads;
  uint64_t next_id = 1, in_use = 0, peak = 0, submitted = 0, completed = 0, running = 0;
  bool stop = false;
  cudaStream_t copy_stream = nullptr;  // copies of submitted device keys

  void worker() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    // cancellation flag, read by the build's leaf kernels (host-mapped)
    uint32_t* flag = nullptr;
    if (cudaHostAlloc((void**)&flag, sizeof(uint32_t), cudaHostAllocMapped) != cudaSuccess) flag = nullptr;
    for (;;) {
      Request* r = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] {
          if (stop) return true;
          if (queue.empty()) return false;
          const uint64_t fp = queue.front()->info.footprint_bytes;
          return in_use + fp <= budget || running == 0;
        });
        if (stop) break;
        r = queue.front();
        queue.pop_front();
        in_use += r->info.footprint_bytes;
        if (in_use > peak) peak = in_use;
        running++;
        r->info.start_ns = now_ns();
        if (flag) *(volatile uint32_t*)flag = 0;
        r->abort = flag;
      }
      shk_keys k;
      k.kind = r->kind;
      k.on_device = r->d_data != nullptr;
      k.data = k.on_device ? r->d_data : r->data.data();
      k.str_offsets = k.on_device ? r->d_offsets : (r->offsets.empty() ? nullptr : r->offsets.data());
      k.n_keys = r->n_keys;
      shk_mphf* m = nullptr;
      shk_status s = shk::no_throw([&] { return shk::build_controlled(&k, &r->opts, st, &m, flag); });
      if (s != SHK_OK) cudaStreamSynchronize(st);
      if (r->d_data) cudaFreeAsync(r->d_data, st);
      if (r->d_offsets) cudaFreeAsync(r->d_offsets, st);
      {
        std::lock_guard<std::mutex> lk(mu);
        r->abort = nullptr;
        r->d_data = nullptr;
        r->d_offsets = nullptr;
        if (r->cancelled && s == SHK_OK) {  // finished before the flag was seen
          shk_free(m);
          m = nullptr;
          s = SHK_ECANCELLED;
        }
        r->result = m;
        r->info.status = s;
        r->info.done = 1;
        r->info.finish_ns = now_ns();
        r->data.clear();
        r->data.shrink_to_fit();
        r->offsets.clear();
        r->offsets.shrink_to_fit();
        in_use -= r->info.footprint_bytes;
        running--;
        completed++;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
    if (st) cudaStreamDestroy(st);
    if (flag) cudaFreeHost(flag);
  }
};

using namespace shk;

static shk_status server_create(uint64_t hbm_budget_bytes, uint32_t workers, shk_server** out) {
  std::unique_ptr<shk_server> s(new shk_server());
  if (cudaGetDevice(&s->device) != cudaSuccess) return fail(SHK_ECUDA, "cudaGetDevice failed");
  if (hbm_budget_bytes == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(SHK_ECUDA, "cudaMemGetInfo failed");
    hbm_budget_bytes = (uint64_t)(free_b * 0.8);
  }
  s->budget = hbm_budget_bytes;
  if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(SHK_ECUDA, "cudaStreamCreate failed");
  const uint32_t w = workers ? workers : 4;
  shk_server* raw = s.get();
  try {
    for (uint32_t i = 0; i < w; i++) s->threads.emplace_back([raw] { raw->worker(); });
  } catch (...) {
    shk_server_destroy(s.release());  // stops and joins the workers already started
    throw;
  }
  *out = s.release();
  return SHK_OK;
}

extern "C" shk_status shk_server_create(uint64_t hbm_budget_bytes, uint32_t workers,
                                        shk_server** out) {
  if (!out) return fail(SHK_EINVAL, "NULL argument");
  *out = nullptr;
  return no_throw([&] { return server_create(hbm_budget_bytes, workers, out); });
}

// Bytes of a key set as the build stages it on the device.
static uint64_t key_bytes(const shk_keys* keys) {
  const uint64_t N = keys->n_keys;
  if (keys->kind == SHK_KEYS_U64) return N * 8;
  if (keys->kind == SHK_KEYS_FP128) return N * 16;
  uint64_t span = 0;
  if (N) {
    uint64_t ends[2] = {0, 0};
    if (keys->on_device) {
      cudaMemcpy(&ends[0], keys->str_offsets, 8, cudaMemcpyDeviceToHost);
      cudaMemcpy(&ends[1], keys->str_offsets + N, 8, cudaMemcpyDeviceToHost);
    } else {
      ends[0] = keys->str_offsets[0];
      ends[1] = keys->str_offsets[N];
    }
    span = ends[1] - ends[0];
  }
  return span + 8 * (N + 1);
}

// Device keys into the library's pool on the server's device (its current
// device is set for the copy and restored): u64 and 128-bit keys as they
// are, string bytes from offsets[0] on with their offsets rebased to 0.
static shk_status copy_device_keys(shk_server* srv, const shk_keys* keys, Request* r) {
  int old = 0;
  SHK_CUDA(cudaGetDevice(&old));
  SHK_CUDA(cudaSetDevice(srv->device));
  auto run = [&]() -> shk_status {
    cudaStream_t cs = srv->copy_stream;
    const uint64_t N = keys->n_keys;
    if (keys->kind == SHK_KEYS_STR) {
      uint64_t ends[2] = {0, 0};
      if (N) {
        SHK_CUDA(cudaMemcpyAsync(&ends[0], keys->str_offsets, 8, cudaMemcpyDeviceToHost, cs));
        SHK_CUDA(cudaMemcpyAsync(&ends[1], keys->str_offsets + N, 8, cudaMemcpyDeviceToHost, cs));
        SHK_CUDA(cudaStreamSynchronize(cs));
      }
      const uint64_t total = ends[1] - ends[0];
      SHK_CUDA(pool_malloc(&r->d_data, total + 8, cs));
      SHK_CUDA(pool_malloc((void**)&r->d_offsets, (N + 1) * 8, cs));
      if (total)
        SHK_CUDA(cudaMemcpyAsync(r->d_data, (const uint8_t*)keys->data + ends[0], total,
                                 cudaMemcpyDeviceToDevice, cs));
      SHK_CUDA(cudaMemcpyAsync(r->d_offsets, keys->str_offsets, (N + 1) * 8, cudaMemcpyDeviceToDevice, cs));
      if (ends[0]) k_rebase<<<(unsigned)((N + 1 + 255) / 256), 256, 0, cs>>>(r->d_offsets, N + 1, ends[0]);
      SHK_CUDA(cudaGetLastError());
    } else {
      const uint64_t bytes = N * (keys->kind == SHK_KEYS_U64 ? 8 : 16);
      SHK_CUDA(pool_malloc(&r->d_data, bytes ? bytes : 16, cs));
      if (bytes) SHK_CUDA(cudaMemcpyAsync(r->d_data, keys->data, bytes, cudaMemcpyDeviceToDevice, cs));
    }
    SHK_CUDA(cudaStreamSynchronize(cs));
    return SHK_OK;
  };
  shk_status s = run();
  if (s != SHK_OK) {
    cudaStreamSynchronize(srv->copy_stream);
    if (r->d_data) cudaFreeAsync(r->d_data, srv->copy_stream);
    if (r->d_offsets) cudaFreeAsync(r->d_offsets, srv->copy_stream);
    r->d_data = nullptr;
    r->d_offsets = nullptr;
  }
  cudaSetDevice(old);
  return s;
}

static shk_status server_submit(shk_server* srv, const shk_keys* keys, const shk_build_opts* opts,
                                uint64_t* req_id) {
  if (keys->kind != SHK_KEYS_U64 && keys->kind != SHK_KEYS_STR && keys->kind != SHK_KEYS_FP128)
    return fail(SHK_EINVAL, "unknown key kind");
  const uint64_t N = keys->n_keys;
  if (N && !keys->data) return fail(SHK_EINVAL, "key data is NULL");
  if (keys->kind == SHK_KEYS_STR && N && !keys->str_offsets)
    return fail(SHK_EINVAL, "string keys need str_offsets");
  std::unique_ptr<Request> r(new Request());
  r->kind = keys->kind;
  r->n_keys = N;
  r->opts = *opts;
  r->opts.profile = 0;
  // copy the keys now: the caller's buffers are only borrowed for this call.
  // Device keys stay on the device (a copy into the library's pool, made on
  // the server's copy stream and waited for); host keys are copied on the host.
  if (keys->on_device) {
    SHK_TRY(copy_device_keys(srv, keys, r.get()));
  } else if (keys->kind == SHK_KEYS_STR) {
    r->offsets.assign(keys->str_offsets, keys->str_offsets + N + 1);
    const uint64_t base = r->offsets[0], total = r->offsets[N] - base;
    r->data.resize(total + 8);
    if (total) memcpy(r->data.data(), (const uint8_t*)keys->data + base, total);
    for (auto& v : r->offsets) v -= base;
  } else {
    const uint64_t bytes = N * (keys->kind == SHK_KEYS_U64 ? 8 : 16);
    r->data.resize(bytes ? bytes : 8);
    if (bytes) memcpy(r->data.data(), keys->data, bytes);
  }
  r->info.n_keys = N;
  r->info.footprint_bytes = footprint(N, *opts, key_bytes(keys));
  r->info.submit_ns = now_ns();
  const uint64_t id = [&] {
    std::lock_guard<std::mutex> lk(srv->mu);
    r->id = srv->next_id++;
    srv->all[r->id] = r.get();
    try {
      srv->queue.push_back(r.get());
    } catch (...) {
      srv->all.erase(r->id);
      throw;
    }
    srv->submitted++;
    return r.release()->id;
  }();
  srv->cv_work.notify_all();
  *req_id = id;
  return SHK_OK;
}

extern "C" shk_status shk_server_submit(shk_server* srv, const shk_keys* keys,
                                        const shk_build_opts* opts, uint64_t* req_id) {
  if (!srv || !keys || !opts || !req_id) return fail(SHK_EINVAL, "NULL argument");
  return no_throw([&] { return server_submit(srv, keys, opts, req_id); });
}

static shk_status poll_locked(shk_server* srv, uint64_t req_id, shk_mphf** out,
                              shk_request_info* info, std::unique_lock<std::mutex>& lk, bool wait) {
  // A waiter looks the request up again after every wake-up: another thread
  // may have collected (and freed) it meanwhile.
  auto it = srv->all.find(req_id);
  if (wait)
    srv->cv_done.wait(lk, [&] {
      it = srv->all.find(req_id);
      return it == srv->all.end() || it->second->info.done != 0;
    });
  if (it == srv->all.end()) return fail(SHK_EINVAL, "unknown request id");
  Request* r = it->second;
  if (info) *info = r->info;
  if (out) *out = nullptr;
  if (!r->info.done) return SHK_OK;
  if (out)
    *out = r->result;
  else if (r->result)
    shk_free(r->result);
  srv->all.erase(it);
  delete r;
  return SHK_OK;
}

extern "C" shk_status shk_server_poll(shk_server* srv, uint64_t req_id, shk_mphf** out,
                                      shk_request_info* info) {
  if (!srv) return fail(SHK_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(srv->mu);
  return poll_locked(srv, req_id, out, info, lk, false);
}

extern "C" shk_status shk_server_wait(shk_server* srv, uint64_t req_id, shk_mphf** out,
                                      shk_request_info* info) {
  if (!srv) return fail(SHK_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(srv->mu);
  return poll_locked(srv, req_id, out, info, lk, true);
}

extern "C" shk_status shk_server_get_stats(shk_server* srv, shk_server_stats* out) {
  if (!srv || !out) return fail(SHK_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  out->submitted = srv->submitted;
  out->completed = srv->completed;
  out->queued = srv->queue.size();
  out->running = srv->running;
  out->budget_bytes = srv->budget;
  out->in_use_bytes = srv->in_use;
  out->peak_in_use_bytes = srv->peak;
  out->workers = (uint32_t)srv->threads.size();
  return SHK_OK;
}

extern "C" void shk_server_destroy(shk_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->threads) t.join();
  for (auto& kv : srv->all) {
    if (kv.second->result) shk_free(kv.second->result);
    if (kv.second->d_data) cudaFreeAsync(kv.second->d_data, srv->copy_stream);
    if (kv.second->d_offsets) cudaFreeAsync(kv.second->d_offsets, srv->copy_stream);
    delete kv.second;
  }
  if (srv->copy_stream) {
    cudaStreamSynchronize(srv->copy_stream);
    cudaStreamDestroy(srv->copy_stream);
  }
  delete srv;
}

extern "C" shk_status shk_server_cancel(shk_server* srv, uint64_t req_id) {
  if (!srv) return fail(SHK_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->all.find(req_id);
  if (it == srv->all.end()) return fail(SHK_EINVAL, "unknown request id");
  Request* r = it->second;
  if (r->info.done) return SHK_OK;
  r->cancelled = true;
  for (auto q = srv->queue.begin(); q != srv->queue.end(); ++q) {
    if (*q != r) continue;  // still queued: it never runs
    srv->queue.erase(q);
    r->info.done = 1;
    r->info.status = SHK_ECANCELLED;
    r->info.finish_ns = now_ns();
    if (r->d_data) cudaFreeAsync(r->d_data, srv->copy_stream);
    if (r->d_offsets) cudaFreeAsync(r->d_offsets, srv->copy_stream);
    r->d_data = nullptr;
    r->d_offsets = nullptr;
    srv->completed++;
    lk.unlock();
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
    return SHK_OK;
  }
  if (r->abort) *r->abort = 1;  // running: its leaf search stops at its next work item
  return SHK_OK;
}

extern "C" shk_status shk_build_footprint(const shk_keys* keys, const shk_build_opts* opts,
                                          uint64_t* bytes) {
  if (!keys || !opts || !bytes) return fail(SHK_EINVAL, "NULL argument");
  if (keys->kind == SHK_KEYS_STR && keys->n_keys && !keys->str_offsets)
    return fail(SHK_EINVAL, "string keys need str_offsets");
  return no_throw([&] {
    *bytes = footprint(keys->n_keys, *opts, key_bytes(keys));
    return SHK_OK;
  });
}
