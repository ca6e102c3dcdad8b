// leaf.cu -- ShockHash leaf seed search (paper Sec. 4, Eq. ShockHash) with the
// bit-mask filter (Sec. 4, Filter by Bit Mask), the union-find pseudoforest test
// of filter survivors (App. A.1) and the orientation of the winning graph
// (Sec. 5, Eq. orientations-cycles).
//
// Warp design: the 32 lanes of a warp test consecutive seeds of one leaf; each
// lane carries U seeds at once, so every key read from shared memory (a
// broadcast) feeds U hash evaluations.  A lane keeps each seed's 64-bit
// candidate mask in two 32-bit registers; a seed survives the filter when the
// mask has all m bits set.  Survivors (rare) are tested by the whole warp:
// lanes hash the edges into shared memory and lane 0 runs a union-find with
// tree/pseudotree labels.  Seeds are taken in increasing order, so the first
// survivor that passes is the leaf's minimum seed within the work item.
#include <algorithm>
#include <mutex>

#include "kernels.cuh"

namespace shk {

constexpr unsigned kFull = 0xFFFFFFFFu;

struct WarpScratch {
  uint64_t x[kMaxLeaf];
  uint8_t e0[kMaxLeaf], e1[kMaxLeaf], parent[kMaxLeaf], cyc[kMaxLeaf];
};

// 1 << h with PTX clamping: shifts of 32 or more give 0.
__device__ __forceinline__ uint32_t bit32(uint32_t h) {
  uint32_t r;
  asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(1u), "r"(h));
  return r;
}

__device__ __forceinline__ uint32_t uf_find(uint8_t* parent, uint32_t v) {
  while (parent[v] != v) {
    const uint32_t p = parent[v];
    parent[v] = parent[p];
    v = parent[p];
  }
  return v;
}

// Union-find pseudoforest test (App. A.1): every set starts as a tree; an edge
// inside a tree makes it a pseudotree, an edge inside a pseudotree or between
// two pseudotrees fails.  Run by the whole warp, result in every lane.
__device__ bool pf_test(WarpScratch* ws, uint32_t m, uint64_t seed) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t c = mix64(kLeafSalt + seed);
  for (uint32_t i = lane; i < m; i += 32) {
    uint32_t h0, h1;
    leaf_cells(ws->x[i], c, m, &h0, &h1);
    ws->e0[i] = (uint8_t)h0;
    ws->e1[i] = (uint8_t)h1;
    ws->parent[i] = (uint8_t)i;
    ws->cyc[i] = 0;
  }
  __syncwarp();
  int ok = 1;
  if (lane == 0) {
    for (uint32_t e = 0; e < m; e++) {
      const uint32_t a = uf_find(ws->parent, ws->e0[e]);
      const uint32_t b = uf_find(ws->parent, ws->e1[e]);
      if (a == b) {
        if (ws->cyc[a]) {
          ok = 0;
          break;
        }
        ws->cyc[a] = 1;
      } else {
        if (ws->cyc[a] & ws->cyc[b]) {
          ok = 0;
          break;
        }
        ws->parent[a] = (uint8_t)b;
        ws->cyc[b] |= ws->cyc[a];
      }
    }
  }
  ok = __shfl_sync(kFull, ok, 0);
  __syncwarp();
  return ok != 0;
}

// Warp-uniform read of a value other warps update.
__device__ __forceinline__ uint64_t read_uniform(const volatile unsigned long long* p) {
  unsigned long long v = 0;
  if ((threadIdx.x & 31) == 0) v = *p;
  return __shfl_sync(0xFFFFFFFFu, v, 0);
}

// Search seeds s0 .. s0 + passes*32*U - 1 of the leaf held in ws->x.
// Returns the smallest passing seed, or ~0 if none (or if *best drops to or
// below the seeds still to test).  Called by a whole warp; *done counts the
// seeds evaluated.

template <int U, int UNROLL, bool WIDE>
__device__ uint64_t search_seeds(WarpScratch* ws, uint32_t m, uint64_t s0, uint32_t passes,
                                 const volatile unsigned long long* best, uint32_t* done) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t full_lo = m >= 32 ? 0xFFFFFFFFu : ((1u << m) - 1u);
  const uint32_t full_hi = m >= 64 ? 0xFFFFFFFFu : (m > 32 ? ((1u << (m - 32)) - 1u) : 0u);
  const uint32_t m1 = m - 1;
  for (uint32_t pass = 0; pass < passes; pass++) {
    const uint64_t base = s0 + (uint64_t)pass * (32u * U);
    if (best != nullptr && base >= read_uniform(best)) return ~0ull;
    *done += 32u * U;
    uint32_t cl[U], ch[U];
    uint64_t mask[U];  // covered cells; bit h = cell h (m <= 32: the low word only)
#pragma unroll
    for (int u = 0; u < U; u++) {
      const uint64_t c = mix64(kLeafSalt + base + (uint64_t)(u * 32) + lane);
      cl[u] = (uint32_t)c;
      ch[u] = (uint32_t)(c >> 32);
      mask[u] = 0;
    }
#pragma unroll UNROLL
    for (uint32_t i = 0; i < m; i++) {
      // ws->x holds (lo32(x), hi32(x) | 1): the key's xor input and multiplier
      const uint64_t x = ws->x[i];
      const uint32_t xl = (uint32_t)x, mult = (uint32_t)(x >> 32);
#pragma unroll
      for (int u = 0; u < U; u++) {
        const uint32_t a = (xl ^ cl[u]) * mult + ch[u];
        const uint64_t w = (uint64_t)a * m;
        const uint32_t h0 = (uint32_t)(w >> 32);
        const uint32_t t = __umulhi((uint32_t)w, m1);
        const uint32_t h1 = t + (t >= h0 ? 1u : 0u);
        if (WIDE)
          mask[u] |= (1ull << h0) | (1ull << h1);
        else
          mask[u] |= bit32(h0) | bit32(h1);
      }
    }
    const uint64_t full = ((uint64_t)full_hi << 32) | full_lo;
    bool any = false;
    bool cov[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      cov[u] = mask[u] == full;
      any |= cov[u];
    }
    if (__ballot_sync(kFull, any)) {
#pragma unroll
      for (int u = 0; u < U; u++) {
        uint32_t bal = __ballot_sync(kFull, cov[u]);
        while (bal) {
          const uint32_t l = __ffs(bal) - 1;
          const uint64_t s = base + (uint64_t)(u * 32) + l;
          if (pf_test(ws, m, s)) return s;
          bal &= bal - 1;
        }
      }
    }
  }
  return ~0ull;
}

template <int U, int UNROLL>
__device__ __forceinline__ uint64_t search_dispatch(WarpScratch* ws, uint32_t m, uint64_t s0,
                                                    uint32_t passes,
                                                    const volatile unsigned long long* best,
                                                    uint32_t* done) {
  return m > 32 ? search_seeds<U, UNROLL, true>(ws, m, s0, passes, best, done)
                : search_seeds<U, UNROLL, false>(ws, m, s0, passes, best, done);
}

// Keys of a leaf into shared memory with the multiplier's low bit set
// (leaf_cells gives the same cells for x and for x with that bit set).
__device__ __forceinline__ uint64_t leaf_input(uint64_t x) { return x | (1ull << 32); }

__device__ __forceinline__ void load_leaf(WarpScratch* ws, const LeafDesc& d, const uint64_t* x) {
  const uint32_t lane = threadIdx.x & 31;
  for (uint32_t i = lane; i < d.m; i += 32) ws->x[i] = leaf_input(x[d.key_off + i]);
  __syncwarp();
}

// Find a leaf whose result is still open (no passing seed yet).  Each lane
// reads one word of the closed-leaf bitmap per step.
__device__ uint32_t find_open_leaf(const uint32_t* closed, uint32_t n_leaves, uint32_t* pos,
                                   uint32_t salt) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwords = (n_leaves + 31) / 32;
  const uint32_t tail = n_leaves & 31;
  for (uint32_t t = 0; t < nwords; t += 32) {
    const uint32_t wi = (*pos + t + lane) % nwords;
    uint32_t open = 0;
    if (t + lane < nwords) {
      const uint32_t valid = (wi == nwords - 1 && tail) ? ((1u << tail) - 1u) : 0xFFFFFFFFu;
      open = ~*(const volatile uint32_t*)&closed[wi] & valid;
    }
    const uint32_t bal = __ballot_sync(kFull, open != 0);
    if (bal) {
      const uint32_t src = __ffs(bal) - 1;
      uint32_t o = __shfl_sync(kFull, open, src);
      const uint32_t w = __shfl_sync(kFull, wi, src);
      *pos = w;
      // spread helpers over the open leaves of the word
      uint32_t k = salt % (uint32_t)__popc(o);
      while (k--) o &= o - 1;
      return w * 32 + (uint32_t)(__ffs(o) - 1);
    }
  }
  return n_leaves;
}

// Persistent kernel: every warp takes fresh leaves from a global counter; when
// none is left it joins leaves that are still open.  Work items are chunks of
// consecutive seeds of one leaf, handed out in increasing order by a per-leaf
// counter; a found seed is committed with atomicMin, so the result is the
// minimum whatever the schedule: every chunk below the final minimum was
// handed out before the chunk that found it and is searched to its end.
template <int U, int WARPS, int UNROLL>
__global__ void __launch_bounds__(WARPS * 32)
    k_leaf_persistent(const LeafDesc* __restrict__ leaves, uint32_t n_leaves,
                      const uint64_t* __restrict__ x, uint64_t seed_start, uint32_t passes,
                      unsigned long long* best, uint32_t* next_chunk, uint32_t* closed,
                      uint32_t* next_leaf, unsigned long long* executed, uint32_t* err, LeafCtl ctl) {
  __shared__ WarpScratch scratch[WARPS];
  const uint32_t lane = threadIdx.x & 31;
  WarpScratch* ws = &scratch[threadIdx.x >> 5];
  const uint32_t gw = blockIdx.x * WARPS + (threadIdx.x >> 5);
  leaf_mark_start(ctl);
  bool stop = false;
  const uint32_t nwords = (n_leaves + 31) / 32;
  uint32_t pos = nwords ? (uint32_t)(((uint64_t)gw * 2654435761u) % nwords) : 0;
  const uint64_t chunk = (uint64_t)passes * 32u * U;
  unsigned long long done_seeds = 0;
  while (!stop) {
    uint32_t leaf = 0;
    if (lane == 0) leaf = atomicAdd(next_leaf, 1u);
    leaf = __shfl_sync(kFull, leaf, 0);
    if (leaf >= n_leaves) {
      leaf = find_open_leaf(closed, n_leaves, &pos, gw);
      if (leaf >= n_leaves) break;
    }
    const LeafDesc d = leaves[leaf];
    if (d.m < 2 || d.m > kMaxLeaf) {  // a 1-key leaf has no hash: its seed is seed_start
      if (lane == 0) {
        if (d.m == 1)
          best[leaf] = seed_start;
        else
          atomicOr(err, kErrLeafSize);
        atomicOr(&closed[leaf >> 5], 1u << (leaf & 31));
      }
      continue;
    }
    load_leaf(ws, d, x);
    for (;;) {
      if (leaf_should_stop(ctl, err)) {
        stop = true;
        break;
      }
      uint32_t ci = 0;
      if (lane == 0) ci = atomicAdd(&next_chunk[leaf], 1u);
      ci = __shfl_sync(kFull, ci, 0);
      const uint64_t s0 = seed_start + (uint64_t)ci * chunk;
      if (s0 >= read_uniform(&best[leaf])) break;
      if (s0 >= kSeedCap) {
        if (lane == 0) {
          atomicOr(err, kErrSeedCap);
          atomicOr(&closed[leaf >> 5], 1u << (leaf & 31));
        }
        break;
      }
      uint32_t done = 0;
      const uint64_t r = search_dispatch<U, UNROLL>(ws, d.m, s0, passes, &best[leaf], &done);
      done_seeds += done;
      if (r != ~0ull) {
        if (lane == 0) {
          atomicMin(&best[leaf], (unsigned long long)r);
          atomicOr(&closed[leaf >> 5], 1u << (leaf & 31));
        }
        break;
      }
    }
    __syncwarp();
  }
  if (lane == 0 && done_seeds) atomicAdd(executed, done_seeds);
  leaf_mark_end(ctl);
}

// One warp per leaf, no sharing: the plain form that is launched once per
// bucket over that bucket's leaves.
template <int U, int WARPS, int UNROLL>
__global__ void __launch_bounds__(WARPS * 32)
    k_leaf_range(const LeafDesc* __restrict__ leaves, uint32_t l0, uint32_t l1,
                 const uint64_t* __restrict__ x, uint64_t seed_start, uint32_t passes,
                 unsigned long long* best, unsigned long long* executed, uint32_t* err,
                 LeafCtl ctl) {
  __shared__ WarpScratch scratch[WARPS];
  const uint32_t lane = threadIdx.x & 31;
  WarpScratch* ws = &scratch[threadIdx.x >> 5];
  const uint32_t leaf = l0 + blockIdx.x * WARPS + (threadIdx.x >> 5);
  if (leaf >= l1) return;
  const LeafDesc d = leaves[leaf];
  load_leaf(ws, d, x);
  const uint64_t chunk = (uint64_t)passes * 32u * U;
  unsigned long long done_seeds = 0;
  for (uint64_t s0 = seed_start;; s0 += chunk) {
    if (s0 >= kSeedCap) {
      if (lane == 0) atomicOr(err, kErrSeedCap);
      break;
    }
    if (leaf_should_stop(ctl, err)) break;
    uint32_t done = 0;
    const uint64_t r = search_dispatch<U, UNROLL>(ws, d.m, s0, passes, nullptr, &done);
    done_seeds += done;
    if (r != ~0ull) {
      if (lane == 0) best[leaf] = r;
      break;
    }
  }
  if (lane == 0) atomicAdd(executed, done_seeds);
}

// Keys of the tuner's synthetic leaves.
__global__ void k_probe_keys(uint64_t* keys, uint64_t n, uint64_t salt) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) keys[i] = mix64(salt + i * 0x9E3779B97F4A7C15ull);
}

// ---------------------------------------------------------------------------
// configurations: seeds per lane x warps per block x key-loop unroll
// ---------------------------------------------------------------------------
struct LeafKernels {
  LeafCfg cfg;
  void (*persistent)(const LeafDesc*, uint32_t, const uint64_t*, uint64_t, uint32_t,
                     unsigned long long*, uint32_t*, uint32_t*, uint32_t*, unsigned long long*,
                     uint32_t*, LeafCtl);
  void (*range)(const LeafDesc*, uint32_t, uint32_t, const uint64_t*, uint64_t, uint32_t,
                unsigned long long*, unsigned long long*, uint32_t*, LeafCtl);
};

#define SHK_LEAF_CFG(U, W, R) {{U, W, R, 0}, k_leaf_persistent<U, W, R>, k_leaf_range<U, W, R>}

static const LeafKernels kLeafTable[] = {
    SHK_LEAF_CFG(1, 8, 2), SHK_LEAF_CFG(2, 4, 2), SHK_LEAF_CFG(2, 8, 2), SHK_LEAF_CFG(2, 8, 4),
    SHK_LEAF_CFG(2, 16, 2), SHK_LEAF_CFG(4, 4, 2), SHK_LEAF_CFG(4, 8, 1), SHK_LEAF_CFG(4, 8, 2),
    SHK_LEAF_CFG(4, 8, 4), SHK_LEAF_CFG(4, 16, 2)};
constexpr int kNumLeafCfg = sizeof(kLeafTable) / sizeof(kLeafTable[0]);

static const LeafKernels* find_kernels(const LeafCfg& c) {
  for (int i = 0; i < kNumLeafCfg; i++) {
    const LeafCfg& t = kLeafTable[i].cfg;
    if (t.seeds_per_lane == c.seeds_per_lane && t.warps == c.warps && t.unroll == c.unroll)
      return &kLeafTable[i];
  }
  return nullptr;
}

bool leaf_cfg_valid(const LeafCfg& c) { return find_kernels(c) != nullptr && c.passes >= 1; }

int leaf_cfg_count() { return kNumLeafCfg; }

LeafCfg leaf_cfg_at(int i) { return kLeafTable[i].cfg; }

static shk_status persistent_blocks(Ctx& c, const LeafKernels* k, uint32_t* blocks) {
  int per_sm = 0;
  SHK_TRY(blocks_per_sm((const void*)k->persistent, (int)k->cfg.warps * 32, 0, &per_sm));
  if (per_sm < 1) per_sm = 1;
  *blocks = (uint32_t)(c.num_sms * per_sm);
  return SHK_OK;
}

// 64-bit atomics (seed minimum, seed counter) need 8-byte aligned targets.
static bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

static shk_status launch_persistent_with(Ctx& c, const LeafSearchArgs& a, uint32_t* state) {
  const LeafKernels* k = find_kernels(a.cfg);
  if (!k) return fail(SHK_EINVAL, "unsupported leaf kernel configuration");
  if (!aligned8(a.best) || !aligned8(a.executed) || !aligned8(a.x))
    return fail(SHK_EINVAL, "seed, counter and key buffers must be 8-byte aligned");
  const uint32_t L = a.n_leaves;
  const uint32_t nwords = (L + 31) / 32;
  uint32_t blocks;
  SHK_TRY(persistent_blocks(c, k, &blocks));
  k->persistent<<<blocks, k->cfg.warps * 32, 0, c.stream>>>(
      a.leaves, L, a.x, a.seed_start, a.cfg.passes, a.best, state, state + L, state + L + nwords,
      a.executed, a.err, a.ctl);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

shk_status launch_leaf_persistent(Ctx& c, const LeafSearchArgs& a) {
  if (a.n_leaves == 0) return SHK_OK;
  uint32_t* state;
  const uint32_t L = a.n_leaves;
  // next_chunk[L] | closed[(L + 31) / 32] | next_leaf[1]
  SHK_TRY(c.arena.alloc(&state, (size_t)L + (L + 31) / 32 + 1, true));
  return launch_persistent_with(c, a, state);
}

// Same launch with the work-distribution state supplied by the caller:
// state = next_chunk[L] | closed[(L + 31) / 32] | next_leaf[1], zeroed here.
shk_status launch_leaf_persistent_state(Ctx& c, const LeafSearchArgs& a, uint32_t* state) {
  if (a.n_leaves == 0) return SHK_OK;
  const uint32_t L = a.n_leaves;
  SHK_CUDA(cudaMemsetAsync(state, 0, ((size_t)L + (L + 31) / 32 + 1) * sizeof(uint32_t), c.stream));
  return launch_persistent_with(c, a, state);
}

shk_status launch_leaf_range(Ctx& c, const LeafSearchArgs& a, uint32_t l0, uint32_t l1) {
  if (l1 <= l0) return SHK_OK;
  const LeafKernels* k = find_kernels(a.cfg);
  if (!k) return fail(SHK_EINVAL, "unsupported leaf kernel configuration");
  if (!aligned8(a.best) || !aligned8(a.executed) || !aligned8(a.x))
    return fail(SHK_EINVAL, "seed, counter and key buffers must be 8-byte aligned");
  const uint32_t W = k->cfg.warps;
  const uint32_t blocks = (l1 - l0 + W - 1) / W;
  k->range<<<blocks, W * 32, 0, c.stream>>>(a.leaves, l0, l1, a.x, a.seed_start, a.cfg.passes,
                                            a.best, a.executed, a.err, a.ctl);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: for each leaf-size bin (m <= 16, 17-32, 33-48, 49-64) time every
// configuration on synthetic leaves of the bin's largest size and keep the
// fastest (key-seed evaluations per second).  Results are cached per device.
// The configuration never changes results, only speed.
// ---------------------------------------------------------------------------
struct TuneSlot {
  bool done = false;
  LeafCfg cfg{4, 8, 2, 8};
  double evals_per_s = 0;
};
static std::mutex g_tune_mutex;
static TuneSlot g_tune[64][4];

static uint32_t default_passes(uint32_t m) { return m <= 16 ? 2u : (m <= 32 ? 4u : 8u); }

__global__ void k_probe_descs(LeafDesc* d, uint32_t n_leaves, uint32_t m) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_leaves) d[i] = LeafDesc{i * m, m, kNoCode, 0};
}

// Rate of a configuration: the persistent kernel itself (same code, registers,
// occupancy and work sharing as in a build) on two synthetic leaves of m keys
// per warp, at the passes per work item a build uses.  The search starts 4096
// seeds below the seed cap, so each leaf ends at its solution or at the cap
// (a runtime bound in the kernel instead would change its code: measured 7 %
// slower at 4 seeds x 8 warps x unroll 4).  Key-seed evaluations per second
// of the best of `runs` timed launches.
shk_status probe_leaf_cfg(Ctx& c, const LeafCfg& cfg, uint32_t m, double* evals_per_s, int runs) {
  const LeafKernels* k = find_kernels(cfg);
  if (!k) return fail(SHK_EINVAL, "unsupported leaf kernel configuration");
  if (m < 2 || m > kMaxLeaf) return fail(SHK_EINVAL, "leaf size must be in [2, 64]");
  uint32_t blocks;
  SHK_TRY(persistent_blocks(c, k, &blocks));
  const uint32_t L = 2 * blocks * cfg.warps, nwords = (L + 31) / 32;
  const uint32_t passes = default_passes(m);
  uint64_t* keys;
  LeafDesc* descs;
  unsigned long long *best, *cnt;
  uint32_t *state, *err;
  SHK_TRY(c.arena.alloc(&keys, (size_t)L * m));
  SHK_TRY(c.arena.alloc(&descs, L));
  SHK_TRY(c.arena.alloc(&best, L));
  SHK_TRY(c.arena.alloc(&cnt, 1));
  SHK_TRY(c.arena.alloc(&state, (size_t)L + nwords + 1));
  SHK_TRY(c.arena.alloc(&err, 1));
  k_probe_keys<<<(unsigned)(((uint64_t)L * m + 255) / 256), 256, 0, c.stream>>>(keys, (uint64_t)L * m,
                                                                              (uint64_t)m << 40);
  k_probe_descs<<<(L + 255) / 256, 256, 0, c.stream>>>(descs, L, m);
  c.launches += 2;
  cudaEvent_t e0, e1;
  SHK_CUDA(cudaEventCreate(&e0));
  SHK_CUDA(cudaEventCreate(&e1));
  double top = 0;
  for (int run = -1; run < runs; run++) {  // run -1: warm-up
    SHK_CUDA(cudaMemsetAsync(best, 0xFF, (size_t)L * 8, c.stream));
    SHK_CUDA(cudaMemsetAsync(state, 0, ((size_t)L + nwords + 1) * 4, c.stream));
    SHK_CUDA(cudaMemsetAsync(cnt, 0, 8, c.stream));
    SHK_CUDA(cudaEventRecord(e0, c.stream));
    k->persistent<<<blocks, cfg.warps * 32, 0, c.stream>>>(descs, L, keys, kSeedCap - 4096, passes,
                                                          best, state, state + L, state + L + nwords,
                                                          cnt, err, LeafCtl{});
    SHK_CUDA(cudaEventRecord(e1, c.stream));
    c.launches++;
    unsigned long long h = 0;
    SHK_CUDA(cudaMemcpyAsync(&h, cnt, 8, cudaMemcpyDeviceToHost, c.stream));
    SHK_CUDA(cudaStreamSynchronize(c.stream));
    float ms = 0;
    SHK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    const double r = ms > 0 ? (double)h * m / (ms * 1e-3) : 0;
    if (run >= 0 && r > top) top = r;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *evals_per_s = top;
  return SHK_OK;
}

shk_status tuned_leaf_cfg(Ctx& c, uint32_t m, LeafCfg* out) {
  const uint32_t bin = m <= 16 ? 0 : (m <= 32 ? 1 : (m <= 48 ? 2 : 3));
  const uint32_t rep = (bin + 1) * 16;
  if (c.device < 0 || c.device >= 64) return fail(SHK_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  TuneSlot& slot = g_tune[c.device][bin];
  if (!slot.done) {
    // Every configuration at its best of 3 probe launches.  The probe's short
    // searches overrate 16-warp blocks by 2-3 % against real builds, where
    // 8-warp blocks were fastest in every sweep (10^6 keys, n = 48: 4/8/4
    // 268.0 ms, 4/4/2 271.5, 4/16/2 272.0, though 4/16/2 probed 2.3 % above
    // 4/8/4): the fastest 8-warp configuration within 3 % of the best rate is
    // taken; failing that, among those within 1 % the one with the fewest
    // warps per block (smaller blocks leave less SM time idle while the last
    // leaves finish).
    double rate[kNumLeafCfg], top = 0;
    for (int i = 0; i < kNumLeafCfg; i++) {
      SHK_TRY(probe_leaf_cfg(c, kLeafTable[i].cfg, rep, &rate[i], 3));
      top = std::max(top, rate[i]);
    }
    int pick = -1;
    for (int i = 0; i < kNumLeafCfg; i++)
      if (kLeafTable[i].cfg.warps == 8 && rate[i] >= 0.97 * top && (pick < 0 || rate[i] > rate[pick])) pick = i;
    const bool have8 = pick >= 0;
    for (int i = 0; !have8 && i < kNumLeafCfg; i++) {
      if (rate[i] < 0.99 * top) continue;
      if (pick < 0 || kLeafTable[i].cfg.warps < kLeafTable[pick].cfg.warps ||
          (kLeafTable[i].cfg.warps == kLeafTable[pick].cfg.warps && rate[i] > rate[pick]))
        pick = i;
    }
    LeafCfg best_cfg = kLeafTable[pick].cfg;
    const double best = rate[pick];
    best_cfg.passes = default_passes(rep);
    slot.cfg = best_cfg;
    slot.evals_per_s = best;
    slot.done = true;
  }
  *out = slot.cfg;
  out->passes = default_passes(m);
  return SHK_OK;
}

// ---------------------------------------------------------------------------
// a6: orientation.  Tree edges are forced (peel cells of degree one); on each
// remaining cycle the smallest-index key takes its cell h0 and the cycle is
// walked from there.  This is the lexicographically smallest f.  One thread per
// leaf; also stores the leaf's seed into its code slot.
// ---------------------------------------------------------------------------
__global__ void k_orient(const LeafDesc* __restrict__ leaves, uint32_t n_leaves,
                         const uint64_t* __restrict__ x, const unsigned long long* __restrict__ best,
                         uint64_t* codes, uint8_t* f_key, uint64_t* f_mask, uint32_t* err,
                         uint32_t leaf_mode) {
  const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_leaves) return;
  const LeafDesc d = leaves[l];
  const uint64_t s = best[l];
  const uint32_t m = d.m;
  if (m == 1 && s != ~0ull) {
    if (f_mask != nullptr) f_mask[l] = 0;
    return;
  }
  if (m < 2 || m > kMaxLeaf || s == ~0ull) {
    atomicOr(err, kErrOrient);
    return;
  }
  if (codes != nullptr && d.code_idx != kNoCode) codes[d.code_idx] = s;
  uint8_t e0[kMaxLeaf], e1[kMaxLeaf], stack[kMaxLeaf];
  uint64_t inc[kMaxLeaf];
  for (uint32_t v = 0; v < m; v++) inc[v] = 0;
  for (uint32_t e = 0; e < m; e++) {
    uint32_t h0, h1;
    value_cells(leaf_mode, x[d.key_off + e], s, m, &h0, &h1);
    e0[e] = (uint8_t)h0;
    e1[e] = (uint8_t)h1;
    inc[h0] |= 1ull << e;
    inc[h1] |= 1ull << e;
  }
  uint64_t live = m == 64 ? ~0ull : ((1ull << m) - 1);
  uint64_t fb = 0;
  int sp = 0;
  for (uint32_t v = 0; v < m; v++)
    if (__popcll(inc[v]) == 1) stack[sp++] = (uint8_t)v;
  bool bad = false;
  while (sp > 0) {
    const uint32_t v = stack[--sp];
    const uint64_t em = inc[v] & live;
    if (em == 0) {  // its last edge was taken from the other side: a tree
      bad = true;
      break;
    }
    if (__popcll(em) != 1) continue;
    const uint32_t e = __ffsll((long long)em) - 1;
    if (e1[e] == v) fb |= 1ull << e;
    live &= ~(1ull << e);
    const uint32_t u = e0[e] == v ? e1[e] : e0[e];
    if (__popcll(inc[u] & live) == 1) stack[sp++] = (uint8_t)u;
  }
  while (!bad && live) {
    const uint32_t e = __ffsll((long long)live) - 1;
    const uint32_t start = e0[e];
    live &= ~(1ull << e);  // e takes h0 (f = 0)
    uint32_t v = e1[e];
    for (uint32_t guard = 0; v != start; guard++) {
      const uint64_t em = inc[v] & live;
      if (em == 0 || guard > m) {
        bad = true;
        break;
      }
      const uint32_t e2 = __ffsll((long long)em) - 1;
      if (e1[e2] == v) fb |= 1ull << e2;
      live &= ~(1ull << e2);
      v = e0[e2] == v ? e1[e2] : e0[e2];
    }
  }
  if (bad) {
    atomicOr(err, kErrOrient);
    return;
  }
  if (f_key != nullptr)
    for (uint32_t e = 0; e < m; e++) f_key[d.key_off + e] = (uint8_t)((fb >> e) & 1);
  if (f_mask != nullptr) f_mask[l] = fb;
}

shk_status launch_orient(Ctx& c, const LeafDesc* leaves, uint32_t n_leaves, const uint64_t* x,
                         const unsigned long long* best, uint64_t* codes, uint8_t* f_key,
                         uint64_t* f_mask, uint32_t* err, uint32_t leaf_mode) {
  if (n_leaves == 0) return SHK_OK;
  k_orient<<<(n_leaves + 127) / 128, 128, 0, c.stream>>>(leaves, n_leaves, x, best, codes, f_key,
                                                         f_mask, err, leaf_mode);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

// Sums over leaves, counted from the results: sums[0] = sum (value + 1),
// sums[1] = sum (value + 1) * m, sums[2] = the hash evaluations of a
// sequential search, sums[3] = its seeds tested (plain: value + 1; rotation
// fitting: floor(value / m) + 1), and (rotation fitting) *cells = its (seed, missed cell)
// steps of the rotation filter; cbar[m * 65 + a] = E[min(cells missed by a
// set A of a keys, K)] for m > 32 (see rf_cell_table).
__global__ void k_leaf_sums(const LeafDesc* leaves, uint32_t n_leaves,
                            const unsigned long long* best, unsigned long long* sums,
                            uint32_t leaf_mode, const uint64_t* x, const double* cbar,
                            double* cells) {
  unsigned long long a = 0, b = 0, h = 0, tested = 0;
  double cl = 0;
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < n_leaves;
       l += gridDim.x * blockDim.x) {
    const LeafDesc d = leaves[l];
    const unsigned long long s = best[l] + 1;
    a += s;
    b += s * d.m;
    if (leaf_mode == 0 || d.m < 2) {
      h += s * d.m;
      tested += s;
    } else {
      const unsigned long long T = best[l] / d.m + 1;
      tested += T;
      if (d.m > 32) {
        uint32_t na = 0;
        for (uint32_t i = 0; i < d.m; i++) na += (mix64(x[d.key_off + i] ^ kRfSalt) >> 63) == 0;
        const unsigned long long G = (T + 7) / 8;
        h += (d.m - na) * T + na * G;
        cl += 8.0 * (double)G * cbar[d.m * 65 + na];
      } else {
        h += T * d.m;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(kFull, a, o);
    b += __shfl_down_sync(kFull, b, o);
    h += __shfl_down_sync(kFull, h, o);
    tested += __shfl_down_sync(kFull, tested, o);
    cl += __shfl_down_sync(kFull, cl, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[0], a);
    atomicAdd(&sums[1], b);
    atomicAdd(&sums[2], h);
    atomicAdd(&sums[3], tested);
    if (cells) atomicAdd(cells, cl);
  }
}

// E[min(Z, K)] where Z = cells of an m-cell leaf missed by a keys that each
// take two distinct uniformly random cells (K = 24 for m = 64, 20 otherwise:
// the missed cells the rotation filter intersects without branches), for
// m = 33..64 and a = 0..m; exact, by the distribution of covered cells.
static void rf_cell_table(double* t) {
  for (int i = 0; i < 65 * 65; i++) t[i] = 0;
  for (int m = 33; m <= 64; m++) {
    const int K = m == 64 ? 24 : 20;
    double p[65] = {0}, q[65];
    p[0] = 1;
    const double pairs = (double)m * (m - 1);
    for (int a = 0; a <= m; a++) {
      double e = 0;
      for (int k = 0; k <= m; k++) e += p[k] * (double)(m - k < K ? m - k : K);
      t[m * 65 + a] = e;
      for (int k = 0; k <= m; k++) q[k] = 0;
      for (int k = 0; k <= m; k++) {
        if (p[k] == 0) continue;
        const double two = (double)(m - k) * (m - k - 1) / pairs;
        const double one = 2.0 * k * (m - k) / pairs;
        const double zero = (double)k * (k - 1) / pairs;
        q[k] += p[k] * zero;
        if (k + 1 <= m) q[k + 1] += p[k] * one;
        if (k + 2 <= m) q[k + 2] += p[k] * two;
      }
      for (int k = 0; k <= m; k++) p[k] = q[k];
    }
  }
}

shk_status launch_leaf_sums(Ctx& c, const LeafDesc* leaves, uint32_t n_leaves,
                            const unsigned long long* best, unsigned long long* sums,
                            uint32_t leaf_mode, const uint64_t* x, double* cells) {
  if (n_leaves == 0) return SHK_OK;
  double* cbar = nullptr;
  if (leaf_mode) {
    double host[65 * 65];
    rf_cell_table(host);
    SHK_TRY(c.arena.alloc(&cbar, 65 * 65));
    SHK_CUDA(cudaMemcpyAsync(cbar, host, sizeof host, cudaMemcpyHostToDevice, c.stream));
    // the host table must outlive the copy
    SHK_CUDA(cudaStreamSynchronize(c.stream));
  }
  uint32_t blocks = (n_leaves + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  k_leaf_sums<<<blocks, 256, 0, c.stream>>>(leaves, n_leaves, best, sums, leaf_mode, x, cbar,
                                            leaf_mode ? cells : nullptr);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

}  // namespace shk
