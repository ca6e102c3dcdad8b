// kernels.cuh -- launch interfaces of the construction kernels.
#pragma once

#include "shk_internal.cuh"

namespace shk {

// Per-call context: stream, stream-ordered allocations, device facts and a
// count of the kernels this call launched.
struct Ctx {
  cudaStream_t stream;
  Arena arena;
  int num_sms = 0;
  int device = 0;
  uint64_t launches = 0;
  explicit Ctx(cudaStream_t s) : stream(s), arena(s) {}
};

shk_status init_ctx(Ctx& c);

// shk_build with an abort flag (host-mapped memory, may be NULL) that stops
// the leaf search with SHK_ECANCELLED once it is non-zero (the server's
// cancellation).
shk_status build_controlled(const shk_keys* keys, const shk_build_opts* o, cudaStream_t st,
                            shk_mphf** out, const volatile uint32_t* abort);

template <class Tin, class T>
shk_status exclusive_scan(Ctx& c, const Tin* in, uint64_t n, T* out);

// a1
shk_status launch_fingerprint(Ctx& c, int kind, const void* data, const uint64_t* offs,
                              uint32_t n_keys, uint64_t B, ulonglong2* fp, uint32_t* counts);
shk_status launch_fingerprint_only(Ctx& c, int kind, const void* data, const uint64_t* offs,
                                   uint64_t n_keys, uint64_t* lo, uint64_t* hi);
// a2
shk_status launch_scatter(Ctx& c, const ulonglong2* fp, uint32_t n_keys, uint64_t B,
                          const uint32_t* K, ulonglong2* sfp);

// tree bookkeeping: per bucket the number of searched leaves (m >= 2), of
// codes (split nodes + searched leaves) and of split nodes; plus the largest
// bucket (atomicMax into *max_bucket).
shk_status launch_tree_count(Ctx& c, const uint32_t* K, uint64_t B, uint32_t n,
                             uint32_t* n_leaves, uint32_t* n_codes, uint32_t* n_splits,
                             uint32_t* max_bucket);
// a3
shk_status launch_split(Ctx& c, const ulonglong2* sfp, const uint32_t* K, uint64_t B, uint32_t n,
                        uint32_t max_bucket, const uint32_t* code_base, const uint32_t* leaf_base,
                        uint64_t* codes, uint8_t* code_k, LeafDesc* leaves, uint64_t* llo,
                        uint64_t* lhi, uint32_t* err);

// a4 + a5: leaf seed search.  best[L] must be preset to ~0.
// Kernel configuration: seeds per lane, warps per block, key-loop unroll and
// passes (of 32 x seeds_per_lane seeds) per work item.  It changes speed only.
struct LeafCfg {
  uint32_t seeds_per_lane, warps, unroll, passes;
};
// Control of a leaf search (every pointer may be NULL): t_range[0] / [1]
// receive the device time the first block started / the last warp ended
// (atomicMin / atomicMax; preset to ~0 / 0); the search stops, setting
// kErrTimeout, once the device time passes *deadline (0 = none), or, setting
// kErrCancelled, once *abort is non-zero (host-mapped memory).  Both are
// checked before every work item.
struct LeafCtl {
  unsigned long long* t_range;
  const unsigned long long* deadline;
  const volatile uint32_t* abort;
};
struct LeafSearchArgs {
  const LeafDesc* leaves;
  uint32_t n_leaves;
  const uint64_t* x;  // leaf inputs, indexed by LeafDesc::key_off
  uint64_t seed_start;
  unsigned long long* best;
  uint32_t* err;
  unsigned long long* executed;  // seeds evaluated (counter)
  LeafCfg cfg;
  LeafCtl ctl;
};

// Warp-uniform: true when the search must stop (sets the error flag).
__device__ __forceinline__ bool leaf_should_stop(const LeafCtl& ctl, uint32_t* err) {
  int stop = 0;
  if ((threadIdx.x & 31) == 0) {
    if (ctl.abort && *ctl.abort) {
      atomicOr(err, kErrCancelled);
      stop = 1;
    } else if (ctl.deadline && *ctl.deadline && global_ns() > *ctl.deadline) {
      atomicOr(err, kErrTimeout);
      stop = 1;
    }
  }
  return __shfl_sync(0xFFFFFFFFu, stop, 0) != 0;
}

__device__ __forceinline__ void leaf_mark_start(const LeafCtl& ctl) {
  if (ctl.t_range && threadIdx.x == 0) atomicMin(&ctl.t_range[0], (unsigned long long)global_ns());
}

__device__ __forceinline__ void leaf_mark_end(const LeafCtl& ctl) {
  if (ctl.t_range && (threadIdx.x & 31) == 0) atomicMax(&ctl.t_range[1], (unsigned long long)global_ns());
}
shk_status launch_leaf_persistent(Ctx& c, const LeafSearchArgs& a);
// As launch_leaf_persistent, with caller-owned state of
// (n_leaves + (n_leaves + 31) / 32 + 1) u32 words (cleared by the launch).
shk_status launch_leaf_persistent_state(Ctx& c, const LeafSearchArgs& a, uint32_t* state);
shk_status launch_leaf_range(Ctx& c, const LeafSearchArgs& a, uint32_t l0, uint32_t l1);
// autotuner: the fastest configuration for leaves of m keys on this device
shk_status tuned_leaf_cfg(Ctx& c, uint32_t m, LeafCfg* out);
shk_status probe_leaf_cfg(Ctx& c, const LeafCfg& cfg, uint32_t m, double* evals_per_s, int runs = 1);
bool leaf_cfg_valid(const LeafCfg& c);
int leaf_cfg_count();
LeafCfg leaf_cfg_at(int i);
// a6: orientation; writes seeds into codes[code_idx], f per key (leaf order)
// and optionally f as a mask per leaf.
shk_status launch_orient(Ctx& c, const LeafDesc* leaves, uint32_t n_leaves, const uint64_t* x,
                         const unsigned long long* best, uint64_t* codes, uint8_t* f_key,
                         uint64_t* f_mask, uint32_t* err, uint32_t leaf_mode = 0);
// rotation fitting (leaf mode 1): best[] receives v = s*m + r
shk_status launch_leaf_rf_persistent(Ctx& c, const LeafSearchArgs& a);
shk_status launch_leaf_rf_range(Ctx& c, const LeafSearchArgs& a, uint32_t l0, uint32_t l1);
// sums[0..3] += sum (value + 1), sum (value + 1) m, hash evaluations and
// seeds tested by a sequential search; *cells += rotation-filter steps
// (leaf mode 1)
shk_status launch_leaf_sums(Ctx& c, const LeafDesc* leaves, uint32_t n_leaves,
                            const unsigned long long* best, unsigned long long* sums,
                            uint32_t leaf_mode, const uint64_t* x, double* cells);

// a7
shk_status launch_rice_bits(Ctx& c, const uint64_t* codes, const uint8_t* code_k,
                            const uint32_t* code_base, uint64_t B, uint64_t* bucket_bits);
shk_status launch_rice_write(Ctx& c, const uint64_t* codes, const uint8_t* code_k,
                             const uint32_t* code_base, uint64_t B, const uint64_t* O,
                             uint64_t* words);
shk_status launch_ef_write_u32(Ctx& c, const uint32_t* v, uint64_t count, uint32_t l,
                               uint64_t* low, uint64_t* high);
shk_status launch_ef_write_u64(Ctx& c, const uint64_t* v, uint64_t count, uint32_t l,
                               uint64_t* low, uint64_t* high);
shk_status launch_ef_decode(Ctx& c, const uint64_t* low, const uint64_t* high, uint64_t hbits,
                            uint32_t l, uint64_t count, uint64_t* out);
// Raise the dynamic shared memory limit of a kernel on the current device to
// at least `bytes`.  The limit only ever grows (under a lock), so builds
// running concurrently on several host threads never lower the limit that
// another thread's launch relies on.
shk_status raise_smem_limit(const void* kernel, size_t bytes);

// Resident blocks per SM of a kernel for a launch shape (cached per device).
shk_status blocks_per_sm(const void* kernel, int threads, size_t smem, int* out);

shk_status launch_validate_index(Ctx& c, const uint32_t* K, const uint64_t* O, uint64_t B,
                                 uint64_t N, uint64_t rice_bits, uint32_t* bad);
// a8
shk_status launch_shard_slots(Ctx& c, const uint32_t* K, uint64_t B, uint32_t S, uint32_t eps_num,
                              uint32_t w, uint64_t num_shards, uint64_t* slots);
// w = 64 or 128; total_slots = all shards' slots, n_keys = all keys (the
// 128-bit solver's global scratch)
shk_status launch_ribbon(Ctx& c, const uint64_t* lo, const uint64_t* hi, const uint8_t* f,
                         const uint32_t* K, uint64_t B, uint32_t S, uint32_t eps_num, uint32_t w,
                         uint64_t num_shards, const uint64_t* shard_off, uint32_t max_shard_slots,
                         uint64_t total_slots, uint64_t n_keys, uint64_t* sol_words, uint8_t* seeds,
                         uint32_t* err);
// device scratch of the 128-bit solve (its persistent warps' sorted rows and
// bands, per-shard state) for these shards
shk_status ribbon128_scratch_bytes(uint64_t num_shards, uint64_t max_shard_slots, uint64_t* bytes);
shk_status launch_max_shard_keys(Ctx& c, const uint32_t* K, uint64_t B, uint32_t S,
                                 uint64_t num_shards, uint32_t* out_max);
// query
shk_status launch_query(Ctx& c, const shk_mphf* m, const uint64_t* lo, const uint64_t* hi,
                        uint64_t n, uint64_t* ranks);
// query index: records of every bucket's codes (qbase: each bucket's first record)
shk_status launch_qindex_build(Ctx& c, const shk_mphf* m, const uint32_t* qbase, QNode* nodes);

}  // namespace shk
