// ribbon.cu -- 1-bit retrieval of the orientation bits of all keys (paper
// Sec. 2 Retrieval: the value is the parity of a hashed row with a segment of
// a solution table; the table solves a nearly diagonal linear system).  A
// standard ribbon of width 64, sharded by runs of buckets; one CTA per shard.
//
// Elimination: each key's row (start, 64-bit coefficient with bit 0 set) is
// reduced by the row stored at its lowest set column until it reaches a free
// column (a new pivot) or vanishes.  The stored solution is the one that is 0
// on every non-pivot column; it does not depend on the order of the keys.
#include "kernels.cuh"

namespace shk {

constexpr int kRibbonThreads = 1024;
constexpr uint32_t kRegions = kRibbonThreads / 32;  // one elimination region per warp

__device__ __forceinline__ uint32_t ctz64(uint64_t v) {  // v != 0
  const uint32_t lo = (uint32_t)v;
  return lo ? (uint32_t)__ffs((int)lo) - 1 : 31u + (uint32_t)__ffs((int)(v >> 32));
}

// Reduce one row against the table until it lands on a free slot (returns 1),
// vanishes (returns 1 if consistent, 0 if not) or reaches slot `limit`
// (returns 2; *st, *cf, *bv then hold the partly reduced row).
__device__ __forceinline__ int eliminate(uint64_t* rows, uint8_t* rhs, uint32_t* st, uint64_t* cf,
                                         uint8_t* bv, uint32_t limit) {
  uint32_t s = *st;
  uint64_t c = *cf;
  uint8_t b = *bv;
  for (;;) {
    if (s >= limit) {
      *st = s;
      *cf = c;
      *bv = b;
      return 2;
    }
    const uint64_t row = rows[s];
    if (row == 0) {
      rows[s] = c;
      rhs[s] = b;
      return 1;
    }
    c ^= row;
    b ^= rhs[s];
    if (c == 0) return b ? 0 : 1;
    const uint32_t tz = ctz64(c);
    c >>= tz;
    s += tz;
  }
}

__global__ void k_shard_slots(const uint32_t* K, uint64_t B, uint32_t S, uint32_t eps_num,
                              uint64_t num_shards, uint64_t* slots) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= num_shards) return;
  const uint64_t b0 = s * S, b1 = b0 + S < B ? b0 + S : B;
  slots[s] = shard_slots(K[b1] - K[b0], eps_num);
}

shk_status launch_shard_slots(Ctx& c, const uint32_t* K, uint64_t B, uint32_t S, uint32_t eps_num,
                              uint64_t num_shards, uint64_t* slots) {
  if (num_shards == 0) return SHK_OK;
  k_shard_slots<<<(unsigned)((num_shards + 255) / 256), 256, 0, c.stream>>>(K, B, S, eps_num,
                                                                            num_shards, slots);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

__global__ void k_max_shard_keys(const uint32_t* K, uint64_t B, uint32_t S, uint64_t num_shards,
                                 uint32_t* out_max) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= num_shards) return;
  const uint64_t b0 = s * S, b1 = b0 + S < B ? b0 + S : B;
  atomicMax(out_max, K[b1] - K[b0]);
}

shk_status launch_max_shard_keys(Ctx& c, const uint32_t* K, uint64_t B, uint32_t S,
                                 uint64_t num_shards, uint32_t* out_max) {
  if (num_shards == 0) return SHK_OK;
  k_max_shard_keys<<<(unsigned)((num_shards + 255) / 256), 256, 0, c.stream>>>(K, B, S, num_shards,
                                                                               out_max);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

// Shared memory of one shard with row precomputation: rows[m] u64 |
// coefficients[keys] u64 | starts[keys] u32 | rhs[m] u8 | bits[keys] u8.
__host__ __device__ inline size_t ribbon_smem(uint64_t m, uint64_t keys, bool pre) {
  return pre ? (size_t)m * 9 + (size_t)keys * 13 + 16 : (size_t)m * 9 + 16;
}

template <bool PRE>
__global__ void __launch_bounds__(kRibbonThreads)
    k_ribbon(const uint64_t* __restrict__ lo, const uint64_t* __restrict__ hi,
             const uint8_t* __restrict__ f, const uint32_t* __restrict__ K, uint64_t B, uint32_t S,
             uint32_t eps_num, const uint64_t* __restrict__ shard_off, uint64_t* sol_words,
             uint8_t* seeds, uint32_t* err) {
  extern __shared__ uint64_t rows[];
  const uint64_t sh = blockIdx.x;
  const uint64_t b0 = sh * S, b1 = b0 + S < B ? b0 + S : B;
  const uint32_t k0 = K[b0], keys = K[b1] - K[b0];
  const uint64_t m = shard_slots(keys, eps_num);
  if (m == 0) {
    if (threadIdx.x == 0) seeds[sh] = 0;
    return;
  }
  uint64_t* pcoef = rows + m;
  uint32_t* pstart = (uint32_t*)(pcoef + (PRE ? keys : 0));
  uint8_t* rhs = PRE ? (uint8_t*)(pstart + keys) : (uint8_t*)(rows + m);
  uint8_t* pbit = rhs + m;
  __shared__ int ok_s;
  __shared__ uint32_t seed_s;
  for (uint32_t r = 0; r < kRibbonSeeds; r++) {
    for (uint64_t i = threadIdx.x; i < m; i += kRibbonThreads) {
      rows[i] = 0;
      rhs[i] = 0;
    }
    if (PRE) {
      for (uint32_t i = threadIdx.x; i < keys; i += kRibbonThreads) {
        uint64_t st, cf;
        ribbon_row(lo[k0 + i], hi[k0 + i], r, m, &st, &cf);
        pcoef[i] = cf;
        pstart[i] = (uint32_t)st;
        pbit[i] = f[k0 + i];
      }
    }
    if (threadIdx.x == 0) {
      ok_s = 1;
      seed_s = r;
    }
    __syncthreads();
    if (PRE) {
      // Phase 1: lane 0 of every warp eliminates, in parallel with the other
      // warps, the rows that start in its own slot range; a row that would
      // step past its range is parked: bit 1 of its pbit is set, its start and
      // coefficient stay as they were (other warps read them), and phase 2
      // reduces it again from the start.  No slot and no row is written by
      // two warps.
      if ((threadIdx.x & 31) == 0) {
        const uint32_t reg = threadIdx.x >> 5;
        const uint32_t w = (uint32_t)((m + kRegions - 1) / kRegions);
        const uint32_t r0 = reg * w, r1 = r0 + w < m ? r0 + w : (uint32_t)m;
        int ok = 1;
        for (uint32_t i = 0; i < keys && ok; i++) {
          uint32_t st = pstart[i];
          if (st < r0 || st >= r1) continue;
          uint64_t cf = pcoef[i];
          uint8_t bv = pbit[i];
          const int res = eliminate(rows, rhs, &st, &cf, &bv, r1);
          if (res == 0) ok = 0;
          if (res == 2) pbit[i] |= 2;
        }
        if (!ok) ok_s = 0;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0 && ok_s) {
      // Phase 2 (or the whole elimination without row precomputation): one
      // thread over the whole table.
      int ok = 1;
      for (uint32_t i = 0; i < keys && ok; i++) {
        uint32_t st;
        uint64_t cf;
        uint8_t bv;
        if (PRE) {
          if (!(pbit[i] & 2)) continue;
          st = pstart[i];
          cf = pcoef[i];
          bv = pbit[i] & 1;
        } else {
          uint64_t st64;
          ribbon_row(lo[k0 + i], hi[k0 + i], r, m, &st64, &cf);
          st = (uint32_t)st64;
          bv = f[k0 + i];
        }
        if (eliminate(rows, rhs, &st, &cf, &bv, 0xFFFFFFFFu) == 0) ok = 0;
      }
      ok_s = ok;
    }
    __syncthreads();
    if (ok_s) break;
    __syncthreads();
  }
  if (!ok_s) {
    if (threadIdx.x == 0) atomicOr(err, kErrRibbon);
    return;
  }
  if (threadIdx.x == 0) {
    seeds[sh] = (uint8_t)seed_s;
    // back substitution from the top; window bit j-1 = solution at i + j
    uint64_t win = 0;
    for (uint64_t i = m; i-- > 0;) {
      const uint64_t row = rows[i];
      uint8_t v = 0;
      if (row) v = (uint8_t)((rhs[i] ^ __popcll((row >> 1) & win)) & 1);
      rhs[i] = v;
      win = (win << 1) | v;
    }
  }
  __syncthreads();
  // pack the solution bits and OR them into the global vector
  const uint64_t base = shard_off[sh];
  for (uint64_t w = threadIdx.x; w * 64 < m; w += kRibbonThreads) {
    uint64_t word = 0;
    const uint64_t lim = m - w * 64 < 64 ? m - w * 64 : 64;
    for (uint64_t j = 0; j < lim; j++) word |= (uint64_t)rhs[w * 64 + j] << j;
    if (word == 0) continue;
    const uint64_t p = base + w * 64;
    const uint32_t s = (uint32_t)(p & 63);
    atomicOr((unsigned long long*)&sol_words[p >> 6], (unsigned long long)(word << s));
    // the next word only when bits land there (it then lies inside the vector)
    if (s && (word >> (64 - s)))
      atomicOr((unsigned long long*)&sol_words[(p >> 6) + 1], (unsigned long long)(word >> (64 - s)));
  }
}

shk_status launch_ribbon(Ctx& c, const uint64_t* lo, const uint64_t* hi, const uint8_t* f,
                         const uint32_t* K, uint64_t B, uint32_t S, uint32_t eps_num,
                         uint64_t num_shards, const uint64_t* shard_off, uint32_t max_shard_slots,
                         uint64_t* sol_words, uint8_t* seeds, uint32_t* err) {
  if (num_shards == 0) return SHK_OK;
  const size_t limit = 227 * 1024;
  // max_shard_slots belongs to the largest shard, so it bounds its keys too
  const size_t smem_pre = ribbon_smem(max_shard_slots, max_shard_slots, true);
  const size_t smem = ribbon_smem(max_shard_slots, 0, false);
  if (smem_pre <= limit) {
    SHK_CUDA(cudaFuncSetAttribute(k_ribbon<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_pre));
    k_ribbon<true><<<(unsigned)num_shards, kRibbonThreads, smem_pre, c.stream>>>(
        lo, hi, f, K, B, S, eps_num, shard_off, sol_words, seeds, err);
  } else {
    if (smem > limit) return fail(SHK_EINVAL, "retrieval shard too large for shared memory");
    SHK_CUDA(cudaFuncSetAttribute(k_ribbon<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_ribbon<false><<<(unsigned)num_shards, kRibbonThreads, smem, c.stream>>>(
        lo, hi, f, K, B, S, eps_num, shard_off, sol_words, seeds, err);
  }
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

}  // namespace shk
