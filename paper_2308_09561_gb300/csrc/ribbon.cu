// ribbon.cu -- 1-bit retrieval of the orientation bits of all keys (paper
// Sec. 2 Retrieval: the value is the parity of a hashed row with a segment of
// a solution table; the table solves a nearly diagonal linear system).  A
// standard ribbon of width 64 (leaf size n <= 24) or 128 (n > 24; Sec. 8.2's
// 128-bit words), sharded by runs of buckets; one CTA per shard.
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

// Eliminates the rows plist[t0 .. t1) one after the other; a row that
// reaches slot `limit` has its state written back and is passed to park(i).
// Returns 0 if a row vanished with right-hand side 1.
template <class Park>
__device__ __forceinline__ int eliminate_list(uint64_t* rows, uint8_t* rhs, uint64_t* pcoef,
                                              uint32_t* pstart, uint8_t* pbit,
                                              const uint16_t* plist, uint32_t t0, uint32_t t1,
                                              uint32_t limit, Park park) {
  for (uint32_t t = t0; t < t1; t++) {
    const uint32_t i = plist[t];
    uint32_t st = pstart[i];
    uint64_t cf = pcoef[i];
    uint8_t bv = pbit[i];
    const int res = eliminate(rows, rhs, &st, &cf, &bv, limit);
    if (res == 0) return 0;
    if (res == 2) {
      pstart[i] = st;
      pcoef[i] = cf;
      pbit[i] = bv;
      park(i);
    }
  }
  return 1;
}

__global__ void k_shard_slots(const uint32_t* K, uint64_t B, uint32_t S, uint32_t eps_num,
                              uint32_t w, uint64_t num_shards, uint64_t* slots) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= num_shards) return;
  const uint64_t b0 = s * S, b1 = b0 + S < B ? b0 + S : B;
  slots[s] = shard_slots(K[b1] - K[b0], eps_num, w);
}

shk_status launch_shard_slots(Ctx& c, const uint32_t* K, uint64_t B, uint32_t S, uint32_t eps_num,
                              uint32_t w, uint64_t num_shards, uint64_t* slots) {
  if (num_shards == 0) return SHK_OK;
  k_shard_slots<<<(unsigned)((num_shards + 255) / 256), 256, 0, c.stream>>>(K, B, S, eps_num, w,
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
// coefficients[keys] u64 | starts[keys] u32 | region lists[keys] u16 |
// rhs[m] u8 | bits[keys] u8.
__host__ __device__ inline size_t ribbon_smem(uint64_t m, uint64_t keys, bool pre) {
  return pre ? (size_t)m * 9 + (size_t)keys * 15 + 32 : (size_t)m * 9 + 16;
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
  const uint64_t m = shard_slots(keys, eps_num, 64);
  if (m == 0) {
    if (threadIdx.x == 0) seeds[sh] = 0;
    return;
  }
  uint64_t* pcoef = rows + m;
  uint32_t* pstart = (uint32_t*)(pcoef + (PRE ? keys : 0));
  uint16_t* plist = (uint16_t*)(pstart + (PRE ? keys : 0));
  uint8_t* rhs = PRE ? (uint8_t*)(plist + keys) : (uint8_t*)(rows + m);
  uint8_t* pbit = rhs + m;
  __shared__ int ok_s;
  __shared__ uint32_t seed_s;
  __shared__ uint32_t rbase[kRegions + 1], rfill[kRegions], rpark[kRegions];
  const uint32_t w = (uint32_t)((m + kRegions - 1) / kRegions);  // region width in slots
  for (uint32_t r = 0; r < kRibbonSeeds; r++) {
    for (uint64_t i = threadIdx.x; i < m; i += kRibbonThreads) {
      rows[i] = 0;
      rhs[i] = 0;
    }
    if (threadIdx.x < kRegions) rfill[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
      ok_s = 1;
      seed_s = r;
    }
    __syncthreads();
    if (PRE) {
      // rows of this seed, listed by the region of their start slot
      for (uint32_t i = threadIdx.x; i < keys; i += kRibbonThreads) {
        uint64_t st, cf, c1;
        ribbon_row(lo[k0 + i], hi[k0 + i], r, m, 64, &st, &cf, &c1);
        pcoef[i] = cf;
        pstart[i] = (uint32_t)st;
        pbit[i] = f[k0 + i];
        atomicAdd(&rfill[(uint32_t)st / w], 1u);
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        // exclusive scan of the kRegions (= 32) counts by one warp
        const uint32_t lane = threadIdx.x, c = rfill[lane];
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
          if (lane >= (uint32_t)o) x += y;
        }
        rbase[lane] = x - c;
        if (lane == 31) rbase[kRegions] = x;
        rfill[lane] = x - c;
      }
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < keys; i += kRibbonThreads)
        plist[atomicAdd(&rfill[pstart[i] / w], 1u)] = (uint16_t)i;
      __syncthreads();
      // Phase 1: lane 0 of warp g eliminates the rows that start in region g,
      // slots [g w, (g + 1) w), in parallel with the other warps.  A row that
      // would step past the region is parked: its partly reduced state is
      // written back (only this lane owns the row) and its index is kept at
      // the front of the region's list.
      if ((threadIdx.x & 31) == 0) {
        const uint32_t g = threadIdx.x >> 5;
        const uint32_t r1 = (g + 1) * w < m ? (g + 1) * w : (uint32_t)m;
        const uint32_t t0 = rbase[g], t1 = rbase[g + 1];
        uint32_t np = t0;
        const int ok = eliminate_list(rows, rhs, pcoef, pstart, pbit, plist, t0, t1, r1,
                                      [&](uint32_t i) { plist[np++] = (uint16_t)i; });
        rpark[g] = np - t0;
        if (!ok) ok_s = 0;
      }
      __syncthreads();
    }
    if (PRE) {
      // Phase 2: the rows parked at the end of region g continue in rounds;
      // in round t they walk through region g + 1 + t (and are parked again
      // at its end).  In a round every region works on a different region's
      // slots, so all lanes run at once, and a row never leaves its region's
      // list.  After a bounded number of rounds thread 0 finishes whatever is
      // still waiting.
      const uint32_t g = threadIdx.x >> 5;
      const bool leader = (threadIdx.x & 31) == 0;
      int pending = __syncthreads_or(leader && rpark[g] != 0);
      uint32_t round = 0;
      for (; pending && ok_s && round < kRegions; round++) {
        if (leader && rpark[g] != 0) {
          const uint32_t end = g + 2 + round;
          const uint32_t lim = end < kRegions ? end * w : 0xFFFFFFFFu;
          uint32_t keep = 0;
          const int ok = eliminate_list(
              rows, rhs, pcoef, pstart, pbit, plist, rbase[g], rbase[g] + rpark[g], lim,
              [&](uint32_t i) { plist[rbase[g] + keep++] = (uint16_t)i; });
          rpark[g] = keep;
          if (!ok) ok_s = 0;
        }
        pending = __syncthreads_or(leader && rpark[g] != 0);
      }
      if (threadIdx.x == 0 && ok_s && pending) {
        int ok = 1;
        for (uint32_t h = 0; h < kRegions && ok; h++)
          ok = eliminate_list(rows, rhs, pcoef, pstart, pbit, plist, rbase[h], rbase[h] + rpark[h],
                              0xFFFFFFFFu, [](uint32_t) {});
        ok_s = ok;
      }
    } else if (threadIdx.x == 0) {
      // without row precomputation: one thread over the whole table
      int ok = 1;
      for (uint32_t i = 0; i < keys && ok; i++) {
        uint64_t st64, cf, c1;
        ribbon_row(lo[k0 + i], hi[k0 + i], r, m, 64, &st64, &cf, &c1);
        uint32_t st = (uint32_t)st64;
        uint8_t bv = f[k0 + i];
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
  if (threadIdx.x == 0) seeds[sh] = (uint8_t)seed_s;
  // Back substitution from the top.  x[i] = rhs[i] + sum of x[i + j] over
  // the set bits j of row i (pivot slots; 0 elsewhere).  With the column
  // masks cm[p] (bit j = bit j of row p - j: the slots below p whose row
  // holds x[p]) the serial step needs no popcount: acc bit t collects the
  // sum for slot i - t, x[i] = rhs[i] + (acc bit 0), then acc ^= x[i] cm[i]
  // and acc >>= 1.  cm and the packed pivot and rhs bits are built by all
  // threads in the key-row arrays, which the elimination no longer needs;
  // a shard too small for that (or without precomputed rows) takes the
  // popcount form.  A finished 64-slot word of solution bits is kept in the
  // first row slot of its range, which is no longer read.
  const uint64_t nw = (m + 63) / 64;
  const bool colmask = PRE && (size_t)keys * 14 >= (size_t)(m + 2 * nw) * 8;
  if (colmask) {
    uint64_t* cm = pcoef;
    uint64_t* piv = cm + m;
    uint64_t* rb = piv + nw;
    for (uint64_t p = threadIdx.x; p < m; p += kRibbonThreads) {
      uint64_t c = 0;
      const uint32_t jmax = p < 63 ? (uint32_t)p : 63u;
      for (uint32_t j = 1; j <= jmax; j++) c |= ((rows[p - j] >> j) & 1ull) << j;
      cm[p] = c;
    }
    for (uint64_t w = threadIdx.x; w < nw; w += kRibbonThreads) {
      uint64_t pv = 0, rv = 0;
      for (uint32_t b = 0; b < 64 && w * 64 + b < m; b++) {
        pv |= (uint64_t)(rows[w * 64 + b] != 0) << b;
        rv |= (uint64_t)(rhs[w * 64 + b] & 1u) << b;
      }
      piv[w] = pv;
      rb[w] = rv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t acc = 0;
      for (int64_t w = (int64_t)nw - 1; w >= 0; w--) {
        const uint64_t pv = piv[w], rv = rb[w];
        const uint64_t* c = cm + (uint64_t)w * 64;
        uint64_t out = 0;
        const int top = (int)(m - 1 - (uint64_t)w * 64 < 63 ? m - 1 - (uint64_t)w * 64 : 63);
        if (top == 63) {
#pragma unroll 16
          for (int b = 63; b >= 0; b--) {
            const uint64_t v = (pv >> b) & ((rv >> b) ^ acc) & 1ull;
            acc = (acc ^ (c[b] & (0ull - v))) >> 1;
            out |= v << b;
          }
        } else {
          for (int b = top; b >= 0; b--) {
            const uint64_t v = (pv >> b) & ((rv >> b) ^ acc) & 1ull;
            acc = (acc ^ (c[b] & (0ull - v))) >> 1;
            out |= v << b;
          }
        }
        rows[(uint64_t)w * 64] = out;
      }
    }
  } else if (threadIdx.x == 0) {
    uint64_t win = 0, word = 0;  // win bit t = solution at slot i + 1 + t
    for (int64_t grp = (int64_t)((m - 1) >> 3); grp >= 0; grp--) {
      const uint64_t base = (uint64_t)grp * 8;
      uint64_t rw[8];
      uint32_t rv[8];
#pragma unroll
      for (int k = 0; k < 8; k++) {
        rw[k] = base + k < m ? rows[base + k] : 0;
        rv[k] = base + k < m ? rhs[base + k] : 0;
      }
#pragma unroll
      for (int k = 7; k >= 0; k--) {
        const uint64_t v = rw[k] ? (uint64_t)((rv[k] ^ __popcll((rw[k] >> 1) & win)) & 1u) : 0ull;
        win = (win << 1) | v;
        word |= v << ((base + k) & 63);
      }
      if ((base & 63) == 0) {
        rows[base] = word;
        word = 0;
      }
    }
  }
  __syncthreads();
  // OR the solution words into the global vector at the shard's bit offset
  const uint64_t base = shard_off[sh];
  for (uint64_t w = threadIdx.x; w * 64 < m; w += kRibbonThreads) {
    const uint64_t word = rows[w * 64];
    if (word == 0) continue;
    const uint64_t p = base + w * 64;
    const uint32_t s = (uint32_t)(p & 63);
    atomicOr((unsigned long long*)&sol_words[p >> 6], (unsigned long long)(word << s));
    // the next word only when bits land there (it then lies inside the vector)
    if (s && (word >> (64 - s)))
      atomicOr((unsigned long long*)&sol_words[(p >> 6) + 1], (unsigned long long)(word >> (64 - s)));
  }
}

// ---------------------------------------------------------------------------
// 128-bit rows (leaf size n > 24).  A shard's band (16 bytes of row and 1 byte
// of right-hand side per slot, ~210 KB at the default ~12,000 keys) lives in
// shared memory (SMEM) -- or, for a shard too large for it, in global scratch
// indexed by global slot -- and the per-key rows (read once per key and
// seed) in global scratch indexed by global key.  Every elimination step reads
// the band, so it must be in shared memory to be fast: in global memory (L2
// round trips) the solve was ~60x slower.  The elimination is the
// region-parallel one of k_ribbon:
// lane 0 of warp g eliminates the rows that start in region g, rows that step
// past their region are parked and continue in rounds through the following
// regions, and thread 0 finishes any rows still parked.
// ---------------------------------------------------------------------------
struct Band128 {
  uint64_t* lo;  // row bits 0..63 at its pivot slot (0: the slot is free)
  uint64_t* hi;  // row bits 64..127
  uint8_t* rhs;
};
struct Rows128 {  // per key, reduced state while it is parked
  uint64_t* lo;
  uint64_t* hi;
  uint32_t* start;
  uint32_t* list;  // keys in ascending order of their start
  uint8_t* bit;
  uint32_t* cnt;   // per start slot (indexed by global slot): counts, then offsets
};

__device__ __forceinline__ int eliminate128(const Band128& bd, uint32_t* st, uint64_t* clo,
                                            uint64_t* chi, uint8_t* bv, uint32_t limit) {
  uint32_t s = *st;
  uint64_t lo = *clo, hi = *chi;
  uint8_t b = *bv;
  for (;;) {
    if (s >= limit) {
      *st = s;
      *clo = lo;
      *chi = hi;
      *bv = b;
      return 2;
    }
    const uint64_t rl = bd.lo[s];
    if (rl == 0) {  // a stored row has bit 0 set, so 0 marks a free slot
      bd.lo[s] = lo;
      bd.hi[s] = hi;
      bd.rhs[s] = b;
      return 1;
    }
    lo ^= rl;
    hi ^= bd.hi[s];
    b ^= bd.rhs[s];
    if ((lo | hi) == 0) return b ? 0 : 1;
    // bit 0 is now clear: shift the row to its next set bit (1 <= tz <= 127)
    const uint32_t tz = lo ? ctz64(lo) : 64u + ctz64(hi);
    if (tz >= 64) {
      lo = hi >> (tz - 64);
      hi = 0;
    } else {
      lo = (lo >> tz) | (hi << (64 - tz));
      hi >>= tz;
    }
    s += tz;
  }
}

template <class Park>
__device__ __forceinline__ int eliminate_list128(const Band128& bd, const Rows128& rw, uint32_t t0,
                                                 uint32_t t1, uint32_t limit, Park park) {
  for (uint32_t t = t0; t < t1; t++) {
    const uint32_t i = rw.list[t];
    uint32_t st = rw.start[i];
    uint64_t lo = rw.lo[i], hi = rw.hi[i];
    uint8_t bv = rw.bit[i];
    const int res = eliminate128(bd, &st, &lo, &hi, &bv, limit);
    if (res == 0) return 0;
    if (res == 2) {
      rw.start[i] = st;
      rw.lo[i] = lo;
      rw.hi[i] = hi;
      rw.bit[i] = bv;
      park(i);
    }
  }
  return 1;
}

// Shared memory of one shard's band: lo[m] u64 | hi[m] u64 | rhs[m] u8.
__host__ __device__ inline size_t ribbon128_smem(uint64_t m) { return (size_t)m * 17 + 16; }

template <bool SMEM>
__global__ void __launch_bounds__(kRibbonThreads)
    k_ribbon128(const uint64_t* __restrict__ lo, const uint64_t* __restrict__ hi,
                const uint8_t* __restrict__ f, const uint32_t* __restrict__ K, uint64_t B, uint32_t S,
                uint32_t eps_num, const uint64_t* __restrict__ shard_off, Band128 band, Rows128 rows,
                uint64_t* sol_words, uint8_t* seeds, uint32_t* err) {
  extern __shared__ uint64_t band_smem[];
  const uint64_t sh = blockIdx.x;
  const uint64_t b0 = sh * S, b1 = b0 + S < B ? b0 + S : B;
  const uint32_t k0 = K[b0], keys = K[b1] - K[b0];
  const uint64_t m = shard_slots(keys, eps_num, 128);
  if (m == 0) {
    if (threadIdx.x == 0) seeds[sh] = 0;
    return;
  }
  const uint64_t base = shard_off[sh];
  const Band128 bd = SMEM ? Band128{band_smem, band_smem + m, (uint8_t*)(band_smem + 2 * m)}
                          : Band128{band.lo + base, band.hi + base, band.rhs + base};
  const Rows128 rw{rows.lo + k0, rows.hi + k0, rows.start + k0, rows.list + k0, rows.bit + k0,
                   rows.cnt + base};
  __shared__ int ok_s;
  __shared__ uint32_t seed_s;
  __shared__ uint32_t rbase[kRegions + 1], rpark[kRegions];
  __shared__ uint32_t part[kRibbonThreads], wtot[kRegions];
  const uint32_t w = (uint32_t)((m + kRegions - 1) / kRegions);  // region width in slots
  const uint32_t ns = (uint32_t)(m - 127);                        // possible start slots
  const uint32_t per = (ns + kRibbonThreads - 1) / kRibbonThreads;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (uint32_t r = 0; r < kRibbonSeeds; r++) {
    for (uint64_t i = tid; i < m; i += kRibbonThreads) bd.lo[i] = 0;
    for (uint32_t s = tid; s < ns; s += kRibbonThreads) rw.cnt[s] = 0;
    if (tid == 0) {
      ok_s = 1;
      seed_s = r;
    }
    __syncthreads();
    for (uint32_t i = tid; i < keys; i += kRibbonThreads) {
      uint64_t st, c0, c1;
      ribbon_row(lo[k0 + i], hi[k0 + i], r, m, 128, &st, &c0, &c1);
      rw.lo[i] = c0;
      rw.hi[i] = c1;
      rw.start[i] = (uint32_t)st;
      rw.bit[i] = f[k0 + i];
      atomicAdd(&rw.cnt[st], 1u);
    }
    __syncthreads();
    // Counting sort of the keys by start slot: exclusive prefix sums of the
    // per-slot counts (each thread a run of `per` slots), then every key takes
    // the next place of its slot.  Inserting a region's rows in ascending
    // start order bounds each walk by 128 slots: every stored row then spans
    // only columns the new row's window already covers.
    {
      const uint32_t s0 = tid * per, s1 = s0 + per < ns ? s0 + per : ns;
      uint32_t sum = 0;
      for (uint32_t s = s0; s < s1; s++) sum += rw.cnt[s];
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
      }
      if (lane == 31) wtot[warp] = x;
      part[tid] = x - sum;  // exclusive within the warp
      __syncthreads();
      if (warp == 0) {
        const uint32_t c = wtot[lane];
        uint32_t y = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t z = __shfl_up_sync(0xFFFFFFFFu, y, o);
          if (lane >= (uint32_t)o) y += z;
        }
        wtot[lane] = y - c;
      }
      __syncthreads();
      uint32_t off = part[tid] + wtot[warp];
      for (uint32_t s = s0; s < s1; s++) {
        const uint32_t c = rw.cnt[s];
        rw.cnt[s] = off;
        off += c;
      }
    }
    __syncthreads();
    for (uint32_t i = tid; i < keys; i += kRibbonThreads) rw.list[atomicAdd(&rw.cnt[rw.start[i]], 1u)] = i;
    __syncthreads();
    // region g's rows (starts in [g w, (g + 1) w)) are list[rbase[g] .. rbase[g + 1]);
    // rw.cnt[s] now holds the end of slot s
    if (tid <= kRegions) {
      const uint64_t s = (uint64_t)tid * w;
      rbase[tid] = s == 0 ? 0u : (s >= ns ? keys : rw.cnt[s - 1]);
    }
    __syncthreads();
    // phase 1: every region's own rows, in parallel
    if ((threadIdx.x & 31) == 0) {
      const uint32_t g = threadIdx.x >> 5;
      const uint32_t r1 = (g + 1) * w < m ? (g + 1) * w : (uint32_t)m;
      const uint32_t t0 = rbase[g], t1 = rbase[g + 1];
      uint32_t np = t0;
      const int ok = eliminate_list128(bd, rw, t0, t1, r1, [&](uint32_t i) { rw.list[np++] = i; });
      rpark[g] = np - t0;
      if (!ok) ok_s = 0;
    }
    __syncthreads();
    // phase 2: parked rows continue through the following regions in rounds
    // (in round t region g's rows walk region g + 1 + t; no two warps share a
    // region in a round), then thread 0 finishes what is left
    const uint32_t g = threadIdx.x >> 5;
    const bool leader = (threadIdx.x & 31) == 0;
    int pending = __syncthreads_or(leader && rpark[g] != 0);
    for (uint32_t round = 0; pending && ok_s && round < kRegions; round++) {
      if (leader && rpark[g] != 0) {
        const uint32_t end = g + 2 + round;
        const uint32_t lim = end < kRegions ? end * w : 0xFFFFFFFFu;
        uint32_t keep = 0;
        const int ok = eliminate_list128(bd, rw, rbase[g], rbase[g] + rpark[g], lim,
                                         [&](uint32_t i) { rw.list[rbase[g] + keep++] = i; });
        rpark[g] = keep;
        if (!ok) ok_s = 0;
      }
      pending = __syncthreads_or(leader && rpark[g] != 0);
    }
    if (threadIdx.x == 0 && ok_s && pending) {
      int ok = 1;
      for (uint32_t h = 0; h < kRegions && ok; h++)
        ok = eliminate_list128(bd, rw, rbase[h], rbase[h] + rpark[h], 0xFFFFFFFFu, [](uint32_t) {});
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
  if (threadIdx.x != 0) return;
  seeds[sh] = (uint8_t)seed_s;
  // Back substitution from the top: x[i] = rhs[i] + parity(row[i] bits
  // 1..127 & x[i+1 .. i+127]) on pivot slots, 0 elsewhere; the window
  // (wlo, whi) holds x[i+1 .. i+128].  Finished 64-bit words of the shard's
  // bits are ORed into the global vector at the shard's bit offset.
  uint64_t wlo = 0, whi = 0, word = 0;
  for (int64_t i = (int64_t)m - 1; i >= 0; i--) {
    uint64_t v = 0;
    const uint64_t rl = bd.lo[i];
    if (rl) {
      const uint64_t rh = bd.hi[i];
      const uint64_t slo = (rl >> 1) | (rh << 63), shi = rh >> 1;
      v = (uint64_t)((bd.rhs[i] ^ __popcll(slo & wlo) ^ __popcll(shi & whi)) & 1);
    }
    whi = (whi << 1) | (wlo >> 63);
    wlo = (wlo << 1) | v;
    word |= v << (i & 63);
    if ((i & 63) == 0) {
      if (word) {
        const uint64_t p = base + (uint64_t)i;
        const uint32_t s = (uint32_t)(p & 63);
        atomicOr((unsigned long long*)&sol_words[p >> 6], (unsigned long long)(word << s));
        if (s && (word >> (64 - s)))
          atomicOr((unsigned long long*)&sol_words[(p >> 6) + 1], (unsigned long long)(word >> (64 - s)));
      }
      word = 0;
    }
  }
}

shk_status launch_ribbon(Ctx& c, const uint64_t* lo, const uint64_t* hi, const uint8_t* f,
                         const uint32_t* K, uint64_t B, uint32_t S, uint32_t eps_num, uint32_t w,
                         uint64_t num_shards, const uint64_t* shard_off, uint32_t max_shard_slots,
                         uint64_t total_slots, uint64_t n_keys, uint64_t* sol_words, uint8_t* seeds,
                         uint32_t* err) {
  if (num_shards == 0) return SHK_OK;
  if (w == 128) {
    Band128 band{nullptr, nullptr, nullptr};
    Rows128 rows;
    SHK_TRY(c.arena.alloc(&rows.lo, n_keys));
    SHK_TRY(c.arena.alloc(&rows.hi, n_keys));
    SHK_TRY(c.arena.alloc(&rows.start, n_keys));
    SHK_TRY(c.arena.alloc(&rows.list, n_keys));
    SHK_TRY(c.arena.alloc(&rows.bit, n_keys));
    SHK_TRY(c.arena.alloc(&rows.cnt, total_slots));
    const size_t smem = ribbon128_smem(max_shard_slots);
    if (smem <= 227 * 1024 - 8192) {  // beside the kernel's static shared memory
      SHK_TRY(raise_smem_limit((const void*)k_ribbon128<true>, smem));
      k_ribbon128<true><<<(unsigned)num_shards, kRibbonThreads, smem, c.stream>>>(
          lo, hi, f, K, B, S, eps_num, shard_off, band, rows, sol_words, seeds, err);
    } else {  // a shard too large for shared memory: the band in global scratch
      SHK_TRY(c.arena.alloc(&band.lo, total_slots));
      SHK_TRY(c.arena.alloc(&band.hi, total_slots));
      SHK_TRY(c.arena.alloc(&band.rhs, total_slots));
      k_ribbon128<false><<<(unsigned)num_shards, kRibbonThreads, 0, c.stream>>>(
          lo, hi, f, K, B, S, eps_num, shard_off, band, rows, sol_words, seeds, err);
    }
    c.launches++;
    SHK_CUDA(cudaGetLastError());
    return SHK_OK;
  }
  const size_t limit = 227 * 1024;
  // max_shard_slots belongs to the largest shard, so it bounds its keys too
  const size_t smem_pre = ribbon_smem(max_shard_slots, max_shard_slots, true);
  const size_t smem = ribbon_smem(max_shard_slots, 0, false);
  if (smem_pre <= limit) {
    SHK_TRY(raise_smem_limit((const void*)k_ribbon<true>, smem_pre));
    k_ribbon<true><<<(unsigned)num_shards, kRibbonThreads, smem_pre, c.stream>>>(
        lo, hi, f, K, B, S, eps_num, shard_off, sol_words, seeds, err);
  } else {
    if (smem > limit) return fail(SHK_EINVAL, "retrieval shard too large for shared memory");
    SHK_TRY(raise_smem_limit((const void*)k_ribbon<false>, smem));
    k_ribbon<false><<<(unsigned)num_shards, kRibbonThreads, smem, c.stream>>>(
        lo, hi, f, K, B, S, eps_num, shard_off, sol_words, seeds, err);
  }
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

}  // namespace shk
