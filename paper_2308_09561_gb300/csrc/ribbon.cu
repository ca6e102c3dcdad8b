// ribbon.cu -- 1-bit retrieval of the orientation bits of all keys (paper
// Sec. 2 Retrieval: the value is the parity of a hashed row with a segment of
// a solution table; the table solves a nearly diagonal linear system).  A
// standard ribbon of width 64 (leaf size n <= 24) or 128 (n > 24; Sec. 8.2's
// 128-bit words), sharded by runs of buckets; one CTA per shard (64-bit rows)
// or one warp per shard (128-bit rows).
//
// Elimination: each key's row (start, coefficient with bit 0 set) is reduced
// by the row stored at its lowest set column until it reaches a free column
// (a new pivot) or vanishes.  The stored solution is the one that is 0 on
// every non-pivot column; it does not depend on the order of the keys.
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
// 128-bit rows (leaf size n > 24): one warp per (shard, seed) attempt; the
// persistent warps and how they share out seeds are described at k_ribbon128.
//
// The keys are counting-sorted by start slot.  In ascending start order a
// row starting at s only ever meets stored rows whose pivots lie in
// [s, s + 127] and whose bits end at or before s + 127, so the elimination
// needs only a window of 128 slots: slots below the current start are final
// and go out to global memory as the window moves up.
//
// The window is kept reduced: no stored row has a 1 in another stored row's
// pivot column.  Reducing a new row X then takes one step instead of a walk
// of ~25 dependent steps: X is XORed with the stored rows at exactly the
// pivots where X itself has a 1, and the result's lowest set column (from
// X's start, cyclically in the ring) is the new pivot (a free column, since
// the result is 0 on every pivot column).
// The new pivot column is then cleared from the stored rows that have it.
// These extra row operations add rows of the system to rows of the system
// with higher pivots, so the pivot set -- and the solution that is 0 on
// every non-pivot column -- is the one plain sequential elimination gives.
//
// Layout: the window is a ring of 128 slots (slot a at ring index a & 127)
// held as 128 bit columns; lane L of the warp holds columns L, L + 32,
// L + 64, L + 96, each 128 bits over the ring's rows.  One reduction is then
// four column parities per lane and four ballots; occupancy and right-hand
// sides of the ring's rows are 128-bit masks every lane holds.  Rows leave
// the window in ring order (rotated into their pivot frame when the band is
// read back for back substitution).
// ---------------------------------------------------------------------------
constexpr int kRib128Warps = 2;    // warps per CTA
constexpr uint32_t kRib128Spec = 8;  // at most this many warps per shard (seed speculation)

struct Band128 {  // per slot of one warp's shard: the row in ring order (all 0: no pivot here)
  uint4* row;
  uint8_t* rhs;
};
struct Sorted128 {  // per key of one warp's shard, in ascending start order
  uint4* row;       // the row rotated into ring order (bit c is slot start + ((c - start) & 127))
  uint32_t* sb;     // start | orientation bit << 31
  uint32_t* cnt;    // per start slot: counts, then offsets (aliases the band's rows)
};
struct Work128 {    // the persistent warps' scratch, `slots` entries each
  uint4* row;       // [warps][slots] sorted rows
  uint32_t* sb;
  uint4* band;      // [warps][slots] band
  uint8_t* rhs;
  uint64_t slots;
};
struct Shard128 {   // per shard
  uint32_t* best;   // smallest seed known to succeed (~0u: none yet)
  uint32_t* lock;   // held while a warp writes the shard's solution bits
};

struct U128 {
  uint64_t lo, hi;
};

__device__ __forceinline__ U128 rotl128(U128 x, uint32_t r) {  // r in 0..127
  if (r & 64) x = U128{x.hi, x.lo};
  r &= 63;
  if (r == 0) return x;
  return U128{(x.lo << r) | (x.hi >> (64 - r)), (x.hi << r) | (x.lo >> (64 - r))};
}
__device__ __forceinline__ U128 rotr128(U128 x, uint32_t r) { return rotl128(x, (128u - r) & 127u); }

// The window's registers are indexed by 32-slot word; the word of a slot is
// warp-uniform, so a switch on it keeps every index a compile-time constant.
#define SHK_ON_WORD(wi, ...)              \
  switch (wi) {                           \
    case 0: {                             \
      constexpr int W = 0;                \
      __VA_ARGS__;                        \
    } break;                              \
    case 1: {                             \
      constexpr int W = 1;                \
      __VA_ARGS__;                        \
    } break;                              \
    case 2: {                             \
      constexpr int W = 2;                \
      __VA_ARGS__;                        \
    } break;                              \
    default: {                            \
      constexpr int W = 3;                \
      __VA_ARGS__;                        \
    } break;                              \
  }

__device__ __forceinline__ uint32_t first_set128(const uint32_t (&v)[4]) {  // v != 0
  return v[0] ? __ffs((int)v[0]) - 1
              : (v[1] ? 31 + __ffs((int)v[1]) : (v[2] ? 63 + __ffs((int)v[2]) : 95 + __ffs((int)v[3])));
}

// One attempt on a shard of m slots whose rows `srt` are in ascending start
// order; the band goes to `bd`.  Returns false if the system is inconsistent
// or a seed below `seed` has succeeded meanwhile (*best).
// Lane L holds ring columns L + 32 k (k = 0..3), each as 4 words over the
// ring's rows (word w: rows 32 w .. 32 w + 31); occupancy and right-hand
// sides of the ring's rows are 4 words every lane holds.
__device__ bool solve_window128(const Sorted128& srt, uint32_t keys, uint32_t m, const Band128& bd,
                                uint32_t lane, const uint32_t* best, uint32_t seed) {
  uint32_t col[4][4], occ[4], rhs[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    occ[k] = rhs[k] = 0;
#pragma unroll
    for (int w = 0; w < 4; w++) col[k][w] = 0;
  }
  uint32_t fin = 0;  // slots below fin are final and written out
  // rows come in chunks of 32 (lane i holds row t0 + i), the next chunk
  // loading while the current one is eliminated
  uint4 a = make_uint4(0, 0, 0, 0), b = a;
  uint32_t asb = 0, bsb = 0;
  if (lane < keys) a = srt.row[lane], asb = srt.sb[lane];
  if (32 + lane < keys) b = srt.row[32 + lane], bsb = srt.sb[32 + lane];
  for (uint32_t t = 0; t <= keys; t++) {
    if ((t & 31u) == 0 && t) {
      // a smaller seed of this shard has succeeded meanwhile: this attempt
      // cannot be the result (checked every 1024 keys)
      if ((t & 1023u) == 0) {
        uint32_t stop = 0;
        if (lane == 0) stop = *(const volatile uint32_t*)best <= seed;
        if (__shfl_sync(0xFFFFFFFFu, stop, 0)) return false;
      }
      a = b, asb = bsb;
      const uint32_t i = t + 32 + lane;
      if (i < keys) b = srt.row[i], bsb = srt.sb[i];
    }
    const int src = (int)(t & 31u);
    const uint32_t x[4] = {__shfl_sync(0xFFFFFFFFu, a.x, src), __shfl_sync(0xFFFFFFFFu, a.y, src),
                           __shfl_sync(0xFFFFFFFFu, a.z, src), __shfl_sync(0xFFFFFFFFu, a.w, src)};
    const uint32_t sb = __shfl_sync(0xFFFFFFFFu, asb, src);
    const uint32_t s = t < keys ? (sb & 0x7FFFFFFFu) : m;
    // move the window up to s: slots [fin, s) are final
    for (; fin < s; fin++) {
      const uint32_t j = fin & 127u, jm = 1u << (j & 31u);
      bool used = false, rb = false, p[4];
      SHK_ON_WORD(j >> 5, {
        used = (occ[W] & jm) != 0;
        rb = (rhs[W] & jm) != 0;
        _Pragma("unroll") for (int k = 0; k < 4; k++) {
          p[k] = (col[k][W] & jm) != 0;
          col[k][W] &= ~jm;
        }
        occ[W] &= ~jm;
        rhs[W] &= ~jm;
      });
      uint4 row = make_uint4(0, 0, 0, 0);
      if (used) {  // the row's ring-order words; rotated by j when read back
        row.x = __ballot_sync(0xFFFFFFFFu, p[0]);
        row.y = __ballot_sync(0xFFFFFFFFu, p[1]);
        row.z = __ballot_sync(0xFFFFFFFFu, p[2]);
        row.w = __ballot_sync(0xFFFFFFFFu, p[3]);
      }
      if (lane == 0) {
        bd.row[fin] = row;
        bd.rhs[fin] = (uint8_t)rb;
      }
    }
    if (t == keys) break;
    // reduce the new row X (ring order) in one step: XOR of the stored rows
    // at the pivots where X has a 1
    uint32_t y[4], R[4];
    bool p[4];
#pragma unroll
    for (int w = 0; w < 4; w++) y[w] = x[w] & occ[w];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t v = (col[k][0] & y[0]) ^ (col[k][1] & y[1]) ^ (col[k][2] & y[2]) ^ (col[k][3] & y[3]);
      p[k] = (((uint32_t)__popc(v) ^ (x[k] >> lane)) & 1u) != 0;  // X's own bit at column lane + 32 k
    }
#pragma unroll
    for (int k = 0; k < 4; k++) R[k] = __ballot_sync(0xFFFFFFFFu, p[k]);
    const uint32_t bb =
        ((sb >> 31) ^ __popc((y[0] & rhs[0]) ^ (y[1] & rhs[1]) ^ (y[2] & rhs[2]) ^ (y[3] & rhs[3]))) & 1u;
    if ((R[0] | R[1] | R[2] | R[3]) == 0) {
      if (bb) return false;  // dependent and inconsistent
      continue;              // dependent and consistent: nothing to store
    }
    // the new pivot: R's first set ring position at or after s's, cyclically
    const uint32_t rot = s & 127u, rm = ~0u << (rot & 31u);
    uint32_t mk[4];
    SHK_ON_WORD(rot >> 5, {
      _Pragma("unroll") for (int w = 0; w < 4; w++) mk[w] = w < W ? 0u : (w == W ? R[w] & rm : R[w]);
    });
    const uint32_t qj = (mk[0] | mk[1] | mk[2] | mk[3]) ? first_set128(mk) : first_set128(R);
    const uint32_t qm = 1u << (qj & 31u);
    // column qj before the insert (the stored rows with a 1 there), plus row qj
    uint32_t cq[4];
    SHK_ON_WORD(qj >> 5, {
      _Pragma("unroll") for (int w = 0; w < 4; w++) cq[w] = __shfl_sync(0xFFFFFFFFu, col[W][w], (int)(qj & 31u));
    });
    if (bb) {
#pragma unroll
      for (int w = 0; w < 4; w++) rhs[w] ^= cq[w];
    }
    SHK_ON_WORD(qj >> 5, {
      cq[W] |= qm;
      occ[W] |= qm;
      if (bb) rhs[W] |= qm;
    });
    // every column c with R_c = 1: rows of column qj get R (clearing qj), row qj becomes R
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t sel = 0u - ((R[k] >> lane) & 1u);  // all ones where R has column lane + 32 k
#pragma unroll
      for (int w = 0; w < 4; w++) col[k][w] ^= cq[w] & sel;
    }
  }
  return true;
}

// Writes one 64-bit word of a shard's solution: plain store inside the
// shard's bit range [p0, p1), clear-and-set on a word it shares with a
// neighbour.
__device__ __forceinline__ void put_word(uint64_t* sol, uint64_t gw, uint64_t bits, uint64_t p0, uint64_t p1) {
  const uint64_t w0 = gw * 64, w1 = w0 + 64;
  if (w0 >= p0 && w1 <= p1) {
    sol[gw] = bits;
    return;
  }
  const uint64_t lo = p0 > w0 ? p0 - w0 : 0, hi = p1 < w1 ? p1 - w0 : 64;
  const uint64_t mask = (hi == 64 ? ~0ull : (1ull << hi) - 1) & ~((1ull << lo) - 1);
  atomicAnd((unsigned long long*)&sol[gw], (unsigned long long)~mask);
  atomicOr((unsigned long long*)&sol[gw], (unsigned long long)(bits & mask));
}

// Persistent warps take (shard, seed) work items in seed-major order from one
// counter: all shards' seed 0, then seed 1 of those not yet solved, and so
// on.  While many shards are open this is one attempt per shard at a time;
// once fewer shards than warps are open, several seeds of a shard run at
// once.  A warp whose seed succeeds takes the shard's lock and, if its seed
// is still the smallest known, back-substitutes and writes the shard's bits
// and seed; seeds are handed out in increasing order and each shard's
// smallest success writes last, so the result is the first successful seed,
// as in a sequential search.
__global__ void __launch_bounds__(kRib128Warps * 32)
    k_ribbon128(const uint64_t* __restrict__ lo, const uint64_t* __restrict__ hi,
                const uint8_t* __restrict__ f, const uint32_t* __restrict__ K, uint64_t B, uint32_t S,
                uint32_t eps_num, uint64_t num_shards, const uint64_t* __restrict__ shard_off,
                Work128 wk, uint32_t n_warps, Shard128 shd, unsigned long long* next_item,
                unsigned long long* solved, uint64_t* sol_words, uint8_t* seeds, uint32_t* err) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t wid = blockIdx.x * kRib128Warps + (threadIdx.x >> 5);
  if (wid >= n_warps) return;
  const Sorted128 srt{wk.row + wid * wk.slots, wk.sb + wid * wk.slots, (uint32_t*)(wk.band + wid * wk.slots)};
  const Band128 bd{wk.band + wid * wk.slots, wk.rhs + wid * wk.slots};
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = *(volatile unsigned long long*)solved < num_shards ? atomicAdd(next_item, 1ull) : ~0ull;
    item = __shfl_sync(0xFFFFFFFFu, item, 0);
    if (item >= num_shards * kRibbonSeeds) break;
    const uint64_t sh = item % num_shards;
    const uint32_t seed = (uint32_t)(item / num_shards);
    if (*(volatile uint32_t*)&shd.best[sh] <= seed) continue;
    const uint64_t b0 = sh * S, b1 = b0 + S < B ? b0 + S : B;
    const uint32_t k0 = K[b0], keys = K[b1] - K[b0];
    const uint32_t m = (uint32_t)shard_slots(keys, eps_num, 128);
    bool ok = true;
    if (m) {
      const uint32_t ns = m - 127u;  // possible start slots
      // counting sort of the shard's keys by start slot
      for (uint32_t s = lane; s < ns; s += 32) srt.cnt[s] = 0;
      __syncwarp();
      for (uint32_t i = lane; i < keys; i += 32) {
        uint64_t st, c0, c1;
        ribbon_row(lo[k0 + i], hi[k0 + i], seed, m, 128, &st, &c0, &c1);
        atomicAdd(&srt.cnt[st], 1u);
      }
      __syncwarp();
      uint32_t run = 0;
      for (uint32_t s0 = 0; s0 < ns; s0 += 128) {  // four chunks of 32 slots per round
        uint32_t c[4], x[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const uint32_t s = s0 + 32 * j + lane;
          c[j] = s < ns ? srt.cnt[s] : 0u;
          x[j] = c[j];
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
          for (int j = 0; j < 4; j++) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x[j], o);
            if (lane >= (uint32_t)o) x[j] += y;
          }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const uint32_t s = s0 + 32 * j + lane;
          if (s < ns) srt.cnt[s] = run + x[j] - c[j];
          run += __shfl_sync(0xFFFFFFFFu, x[j], 31);
        }
      }
      __syncwarp();
      for (uint32_t i0 = 0; i0 < keys; i0 += 128) {  // four keys per lane in flight
        uint64_t st[4];
        U128 X[4];
        uint32_t pos[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const uint32_t i = i0 + 32 * j + lane;
          if (i < keys) {
            uint64_t c0, c1;
            ribbon_row(lo[k0 + i], hi[k0 + i], seed, m, 128, &st[j], &c0, &c1);
            X[j] = rotl128(U128{c0, c1}, (uint32_t)st[j] & 127u);
            pos[j] = atomicAdd(&srt.cnt[st[j]], 1u);
          }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const uint32_t i = i0 + 32 * j + lane;
          if (i < keys) {
            srt.row[pos[j]] = make_uint4((uint32_t)X[j].lo, (uint32_t)(X[j].lo >> 32), (uint32_t)X[j].hi,
                                         (uint32_t)(X[j].hi >> 32));
            srt.sb[pos[j]] = (uint32_t)st[j] | ((uint32_t)(f[k0 + i] & 1u) << 31);
          }
        }
      }
      __syncwarp();  // the band's first words held the counts
      ok = solve_window128(srt, keys, m, bd, lane, &shd.best[sh], seed);
      __syncwarp();
    }
    if (!ok) continue;
    // the shard's lock (held only while a solution is written; bounded wait)
    uint32_t got = 0;
    if (lane == 0) {
      for (uint32_t it = 0; it < (1u << 24); it++) {
        if (atomicCAS(&shd.lock[sh], 0u, 1u) == 0u) {
          got = 1;
          break;
        }
        __nanosleep(256);
      }
      if (!got) atomicOr(err, kErrRibbon);
      __threadfence();
    }
    got = __shfl_sync(0xFFFFFFFFu, got, 0);
    if (!got) continue;
    const uint32_t prev = *(volatile uint32_t*)&shd.best[sh];
    if (seed < prev) {
      // Back substitution from the top: x[i] = rhs[i] + parity(row[i] bits
      // 1..127 & x[i+1 .. i+127]) on pivot slots, 0 elsewhere; the window
      // (wlo, whi) holds x[i+1 .. i+128].  Every lane runs the recurrence;
      // the band comes in chunks of 32 slots (lane i: slot top - i, rotated
      // from ring order into its pivot frame), the next chunk loading
      // meanwhile.  Lane 0 writes each finished word of the global vector.
      const uint64_t base = shard_off[sh];
      uint64_t wlo = 0, whi = 0, word = 0;
      uint64_t alo = 0, ahi = 0, blo = 0, bhi = 0;
      uint32_t ar = 0, br = 0;
      const int64_t top = (int64_t)m - 1;
      auto load = [&](int64_t i, uint64_t& l, uint64_t& h, uint32_t& r) {
        l = 0, h = 0, r = 0;
        if (i >= 0) {
          const uint4 q = bd.row[i];
          const U128 v = rotr128(U128{q.x | ((uint64_t)q.y << 32), q.z | ((uint64_t)q.w << 32)}, (uint32_t)i & 127u);
          l = v.lo, h = v.hi, r = bd.rhs[i];
        }
      };
      load(top - (int64_t)lane, alo, ahi, ar);
      load(top - 32 - (int64_t)lane, blo, bhi, br);
      for (int64_t c0 = top; c0 >= 0; c0 -= 32) {
        const int n = c0 >= 31 ? 32 : (int)c0 + 1;
        for (int u = 0; u < n; u++) {
          const int64_t i = c0 - u;
          const uint64_t rl = __shfl_sync(0xFFFFFFFFu, alo, u), rh = __shfl_sync(0xFFFFFFFFu, ahi, u);
          const uint32_t rr = __shfl_sync(0xFFFFFFFFu, ar, u);
          uint64_t v = 0;
          if (rl) {
            const uint64_t slo = (rl >> 1) | (rh << 63), shi = rh >> 1;
            v = (uint64_t)((rr ^ __popcll(slo & wlo) ^ __popcll(shi & whi)) & 1u);
          }
          whi = (whi << 1) | (wlo >> 63);
          wlo = (wlo << 1) | v;
          const uint64_t p = base + (uint64_t)i;
          word |= v << (p & 63);
          if ((p & 63) == 0 || i == 0) {
            if (lane == 0) put_word(sol_words, p >> 6, word, base, base + m);
            word = 0;
          }
        }
        alo = blo, ahi = bhi, ar = br;
        load(c0 - 64 - (int64_t)lane, blo, bhi, br);
      }
      if (lane == 0) {
        seeds[sh] = (uint8_t)seed;
        shd.best[sh] = seed;
        if (prev == ~0u) atomicAdd(solved, 1ull);
      }
    }
    if (lane == 0) {
      __threadfence();
      atomicExch(&shd.lock[sh], 0u);
    }
    __syncwarp();
  }
}

__global__ void k_ribbon128_check(const unsigned long long* solved, uint64_t num_shards, uint32_t* err) {
  if (*solved < num_shards) atomicOr(err, kErrRibbon);
}

// Persistent warps for the 128-bit solve: those resident at once, at most
// kRib128Spec per shard.
static shk_status ribbon128_warps(uint64_t num_shards, uint32_t* out) {
  int dev = 0, sms = 0, per_sm = 0;
  SHK_CUDA(cudaGetDevice(&dev));
  SHK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SHK_TRY(blocks_per_sm((const void*)k_ribbon128, kRib128Warps * 32, 0, &per_sm));
  const uint64_t resident = (uint64_t)sms * (per_sm > 0 ? per_sm : 1) * kRib128Warps;
  const uint64_t want = num_shards * kRib128Spec;
  *out = (uint32_t)(want < resident ? want : resident);
  return SHK_OK;
}

// Scratch bytes per persistent warp and slot: sorted rows (16 + 4 per key, at
// most one key per slot) and the band (16 + 1).
constexpr uint64_t kRib128BytesPerSlot = 37;

shk_status ribbon128_scratch_bytes(uint64_t num_shards, uint64_t max_shard_slots, uint64_t* bytes) {
  uint32_t w = 0;
  SHK_TRY(ribbon128_warps(num_shards, &w));
  *bytes = (uint64_t)w * max_shard_slots * kRib128BytesPerSlot + num_shards * 8 + 64;
  return SHK_OK;
}

shk_status launch_ribbon(Ctx& c, const uint64_t* lo, const uint64_t* hi, const uint8_t* f,
                         const uint32_t* K, uint64_t B, uint32_t S, uint32_t eps_num, uint32_t w,
                         uint64_t num_shards, const uint64_t* shard_off, uint32_t max_shard_slots,
                         uint64_t total_slots, uint64_t n_keys, uint64_t* sol_words, uint8_t* seeds,
                         uint32_t* err) {
  if (num_shards == 0) return SHK_OK;
  if (w == 128) {
    // starts and the orientation bit share a 32-bit word
    if (max_shard_slots >= 0x80000000u) return fail(SHK_EINVAL, "retrieval shard too large");
    uint32_t nw = 0;
    SHK_TRY(ribbon128_warps(num_shards, &nw));
    Work128 wk;
    wk.slots = max_shard_slots;
    const uint64_t cells = (uint64_t)nw * max_shard_slots;
    SHK_TRY(c.arena.alloc(&wk.row, cells));
    SHK_TRY(c.arena.alloc(&wk.sb, cells));
    SHK_TRY(c.arena.alloc(&wk.band, cells));
    SHK_TRY(c.arena.alloc(&wk.rhs, cells));
    Shard128 shd;
    unsigned long long* ctr;
    SHK_TRY(c.arena.alloc(&shd.best, num_shards));
    SHK_TRY(c.arena.alloc(&shd.lock, num_shards));
    SHK_TRY(c.arena.alloc(&ctr, 2));
    SHK_CUDA(cudaMemsetAsync(shd.best, 0xFF, num_shards * 4, c.stream));
    SHK_CUDA(cudaMemsetAsync(shd.lock, 0, num_shards * 4, c.stream));
    SHK_CUDA(cudaMemsetAsync(ctr, 0, 16, c.stream));
    const uint32_t blocks = (nw + kRib128Warps - 1) / kRib128Warps;
    k_ribbon128<<<blocks, kRib128Warps * 32, 0, c.stream>>>(lo, hi, f, K, B, S, eps_num, num_shards,
                                                            shard_off, wk, nw, shd, ctr, ctr + 1,
                                                            sol_words, seeds, err);
    k_ribbon128_check<<<1, 1, 0, c.stream>>>(ctr + 1, num_shards, err);
    c.launches += 2;
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
