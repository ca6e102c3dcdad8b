// leaf_rf.cu -- ShockHash leaves with rotation fitting (paper Sec. 4, Rotation
// Fitting) and partial hash calculation (App. A.2).
//
// A fixed 1-bit hash splits a leaf's keys into sets A and B.  Candidate
// v = s*m + r (seed s, rotation r < m) gives the keys of A the cells of seed
// s_A and the keys of B the cells of seed s moved by r (mod m); s_A = s -
// (s mod 8) for leaves of more than 32 keys, s_A = s otherwise.  The leaf value
// is the smallest v whose graph is a pseudoforest.
//
// Warp design: a lane owns 8 consecutive seeds (aligned to 8), so with partial
// hashing set A's bit mask is built once per lane and set B's 8 times.  The
// rotations that pass the coverage filter (A | rot(B, r) has all m bits) are
// found bit-parallel: r is valid iff every cell z that A misses is reached by
// B moved by r, so the valid set is the intersection over those z of the
// reflected B mask rotated by z.  Survivors are tested by the whole warp with
// the peeling characterisation of pseudoforests used in the proof of Thm.
// constructionTries (Sec. 5): after repeatedly removing cells of degree one,
// every remaining cell has degree exactly two.
#include "kernels.cuh"

namespace shk {

constexpr unsigned kFullMask = 0xFFFFFFFFu;
constexpr int kRfSeeds = 8;  // seeds per lane (= the partial-hash period)
// Missed cells of each 32-cell half (m = 64) intersected without branches
// before the surviving rotations are checked one by one (even; the result
// does not depend on it).
#ifndef SHK_RF_HALF
#define SHK_RF_HALF 10
#endif

struct RfScratch {
  uint64_t x[kMaxLeaf];  // leaf inputs (multiplier bit set), set A first
  uint32_t deg[kMaxLeaf];
  uint32_t peeled[kMaxLeaf];
};

__device__ __forceinline__ uint32_t rf_set_dev(uint64_t x) { return (uint32_t)(mix64(x ^ kRfSalt) >> 63); }

// rotate the low m bits left by k (0 <= k < m)
__device__ __forceinline__ uint64_t rotm(uint64_t v, uint32_t k, uint32_t m, uint64_t full) {
  if (k == 0) return v;
  return ((v << k) | (v >> (m - k))) & full;
}

// bit b -> bit (m - b) mod m
__device__ __forceinline__ uint64_t reflectm(uint64_t v, uint32_t m, uint64_t full) {
  return rotm(__brevll(v) >> (64 - m), 1, m, full);
}

// rotations r with A | rot(B, r) == full
__device__ __forceinline__ uint64_t rf_rotations(uint64_t ma, uint64_t mb, uint32_t m,
                                                 uint64_t full) {
  uint64_t z = ~ma & full;
  if (z == 0) return full;
  const uint64_t bh = reflectm(mb, m, full);
  uint64_t r = full;
  while (z) {
    const uint32_t c = __ffsll((long long)z) - 1;
    z &= z - 1;
    r &= rotm(bh, c, m, full);
    if (r == 0) break;
  }
  return r;
}

// 64-bit rotation left by k (0 <= k < 64) from two funnel shifts
__device__ __forceinline__ uint64_t rot64(uint64_t v, uint32_t k) {
  const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
  const uint32_t a = (k & 32) ? hi : lo, b = (k & 32) ? lo : hi;
  return ((uint64_t)__funnelshift_l(a, b, k) << 32) | __funnelshift_l(b, a, k);
}

// Valid rotations of the 8 seeds of a lane that share the set-A mask ma
// (m > 32).  First, for up to K0 cells z missed by A, every seed's set is
// intersected with rot(reflect(B_u), z) without branches (the 8 seeds give
// independent instruction streams and all lanes stay in step); then the few
// rotations left are checked one by one against the remaining cells.  The
// result is the same set as the plain intersection over all missed cells.
template <bool M64>
__device__ __forceinline__ void rf_rotations8(uint64_t ma, const uint64_t* mb, uint32_t m,
                                              uint64_t full, uint64_t* rot) {
  uint64_t z;
  if (M64) {
    // the 64 cells as two 32-bit halves: a rotation by c < 32 (cells of the
    // low half) or by 32 + c (high half) is a pair of funnel shifts; up to
    // kHalf missed cells of each half are intersected without branches
    constexpr int kHalf = SHK_RF_HALF;
    uint32_t zl = ~(uint32_t)ma, zh = ~(uint32_t)(ma >> 32);
    uint32_t rl[kRfSeeds], rh[kRfSeeds], bl[kRfSeeds], bh[kRfSeeds];
#pragma unroll
    for (int u = 0; u < kRfSeeds; u++) {
      const uint64_t b = rot64(__brevll(mb[u]), 1);  // reflect: bit b -> bit (64 - b) mod 64
      bl[u] = (uint32_t)b;
      bh[u] = (uint32_t)(b >> 32);
      rl[u] = ~0u;
      rh[u] = ~0u;
    }
    // two cells per step (a lone last cell is taken twice: the AND is
    // idempotent), so each seed's pair of words takes one three-input AND
    for (int it = 0; it < kHalf / 2 && zl; it++) {
      const uint32_t c = __ffs(zl) - 1;
      zl &= zl - 1;
      const uint32_t d = zl ? __ffs(zl) - 1 : c;
      zl &= zl - 1;
#pragma unroll
      for (int u = 0; u < kRfSeeds; u++) {
        rh[u] &= __funnelshift_l(bl[u], bh[u], c) & __funnelshift_l(bl[u], bh[u], d);
        rl[u] &= __funnelshift_l(bh[u], bl[u], c) & __funnelshift_l(bh[u], bl[u], d);
      }
    }
    for (int it = 0; it < kHalf / 2 && zh; it++) {
      const uint32_t c = __ffs(zh) - 1;
      zh &= zh - 1;
      const uint32_t d = zh ? __ffs(zh) - 1 : c;
      zh &= zh - 1;
#pragma unroll
      for (int u = 0; u < kRfSeeds; u++) {
        rh[u] &= __funnelshift_l(bh[u], bl[u], c) & __funnelshift_l(bh[u], bl[u], d);
        rl[u] &= __funnelshift_l(bl[u], bh[u], c) & __funnelshift_l(bl[u], bh[u], d);
      }
    }
#pragma unroll
    for (int u = 0; u < kRfSeeds; u++) rot[u] = ((uint64_t)rh[u] << 32) | rl[u];
    z = ((uint64_t)zh << 32) | zl;
  } else {
    constexpr int kSteps = 20;
    z = ~ma & full;
    uint64_t bh[kRfSeeds];
#pragma unroll
    for (int u = 0; u < kRfSeeds; u++) {
      bh[u] = reflectm(mb[u], m, full);
      rot[u] = full;
    }
    for (int it = 0; it < kSteps && z; it++) {
      const uint32_t c = __ffsll((long long)z) - 1;
      z &= z - 1;
#pragma unroll
      for (int u = 0; u < kRfSeeds; u++) rot[u] &= rotm(bh[u], c, m, full);
    }
  }
  if (z) {
    // rotation r survives iff every remaining missed cell is in rot(B, r)
#pragma unroll
    for (int u = 0; u < kRfSeeds; u++) {
      uint64_t rr = rot[u], keep = 0;
      while (rr) {
        const uint32_t r = __ffsll((long long)rr) - 1;
        rr &= rr - 1;
        const uint64_t moved = M64 ? rot64(mb[u], r) : rotm(mb[u], r, m, full);
        if ((z & ~moved) == 0) keep |= 1ull << r;
      }
      rot[u] = keep;
    }
  }
}

__device__ __forceinline__ uint32_t add_mod(uint32_t h, uint32_t r, uint32_t m) {
  const uint32_t t = h + r;
  return t >= m ? t - m : t;
}

// Pseudoforest test of candidate (s, r) by parallel peeling; whole warp.
__device__ bool pf_peel(RfScratch* ws, uint32_t m, uint32_t na, uint64_t sa, uint64_t s,
                        uint32_t r) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t ca = mix64(kLeafSalt + sa), cb = mix64(kLeafSalt + s);
  for (uint32_t v = lane; v < m; v += 32) {
    ws->deg[v] = 0;
    ws->peeled[v] = 0;
  }
  __syncwarp();
  uint32_t ea[2] = {0, 0}, eb[2] = {0, 0};
  bool live[2] = {false, false};
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const uint32_t i = lane + 32u * k;
    if (i < m) {
      uint32_t h0, h1;
      leaf_cells(ws->x[i], i < na ? ca : cb, m, &h0, &h1);
      if (i >= na) {
        h0 = add_mod(h0, r, m);
        h1 = add_mod(h1, r, m);
      }
      ea[k] = h0;
      eb[k] = h1;
      live[k] = true;
      atomicAdd(&ws->deg[h0], 1u);
      atomicAdd(&ws->deg[h1], 1u);
    }
  }
  __syncwarp();
  bool ok = true;
  for (int round = 0; round < (int)kMaxLeaf; round++) {
    bool rm[2] = {false, false}, pa[2] = {false, false}, pb[2] = {false, false}, bad = false;
#pragma unroll
    for (int k = 0; k < 2; k++) {
      if (!live[k]) continue;
      const uint32_t da = ws->deg[ea[k]], db = ws->deg[eb[k]];
      if (da == 1 && db == 1) bad = true;  // an edge on its own: a tree
      else if (da == 1 || db == 1) {
        rm[k] = true;
        pa[k] = da == 1;
        pb[k] = db == 1;
      }
    }
    if (__any_sync(kFullMask, bad)) {
      ok = false;
      break;
    }
    if (!__any_sync(kFullMask, rm[0] || rm[1])) break;
    __syncwarp();  // every lane has read the degrees of this round
#pragma unroll
    for (int k = 0; k < 2; k++) {
      if (!rm[k]) continue;
      live[k] = false;
      atomicSub(&ws->deg[ea[k]], 1u);
      atomicSub(&ws->deg[eb[k]], 1u);
      if (pa[k]) ws->peeled[ea[k]] = 1;
      if (pb[k]) ws->peeled[eb[k]] = 1;
    }
    __syncwarp();
  }
  if (ok) {
    bool bad = false;
    for (uint32_t v = lane; v < m; v += 32) {
      const uint32_t d = ws->deg[v];
      if (!(d == 2 || (d == 0 && ws->peeled[v]))) bad = true;
    }
    ok = !__any_sync(kFullMask, bad);
  }
  __syncwarp();
  return ok;
}

// Leaf into shared memory, keys of set A first; returns |A|.
__device__ uint32_t load_leaf_rf(RfScratch* ws, const LeafDesc& d, const uint64_t* x) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  uint64_t xv[2];
  uint32_t ina[2], inb[2], na = 0;
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const uint32_t i = lane + 32u * k;
    const bool valid = i < d.m;
    xv[k] = valid ? x[d.key_off + i] : 0;
    const bool b = valid && rf_set_dev(xv[k]);
    ina[k] = __ballot_sync(kFullMask, valid && !b);
    inb[k] = __ballot_sync(kFullMask, b);
    na += __popc(ina[k]);
  }
  uint32_t pa = 0, pb = na;
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const uint32_t i = lane + 32u * k;
    if (i < d.m) {
      const uint64_t v = xv[k] | (1ull << 32);
      if ((ina[k] >> lane) & 1u)
        ws->x[pa + __popc(ina[k] & lt)] = v;
      else
        ws->x[pb + __popc(inb[k] & lt)] = v;
    }
    pa += __popc(ina[k]);
    pb += __popc(inb[k]);
  }
  __syncwarp();
  return na;
}

__device__ __forceinline__ uint64_t read_uniform_rf(const volatile unsigned long long* p) {
  unsigned long long v = 0;
  if ((threadIdx.x & 31) == 0) v = *p;
  return __shfl_sync(kFullMask, v, 0);
}

// Search seeds s0 .. s0 + passes*256 - 1 (s0 a multiple of 256); returns the
// smallest passing v = s*m + r, or ~0.  WIDE: m > 32 (64-bit masks, partial
// hashing of set A).
template <bool WIDE>
__device__ uint64_t search_rf(RfScratch* ws, uint32_t m, uint32_t na, uint64_t s0,
                              uint32_t passes, const volatile unsigned long long* best,
                              uint32_t* done) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t full = m == 64 ? ~0ull : ((1ull << m) - 1);
  const uint32_t m1 = m - 1;
  for (uint32_t pass = 0; pass < passes; pass++) {
    const uint64_t base = s0 + (uint64_t)pass * (32u * kRfSeeds);
    if (best != nullptr && base * m >= read_uniform_rf(best)) return ~0ull;
    *done += 32u * kRfSeeds;
    const uint64_t sl = base + (uint64_t)lane * kRfSeeds;  // this lane's seeds sl .. sl+7
    uint32_t cl[kRfSeeds], ch[kRfSeeds];
    uint64_t mb[kRfSeeds], ma[kRfSeeds];
#pragma unroll
    for (int u = 0; u < kRfSeeds; u++) {
      const uint64_t c = mix64(kLeafSalt + sl + u);
      cl[u] = (uint32_t)c;
      ch[u] = (uint32_t)(c >> 32);
      mb[u] = 0;
      ma[u] = 0;
    }
    if (WIDE) {
      // set A: one mask for all 8 seeds (seed sl = s - s mod 8)
      uint64_t a = 0;
#pragma unroll 2
      for (uint32_t i = 0; i < na; i++) {
        const uint64_t x = ws->x[i];
        const uint32_t aa = ((uint32_t)x ^ cl[0]) * (uint32_t)(x >> 32) + ch[0];
        const uint64_t w = (uint64_t)aa * m;
        const uint32_t h0 = (uint32_t)(w >> 32);
        const uint32_t t = __umulhi((uint32_t)w, m1);
        const uint32_t h1 = t + (t >= h0 ? 1u : 0u);
        a |= (1ull << h0) | (1ull << h1);
      }
      ma[0] = a;
#pragma unroll 2
      for (uint32_t i = na; i < m; i++) {
        const uint64_t x = ws->x[i];
        const uint32_t xl = (uint32_t)x, mult = (uint32_t)(x >> 32);
#pragma unroll
        for (int u = 0; u < kRfSeeds; u++) {
          const uint32_t aa = (xl ^ cl[u]) * mult + ch[u];
          const uint64_t w = (uint64_t)aa * m;
          const uint32_t h0 = (uint32_t)(w >> 32);
          const uint32_t t = __umulhi((uint32_t)w, m1);
          const uint32_t h1 = t + (t >= h0 ? 1u : 0u);
          mb[u] |= (1ull << h0) | (1ull << h1);
        }
      }
    } else {
#pragma unroll 2
      for (uint32_t i = 0; i < m; i++) {
        const uint64_t x = ws->x[i];
        const uint32_t xl = (uint32_t)x, mult = (uint32_t)(x >> 32);
        const bool in_a = i < na;
#pragma unroll
        for (int u = 0; u < kRfSeeds; u++) {
          const uint32_t aa = (xl ^ cl[u]) * mult + ch[u];
          const uint64_t w = (uint64_t)aa * m;
          const uint32_t h0 = (uint32_t)(w >> 32);
          const uint32_t t = __umulhi((uint32_t)w, m1);
          const uint32_t h1 = t + (t >= h0 ? 1u : 0u);
          const uint64_t bits = (1ull << h0) | (1ull << h1);
          if (in_a)
            ma[u] |= bits;
          else
            mb[u] |= bits;
        }
      }
    }
    uint64_t rot[kRfSeeds];
    if (WIDE) {
      if (m == 64)
        rf_rotations8<true>(ma[0], mb, m, full, rot);
      else
        rf_rotations8<false>(ma[0], mb, m, full, rot);
    } else {
#pragma unroll
      for (int u = 0; u < kRfSeeds; u++) rot[u] = rf_rotations(ma[u], mb[u], m, full);
    }
    bool any = false;
#pragma unroll
    for (int u = 0; u < kRfSeeds; u++) any |= rot[u] != 0;
    uint32_t lanes = __ballot_sync(kFullMask, any);
    while (lanes) {
      const uint32_t l = __ffs(lanes) - 1;
      lanes &= lanes - 1;
      const uint64_t ls = base + (uint64_t)l * kRfSeeds;
#pragma unroll
      for (int u = 0; u < kRfSeeds; u++) {
        uint64_t rr = __shfl_sync(kFullMask, rot[u], l);
        const uint64_t s = ls + u;
        const uint64_t sa = WIDE ? ls : s;
        while (rr) {
          const uint32_t r = __ffsll((long long)rr) - 1;
          rr &= rr - 1;
          if (pf_peel(ws, m, na, sa, s, r)) return s * m + r;
        }
      }
    }
  }
  return ~0ull;
}

__device__ __forceinline__ uint64_t search_rf_dispatch(RfScratch* ws, uint32_t m, uint32_t na,
                                                       uint64_t s0, uint32_t passes,
                                                       const volatile unsigned long long* best,
                                                       uint32_t* done) {
  return m > 32 ? search_rf<true>(ws, m, na, s0, passes, best, done)
                : search_rf<false>(ws, m, na, s0, passes, best, done);
}

__device__ uint32_t find_open_leaf_rf(const uint32_t* closed, uint32_t n_leaves, uint32_t* pos,
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
    const uint32_t bal = __ballot_sync(kFullMask, open != 0);
    if (bal) {
      const uint32_t src = __ffs(bal) - 1;
      uint32_t o = __shfl_sync(kFullMask, open, src);
      const uint32_t w = __shfl_sync(kFullMask, wi, src);
      *pos = w;
      uint32_t k = salt % (uint32_t)__popc(o);
      while (k--) o &= o - 1;
      return w * 32 + (uint32_t)(__ffs(o) - 1);
    }
  }
  return n_leaves;
}

constexpr int kRfWarps = 8;
// Resident blocks per SM the persistent kernel is compiled for (a register
// budget: 65536 / (256 x this)); measured in the tuning notes.
#ifndef SHK_RF_MIN_BLOCKS
#define SHK_RF_MIN_BLOCKS 2
#endif

// Persistent search over all leaves with work stealing; as in plain mode the
// work items are chunks of consecutive seeds handed out in increasing order,
// and the minimum value is committed with atomicMin (values are v = s*m + r,
// so seed order is value order).
__global__ void __launch_bounds__(kRfWarps * 32, SHK_RF_MIN_BLOCKS)
    k_leaf_rf_persistent(const LeafDesc* __restrict__ leaves, uint32_t n_leaves,
                         const uint64_t* __restrict__ x, uint32_t passes,
                         unsigned long long* best, uint32_t* next_chunk, uint32_t* closed,
                         uint32_t* next_leaf, unsigned long long* executed, uint32_t* err,
                         LeafCtl ctl) {
  __shared__ RfScratch scratch[kRfWarps];
  const uint32_t lane = threadIdx.x & 31;
  RfScratch* ws = &scratch[threadIdx.x >> 5];
  const uint32_t gw = blockIdx.x * kRfWarps + (threadIdx.x >> 5);
  leaf_mark_start(ctl);
  bool stop = false;
  const uint32_t nwords = (n_leaves + 31) / 32;
  uint32_t pos = nwords ? (uint32_t)(((uint64_t)gw * 2654435761u) % nwords) : 0;
  const uint64_t chunk = (uint64_t)passes * 32u * kRfSeeds;
  unsigned long long done_seeds = 0;
  while (!stop) {
    uint32_t leaf = 0;
    if (lane == 0) leaf = atomicAdd(next_leaf, 1u);
    leaf = __shfl_sync(kFullMask, leaf, 0);
    if (leaf >= n_leaves) {
      leaf = find_open_leaf_rf(closed, n_leaves, &pos, gw);
      if (leaf >= n_leaves) break;
    }
    const LeafDesc d = leaves[leaf];
    if (d.m < 2 || d.m > kMaxLeaf) {
      if (lane == 0) {
        if (d.m == 1)
          best[leaf] = 0;
        else
          atomicOr(err, kErrLeafSize);
        atomicOr(&closed[leaf >> 5], 1u << (leaf & 31));
      }
      continue;
    }
    const uint32_t na = load_leaf_rf(ws, d, x);
    const uint64_t cap = kSeedCap / d.m;
    for (;;) {
      if (leaf_should_stop(ctl, err)) {
        stop = true;
        break;
      }
      uint32_t ci = 0;
      if (lane == 0) ci = atomicAdd(&next_chunk[leaf], 1u);
      ci = __shfl_sync(kFullMask, ci, 0);
      const uint64_t s0 = (uint64_t)ci * chunk;
      if (s0 * d.m >= read_uniform_rf(&best[leaf])) break;
      if (s0 >= cap) {
        if (lane == 0) {
          atomicOr(err, kErrSeedCap);
          atomicOr(&closed[leaf >> 5], 1u << (leaf & 31));
        }
        break;
      }
      uint32_t done = 0;
      const uint64_t r = search_rf_dispatch(ws, d.m, na, s0, passes, &best[leaf], &done);
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

// The plain form: one warp per leaf, one launch per bucket.
__global__ void __launch_bounds__(kRfWarps * 32)
    k_leaf_rf_range(const LeafDesc* __restrict__ leaves, uint32_t l0, uint32_t l1,
                    const uint64_t* __restrict__ x, uint32_t passes, unsigned long long* best,
                    unsigned long long* executed, uint32_t* err, LeafCtl ctl) {
  __shared__ RfScratch scratch[kRfWarps];
  const uint32_t lane = threadIdx.x & 31;
  RfScratch* ws = &scratch[threadIdx.x >> 5];
  const uint32_t leaf = l0 + blockIdx.x * kRfWarps + (threadIdx.x >> 5);
  if (leaf >= l1) return;
  const LeafDesc d = leaves[leaf];
  const uint32_t na = load_leaf_rf(ws, d, x);
  const uint64_t chunk = (uint64_t)passes * 32u * kRfSeeds;
  const uint64_t cap = kSeedCap / d.m;
  unsigned long long done_seeds = 0;
  for (uint64_t s0 = 0;; s0 += chunk) {
    if (s0 >= cap) {
      if (lane == 0) atomicOr(err, kErrSeedCap);
      break;
    }
    if (leaf_should_stop(ctl, err)) break;
    uint32_t done = 0;
    const uint64_t r = search_rf_dispatch(ws, d.m, na, s0, passes, nullptr, &done);
    done_seeds += done;
    if (r != ~0ull) {
      if (lane == 0) best[leaf] = r;
      break;
    }
  }
  if (lane == 0) atomicAdd(executed, done_seeds);
}

static bool aligned8_rf(const void* p) { return ((uintptr_t)p & 7u) == 0; }

shk_status launch_leaf_rf_persistent(Ctx& c, const LeafSearchArgs& a) {
  if (a.n_leaves == 0) return SHK_OK;
  if (!aligned8_rf(a.best) || !aligned8_rf(a.executed) || !aligned8_rf(a.x))
    return fail(SHK_EINVAL, "seed, counter and key buffers must be 8-byte aligned");
  const uint32_t L = a.n_leaves;
  const uint32_t nwords = (L + 31) / 32;
  uint32_t* state;
  SHK_TRY(c.arena.alloc(&state, (size_t)L + nwords + 1, true));
  int per_sm = 0;
  SHK_TRY(blocks_per_sm((const void*)k_leaf_rf_persistent, kRfWarps * 32, 0, &per_sm));
  if (per_sm < 1) per_sm = 1;
  const uint32_t blocks = (uint32_t)(c.num_sms * per_sm);
  k_leaf_rf_persistent<<<blocks, kRfWarps * 32, 0, c.stream>>>(
      a.leaves, L, a.x, a.cfg.passes, a.best, state, state + L, state + L + nwords, a.executed,
      a.err, a.ctl);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

shk_status launch_leaf_rf_range(Ctx& c, const LeafSearchArgs& a, uint32_t l0, uint32_t l1) {
  if (l1 <= l0) return SHK_OK;
  if (!aligned8_rf(a.best) || !aligned8_rf(a.executed) || !aligned8_rf(a.x))
    return fail(SHK_EINVAL, "seed, counter and key buffers must be 8-byte aligned");
  const uint32_t blocks = (l1 - l0 + kRfWarps - 1) / kRfWarps;
  k_leaf_rf_range<<<blocks, kRfWarps * 32, 0, c.stream>>>(a.leaves, l0, l1, a.x, a.cfg.passes,
                                                           a.best, a.executed, a.err, a.ctl);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

}  // namespace shk
