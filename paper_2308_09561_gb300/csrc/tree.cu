// tree.cu -- the RecSplit splitting tree of every bucket (paper Sec. 2: a
// bucket is split recursively by searching splitting seeds; the shape depends
// only on the node size; Sec. 6: fanouts of the two lowest levels).
#include "kernels.cuh"

namespace shk {

// ---------------------------------------------------------------------------
// shape bookkeeping: one thread per bucket walks the size-only tree
// ---------------------------------------------------------------------------
__global__ void k_tree_count(const uint32_t* K, uint64_t B, uint32_t n, uint32_t* n_leaves,
                             uint32_t* n_codes, uint32_t* n_splits, uint32_t* max_bucket) {
  const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const uint32_t size = K[b + 1] - K[b];
  atomicMax(max_bucket, size);
  uint32_t leaves = 0, codes = 0, splits = 0;
  if (size > 0 && size <= kMaxBucketKeys) {
    uint32_t stack[64];
    int sp = 0;
    stack[sp++] = size;
    while (sp > 0) {
      const uint32_t m = stack[--sp];
      SplitShape s;
      if (split_shape(m, n, &s)) {
        splits++;
        codes++;
        for (uint32_t j = 0; j < s.fanout && sp < 64; j++) stack[sp++] = part_size(m, s, j);
      } else if (m >= 2) {
        leaves++;
        codes++;
      }
    }
  }
  n_leaves[b] = leaves;
  n_codes[b] = codes;
  n_splits[b] = splits;
}

shk_status launch_tree_count(Ctx& c, const uint32_t* K, uint64_t B, uint32_t n,
                             uint32_t* n_leaves, uint32_t* n_codes, uint32_t* n_splits,
                             uint32_t* max_bucket) {
  if (B == 0) return SHK_OK;
  k_tree_count<<<(unsigned)((B + 127) / 128), 128, 0, c.stream>>>(K, B, n, n_leaves, n_codes,
                                                                 n_splits, max_bucket);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

// ---------------------------------------------------------------------------
// a3: split seeds.  One CTA per bucket walks the tree in depth-first preorder;
// for every split node all threads test consecutive seeds (one seed per
// thread per round) until some seed sends exactly the prescribed number of
// keys to every child; the smallest such seed wins.  The node's keys are then
// partitioned stably by child, so leaves keep ascending fingerprint order.
// ---------------------------------------------------------------------------
constexpr int kSplitThreads = 256;

// Split hash: a = (hi32(x) ^ lo32(d)) * (lo32(x) | 1) + hi32(d), v = hi32(a * m).
__device__ __forceinline__ uint32_t split_value(uint64_t x, uint64_t d, uint32_t m) {
  const uint32_t a = ((uint32_t)(x >> 32) ^ (uint32_t)d) * ((uint32_t)x | 1u) + (uint32_t)(d >> 32);
  return __umulhi(a, m);
}

__device__ __forceinline__ uint32_t split_child_dev(uint64_t x, uint64_t d, uint32_t m,
                                                    uint32_t t1, uint32_t t2, uint32_t t3) {
  const uint32_t v = split_value(x, d, m);
  return (uint32_t)(v >= t1) + (uint32_t)(v >= t2) + (uint32_t)(v >= t3);
}

__device__ uint64_t block_exclusive_scan_u64(uint64_t v) {
  __shared__ uint64_t wt[kSplitThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wt[w] = x;
  __syncthreads();
  if (w == 0) {
    uint64_t t = lane < kSplitThreads / 32 ? wt[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kSplitThreads / 32) wt[lane] = t;
  }
  __syncthreads();
  const uint64_t before = w ? wt[w - 1] : 0;
  __syncthreads();
  return before + x - v;
}

// Sort of one bucket by (hi, lo) in shared memory.  Inside bucket b the
// low 64 bits of hi * B grow with hi, so their top bits give sub-bins in key
// order: a counting sort into about one sub-bin per key, then an insertion
// sort inside each sub-bin (a handful of keys).  lo/hi/idx receive the sorted
// keys and their positions in the bucket's input range; adjacent equal
// fingerprints are duplicate keys.
__device__ void sort_bucket(const ulonglong2* __restrict__ in, uint32_t size, uint64_t B,
                           uint32_t sub_bits, uint32_t* cnt, uint64_t* lo, uint64_t* hi,
                           uint16_t* idx, uint32_t* err) {
  const uint32_t tid = threadIdx.x, nsub = 1u << sub_bits, sh = 64 - sub_bits;
  for (uint32_t i = tid; i < nsub; i += kSplitThreads) cnt[i] = 0;
  __syncthreads();
  for (uint32_t j = tid; j < size; j += kSplitThreads) atomicAdd(&cnt[(in[j].y * B) >> sh], 1u);
  __syncthreads();
  // exclusive prefix sums of the sub-bin counts: thread t owns a contiguous run
  const uint32_t per = (nsub + kSplitThreads - 1) / kSplitThreads;
  const uint32_t i0 = tid * per < nsub ? tid * per : nsub, i1 = i0 + per < nsub ? i0 + per : nsub;
  uint64_t run = 0;
  for (uint32_t i = i0; i < i1; i++) run += cnt[i];
  uint64_t pre = block_exclusive_scan_u64(run);
  for (uint32_t i = i0; i < i1; i++) {
    const uint32_t c = cnt[i];
    cnt[i] = (uint32_t)pre;
    pre += c;
  }
  __syncthreads();
  for (uint32_t j = tid; j < size; j += kSplitThreads) {
    const ulonglong2 v = in[j];
    const uint32_t p = atomicAdd(&cnt[(v.y * B) >> sh], 1u);
    lo[p] = v.x;
    hi[p] = v.y;
    idx[p] = (uint16_t)j;
  }
  __syncthreads();
  // cnt[s] is now the end of sub-bin s
  for (uint32_t sb = tid; sb < nsub; sb += kSplitThreads) {
    const uint32_t e = cnt[sb], b0 = sb ? cnt[sb - 1] : 0;
    for (uint32_t i = b0 + 1; i < e; i++) {
      const uint64_t kh = hi[i], kl = lo[i];
      const uint16_t ki = idx[i];
      uint32_t j = i;
      while (j > b0 && (hi[j - 1] > kh || (hi[j - 1] == kh && lo[j - 1] > kl))) {
        hi[j] = hi[j - 1];
        lo[j] = lo[j - 1];
        idx[j] = idx[j - 1];
        j--;
      }
      hi[j] = kh;
      lo[j] = kl;
      idx[j] = ki;
    }
  }
  __syncthreads();
  for (uint32_t j = tid; j + 1 < size; j += kSplitThreads)
    if (hi[j] == hi[j + 1] && lo[j] == lo[j + 1]) atomicOr(err, kErrDup);
  __syncthreads();
}

__global__ void __launch_bounds__(kSplitThreads)
    k_split(const ulonglong2* __restrict__ sfp, const uint32_t* __restrict__ K, uint64_t B,
            uint32_t n, uint32_t cap, uint32_t sub_bits, const uint32_t* __restrict__ code_base,
            const uint32_t* __restrict__ leaf_base, uint64_t* __restrict__ codes,
            uint8_t* __restrict__ code_k, LeafDesc* __restrict__ leaves,
            uint64_t* __restrict__ llo, uint64_t* __restrict__ lhi, uint32_t* err) {
  extern __shared__ uint64_t smem[];
  const uint32_t b = blockIdx.x;
  const uint32_t start = K[b], size = K[b + 1] - start;
  if (size == 0 || size > kMaxBucketKeys) return;
  uint64_t* lo = smem;
  uint64_t* tlo = lo + cap;
  uint16_t* idx = (uint16_t*)(tlo + cap);
  uint16_t* tidx = idx + cap;
  uint32_t* cnt = (uint32_t*)(tidx + cap);

  __shared__ uint32_t st_off[64], st_m[64];
  __shared__ int sp;
  __shared__ uint32_t cc, lc, cur_off, cur_m;
  __shared__ unsigned long long found;
  const uint32_t tid = threadIdx.x;

  // a2 (second half): the bucket in (hi, lo) order; tlo holds hi until the
  // first split, which only needs lo
  sort_bucket(sfp + start, size, B, sub_bits, cnt, lo, tlo, idx, err);
  if (tid == 0) {
    sp = 0;
    st_off[sp] = 0;
    st_m[sp] = size;
    sp++;
    cc = code_base[b];
    lc = leaf_base[b];
  }
  __syncthreads();

  for (;;) {
    if (sp == 0) break;
    __syncthreads();
    if (tid == 0) {
      sp--;
      cur_off = st_off[sp];
      cur_m = st_m[sp];
      found = ~0ull;
    }
    __syncthreads();
    const uint32_t off = cur_off, m = cur_m;
    SplitShape sh;
    if (!split_shape(m, n, &sh)) {
      if (tid == 0 && m >= 2) {
        LeafDesc d;
        d.key_off = start + off;
        d.m = m;
        d.code_idx = cc;
        d.bucket = b;
        leaves[lc] = d;
        code_k[cc] = (uint8_t)rice_k_leaf(m);
        cc++;
        lc++;
      }
      __syncthreads();
      continue;
    }
    // thresholds of the children and the expected counts of "v >= t_j"
    const uint32_t u = sh.unit, f = sh.fanout;
    const uint32_t t1 = u, t2 = f > 2 ? 2 * u : 0xFFFFFFFFu, t3 = f > 3 ? 3 * u : 0xFFFFFFFFu;
    const uint32_t e1 = m - u, e2 = f > 2 ? m - 2 * u : 0, e3 = f > 3 ? m - 3 * u : 0;
    const uint64_t g = mix64(kSplitSalt + m);
    // the node's keys as (xor input, multiplier) pairs for the search; tlo is
    // free until the partition below
    uint2* xk = (uint2*)tlo;
    for (uint32_t j = tid; j < m; j += kSplitThreads) {
      const uint64_t x = lo[off + j];
      xk[j] = make_uint2((uint32_t)(x >> 32), (uint32_t)x | 1u);
    }
    __syncthreads();
    // Four equal parts (m = 4u <= 256): the child floor(v / u) of
    // v = floor(a m / 2^32) is floor(4 a / 2^32), and 8 times it is
    // floor(32 a / 2^32) with the low 3 bits cleared; the counts are kept in
    // the four bytes of one word (a byte overflows only when all 256 keys
    // fall into one child, which never matches the expected counts).
    const bool equal4 = f == 4 && m == 4 * u && m <= 256;
    bool capped = false;
    for (uint64_t base = 0;; base += kSplitThreads) {
      const uint64_t s = base + tid;
      const uint64_t d = mix64(g + s);
      const uint32_t dl = (uint32_t)d, dh = (uint32_t)(d >> 32);
      bool hit;
      if (equal4) {
        uint32_t acc = 0;
        for (uint32_t j = 0; j < m; j++) {
          const uint32_t a = (xk[j].x ^ dl) * xk[j].y + dh;
          acc += 1u << (__umulhi(a, 32u) & ~7u);
        }
        hit = acc == u * 0x01010101u;
      } else if (f == 2) {
        uint32_t c1 = 0;
        for (uint32_t j = 0; j < m; j++) c1 += __umulhi((xk[j].x ^ dl) * xk[j].y + dh, m) >= t1;
        hit = c1 == e1;
      } else if (f == 3) {
        uint32_t c1 = 0, c2 = 0;
        for (uint32_t j = 0; j < m; j++) {
          const uint32_t v = __umulhi((xk[j].x ^ dl) * xk[j].y + dh, m);
          c1 += v >= t1;
          c2 += v >= t2;
        }
        hit = c1 == e1 && c2 == e2;
      } else {
        uint32_t c1 = 0, c2 = 0, c3 = 0;
        for (uint32_t j = 0; j < m; j++) {
          const uint32_t v = __umulhi((xk[j].x ^ dl) * xk[j].y + dh, m);
          c1 += v >= t1;
          c2 += v >= t2;
          c3 += v >= t3;
        }
        hit = c1 == e1 && c2 == e2 && c3 == e3;
      }
      if (hit) atomicMin(&found, (unsigned long long)s);
      __syncthreads();
      const unsigned long long fnd = found;
      __syncthreads();
      if (fnd != ~0ull) break;
      if (base + kSplitThreads >= kSeedCap) {
        capped = true;
        break;
      }
    }
    if (capped) {
      if (tid == 0) atomicOr(err, kErrSeedCap);
      break;
    }
    const uint64_t seed = found;
    const uint64_t d = mix64(g + seed);
    if (tid == 0) {
      codes[cc] = seed;
      code_k[cc] = (uint8_t)rice_k_split(m, n);
      cc++;
    }
    // stable partition by child: packed 16-bit child counters, block scan
    const uint32_t ipt = (m + kSplitThreads - 1) / kSplitThreads;
    const uint32_t j0 = tid * ipt < m ? tid * ipt : m;
    const uint32_t j1 = j0 + ipt < m ? j0 + ipt : m;
    uint64_t cnt = 0;
    for (uint32_t j = j0; j < j1; j++)
      cnt += 1ull << (16 * split_child_dev(lo[off + j], d, m, t1, t2, t3));
    uint64_t pre = block_exclusive_scan_u64(cnt);
    for (uint32_t j = j0; j < j1; j++) {
      const uint32_t ch = split_child_dev(lo[off + j], d, m, t1, t2, t3);
      const uint32_t pos = ch * u + (uint32_t)((pre >> (16 * ch)) & 0xFFFFu);
      pre += 1ull << (16 * ch);
      tlo[off + pos] = lo[off + j];
      tidx[off + pos] = idx[off + j];
    }
    __syncthreads();
    for (uint32_t j = tid; j < m; j += kSplitThreads) {
      lo[off + j] = tlo[off + j];
      idx[off + j] = tidx[off + j];
    }
    if (tid == 0) {
      for (int j = (int)f - 1; j >= 0; j--) {
        st_off[sp] = off + (uint32_t)j * u;
        st_m[sp] = part_size(m, sh, (uint32_t)j);
        sp++;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  for (uint32_t j = tid; j < size; j += kSplitThreads) {
    llo[start + j] = lo[j];
    lhi[start + j] = sfp[start + idx[j]].y;
  }
}

shk_status launch_split(Ctx& c, const ulonglong2* sfp, const uint32_t* K, uint64_t B, uint32_t n,
                        uint32_t max_bucket, const uint32_t* code_base, const uint32_t* leaf_base,
                        uint64_t* codes, uint8_t* code_k, LeafDesc* leaves, uint64_t* llo,
                        uint64_t* lhi, uint32_t* err) {
  if (B == 0) return SHK_OK;
  const uint32_t cap = (max_bucket + 7) & ~7u;
  uint32_t sub_bits = 5;  // about one sub-bin per key, at least 32
  while ((1u << sub_bits) < max_bucket) sub_bits++;
  const size_t smem = (size_t)cap * (8 + 8 + 2 + 2) + ((size_t)4 << sub_bits);
  SHK_TRY(raise_smem_limit((const void*)k_split, smem));
  k_split<<<(unsigned)B, kSplitThreads, smem, c.stream>>>(sfp, K, B, n, cap, sub_bits, code_base,
                                                          leaf_base, codes, code_k, leaves, llo,
                                                          lhi, err);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

}  // namespace shk
