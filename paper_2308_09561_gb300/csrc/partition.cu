// partition.cu -- master hash, bucket histogram, prefix sums and the radix
// partition into buckets (paper Sec. 2 RecSplit: keys are hashed to buckets;
// Sec. 8: every key is first reduced to a master hash).
#include "kernels.cuh"

namespace shk {

// ---------------------------------------------------------------------------
// fingerprints
// ---------------------------------------------------------------------------
// String fingerprint: SipHash-2-4 (Aumasson, Bernstein, INDOCRYPT 2012) of the
// key's bytes under two fixed 128-bit keys, lo under (kStrSaltA, kStrSaltB)
// and hi under (kStrSaltB, kStrSaltA); both instances share the word loads.
// load(j) returns the j-th 8-byte little-endian word of the key (bytes past
// the end may hold anything: they are masked off here).
__device__ __forceinline__ uint64_t rotl64d(uint64_t v, int r) { return (v << r) | (v >> (64 - r)); }

__device__ __forceinline__ void sip_round(uint64_t& v0, uint64_t& v1, uint64_t& v2, uint64_t& v3) {
  v0 += v1;
  v1 = rotl64d(v1, 13) ^ v0;
  v0 = rotl64d(v0, 32);
  v2 += v3;
  v3 = rotl64d(v3, 16) ^ v2;
  v0 += v3;
  v3 = rotl64d(v3, 21) ^ v0;
  v2 += v1;
  v1 = rotl64d(v1, 17) ^ v2;
  v2 = rotl64d(v2, 32);
}

struct Sip2 {
  uint64_t a0, a1, a2, a3, b0, b1, b2, b3;
  __device__ __forceinline__ Sip2() {
    a0 = kStrSaltA ^ 0x736f6d6570736575ull;
    a1 = kStrSaltB ^ 0x646f72616e646f6dull;
    a2 = kStrSaltA ^ 0x6c7967656e657261ull;
    a3 = kStrSaltB ^ 0x7465646279746573ull;
    b0 = kStrSaltB ^ 0x736f6d6570736575ull;
    b1 = kStrSaltA ^ 0x646f72616e646f6dull;
    b2 = kStrSaltB ^ 0x6c7967656e657261ull;
    b3 = kStrSaltA ^ 0x7465646279746573ull;
  }
  __device__ __forceinline__ void block(uint64_t w) {
    a3 ^= w;
    b3 ^= w;
    sip_round(a0, a1, a2, a3);
    sip_round(b0, b1, b2, b3);
    sip_round(a0, a1, a2, a3);
    sip_round(b0, b1, b2, b3);
    a0 ^= w;
    b0 ^= w;
  }
  __device__ __forceinline__ void finish(uint64_t* lo, uint64_t* hi) {
    a2 ^= 0xFF;
    b2 ^= 0xFF;
#pragma unroll
    for (int r = 0; r < 4; r++) {
      sip_round(a0, a1, a2, a3);
      sip_round(b0, b1, b2, b3);
    }
    *lo = a0 ^ a1 ^ a2 ^ a3;
    *hi = b0 ^ b1 ^ b2 ^ b3;
  }
};

template <class Load>
__device__ __forceinline__ void sip2_string(Load load, uint64_t len, uint64_t* lo, uint64_t* hi) {
  Sip2 h;
  const uint64_t full = len >> 3;
  for (uint64_t j = 0; j < full; j++) h.block(load(j));
  const uint32_t rem = (uint32_t)(len & 7);
  uint64_t last = (len & 0xFF) << 56;
  if (rem) last |= load(full) & ((1ull << (8 * rem)) - 1);
  h.block(last);
  h.finish(lo, hi);
}

__device__ __forceinline__ void fp_of_string(const uint8_t* p, uint64_t len, uint64_t* lo,
                                             uint64_t* hi) {
  auto load = [&](uint64_t j) {
    uint64_t w = 0;
    const uint64_t rem = len - 8 * j < 8 ? len - 8 * j : 8;
    for (uint64_t t = 0; t < rem; t++) w |= (uint64_t)p[8 * j + t] << (8 * t);
    return w;
  };
  sip2_string(load, len, lo, hi);
}

__device__ __forceinline__ void key_fp(int kind, const void* data, const uint64_t* offs,
                                       uint64_t i, uint64_t* lo, uint64_t* hi) {
  if (kind == SHK_KEYS_U64) {
    const uint64_t k = ((const uint64_t*)data)[i];
    *lo = mix64(k);
    *hi = mix64(k ^ kFpHiSalt);
  } else if (kind == SHK_KEYS_FP128) {
    const ulonglong2 v = ((const ulonglong2*)data)[i];
    *lo = v.x;
    *hi = v.y;
  } else {
    const uint64_t a = offs[i], e = offs[i + 1];
    fp_of_string((const uint8_t*)data + a, e - a, lo, hi);
  }
}

// ---------------------------------------------------------------------------
// bucket histogram in shared memory.  Mode 1: a 32-bit counter per bucket.
// Mode 2 (more buckets): two 16-bit counters per word; an add that takes a
// counter to 2^15 moves 2^15 to the global count, so with fewer than 2^15
// threads in the block no counter reaches 2^16.  Mode 0: global atomics.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void hist_add(uint32_t* hist, uint32_t* counts, uint32_t b, int mode) {
  if (mode == 1) {
    atomicAdd(&hist[b], 1u);
  } else if (mode == 2) {
    const uint32_t sh = (b & 1u) * 16;
    const uint32_t old = atomicAdd(&hist[b >> 1], 1u << sh);
    if (((old >> sh) & 0xFFFFu) == 0x7FFFu) {
      atomicSub(&hist[b >> 1], 0x8000u << sh);
      atomicAdd(&counts[b], 0x8000u);
    }
  } else {
    atomicAdd(&counts[b], 1u);
  }
}

__device__ __forceinline__ uint32_t hist_words(uint64_t B, int mode) {
  return mode == 1 ? (uint32_t)B : mode == 2 ? (uint32_t)((B + 1) / 2) : 0u;
}

__device__ __forceinline__ void hist_flush(const uint32_t* hist, uint32_t* counts, uint64_t B,
                                           int mode) {
  if (mode == 1) {
    for (uint32_t i = threadIdx.x; i < B; i += blockDim.x)
      if (hist[i]) atomicAdd(&counts[i], hist[i]);
  } else if (mode == 2) {
    for (uint32_t i = threadIdx.x; i < B; i += blockDim.x) {
      const uint32_t c = (hist[i >> 1] >> ((i & 1u) * 16)) & 0xFFFFu;
      if (c) atomicAdd(&counts[i], c);
    }
  }
}

// String keys, one warp per 32 consecutive keys: the warp copies the keys'
// bytes (contiguous in the input) into shared memory with aligned 16-byte
// loads -- plain byte loads only for the unaligned head and tail, so nothing
// outside [offs[i0], offs[i0 + cnt]) is read -- and each lane then hashes its
// key from shared memory 8 bytes at a time (the arithmetic of fp_of_string).  Returns false (warp-uniform) when the keys' bytes exceed the
// buffer; the caller then hashes from global memory.
constexpr uint32_t kStrBuf = 2048;  // bytes of shared memory per warp

__device__ __forceinline__ uint64_t load8_smem(const uint8_t* buf, uint32_t q) {
  const uint64_t* w = (const uint64_t*)(buf + (q & ~7u));
  const uint32_t r = 8 * (q & 7u);
  return r ? (w[0] >> r) | (w[1] << (64 - r)) : w[0];
}

// s, e: the warp's byte range [offs[i0], offs[i0 + cnt]); o, oe: this lane's
// key range (lanes below cnt).
__device__ bool string_fp_warp(const uint8_t* data, uint64_t s, uint64_t e, uint64_t o, uint64_t oe,
                               uint32_t cnt, uint8_t* buf, uint64_t* lo, uint64_t* hi) {
  const uint32_t lane = threadIdx.x & 31;
  const uintptr_t ps = (uintptr_t)(data + s), pe = (uintptr_t)(data + e);
  const uintptr_t a0 = ps & ~(uintptr_t)15;
  if (pe - a0 + 16 > kStrBuf) return false;
  const uintptr_t full0 = (ps + 15) & ~(uintptr_t)15, full1 = pe & ~(uintptr_t)15;
  if (full0 < full1) {
    for (uintptr_t a = full0 + 16 * lane; a < full1; a += 16 * 32)
      *(uint4*)(buf + (a - a0)) = *(const uint4*)a;
  }
  // head [ps, min(full0, pe)) and tail [max(full1, full0), pe): under 16 bytes each
  const uintptr_t h1 = full0 < pe ? full0 : pe;
  if (lane < 16 && ps + lane < h1) buf[ps + lane - a0] = *(const uint8_t*)(ps + lane);
  const uintptr_t t0 = full1 > full0 ? full1 : full0;
  if (lane < 16 && t0 + lane < pe) buf[t0 + lane - a0] = *(const uint8_t*)(t0 + lane);
  __syncwarp();
  if (lane < cnt) {
    const uint64_t len = oe - o;
    const uint32_t q = (uint32_t)((uintptr_t)(data + o) - a0);
    sip2_string([&](uint64_t j) { return load8_smem(buf, q + 8 * (uint32_t)j); }, len, lo, hi);
  }
  __syncwarp();
  return true;
}

// Offsets of warp group g: lane l < cnt gets offs[32 g + l]; all lanes get
// the group's end offs[32 g + cnt].
__device__ __forceinline__ void group_offsets(const uint64_t* offs, uint64_t n_keys, uint64_t g,
                                              uint64_t* o, uint64_t* e) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t i0 = g * 32;
  const uint32_t cnt = n_keys - i0 < 32 ? (uint32_t)(n_keys - i0) : 32u;
  *o = lane < cnt ? offs[i0 + lane] : 0;
  *e = offs[i0 + cnt];
}

// a1 for string keys: fingerprints and histogram, one warp per 32 keys; the
// next group's offsets are loaded while the current group is hashed.
// Dynamic shared memory: the histogram words, then kStrBuf bytes per warp.
// Without fp, fingerprints go to lo_out / hi_out (queries) and B is unused.
constexpr int kStrThreadsMax = 1024;

__global__ void __launch_bounds__(kStrThreadsMax)
    k_fingerprint_str(const uint8_t* data, const uint64_t* offs, uint64_t n_keys, uint64_t B,
                      ulonglong2* fp, uint64_t* lo_out, uint64_t* hi_out, uint32_t* counts,
                      int mode) {
  extern __shared__ __align__(16) uint32_t dyn[];
  const uint32_t hw = (hist_words(B, mode) + 3) & ~3u;
  uint32_t* hist = dyn;
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint8_t* buf = (uint8_t*)(dyn + hw) + (size_t)w * kStrBuf;
  for (uint32_t i = threadIdx.x; i < hw; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const uint64_t groups = (n_keys + 31) / 32, stride = (uint64_t)gridDim.x * nw;
  uint64_t g = (uint64_t)blockIdx.x * nw + w;
  uint64_t o = 0, e = 0;
  if (g < groups) group_offsets(offs, n_keys, g, &o, &e);
  while (g < groups) {
    const uint64_t gn = g + stride;
    uint64_t on = 0, en = 0;
    if (gn < groups) group_offsets(offs, n_keys, gn, &on, &en);
    const uint64_t i0 = g * 32;
    const uint32_t cnt = n_keys - i0 < 32 ? (uint32_t)(n_keys - i0) : 32u;
    const uint64_t s = __shfl_sync(0xFFFFFFFFu, o, 0);
    const uint64_t nx = __shfl_down_sync(0xFFFFFFFFu, o, 1);
    const uint64_t oe = lane + 1 < cnt ? nx : e;
    uint64_t l = 0, h = 0;
    if (!string_fp_warp(data, s, e, o, oe, cnt, buf, &l, &h) && lane < cnt)
      fp_of_string(data + o, oe - o, &l, &h);
    if (lane < cnt) {
      const uint64_t i = i0 + lane;
      if (fp) {
        fp[i] = make_ulonglong2(l, h);
        hist_add(hist, counts, (uint32_t)mulhi64(h, B), mode);
      } else {
        lo_out[i] = l;
        hi_out[i] = h;
      }
    }
    g = gn;
    o = on;
    e = en;
  }
  __syncthreads();
  if (fp) hist_flush(hist, counts, B, mode);
}

// a1: fingerprints (one 16-byte record per key: lo, hi) and the bucket
// histogram.  The bucket of a key is mulhi(hi, B) and is recomputed where
// needed rather than stored.
__global__ void k_fingerprint(int kind, const void* data, const uint64_t* offs, uint32_t n_keys,
                              uint64_t B, ulonglong2* fp, uint32_t* counts, int mode) {
  extern __shared__ uint32_t hist[];
  for (uint32_t i = threadIdx.x; i < hist_words(B, mode); i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_keys; i += stride) {
    uint64_t l, h;
    key_fp(kind, data, offs, i, &l, &h);
    fp[i] = make_ulonglong2(l, h);
    hist_add(hist, counts, (uint32_t)mulhi64(h, B), mode);
  }
  __syncthreads();
  hist_flush(hist, counts, B, mode);
}

// Fingerprints only (queries).
__global__ void k_fingerprint_only(int kind, const void* data, const uint64_t* offs,
                                   uint64_t n_keys, uint64_t* lo, uint64_t* hi) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_keys; i += stride)
    key_fp(kind, data, offs, i, &lo[i], &hi[i]);
}

// ---------------------------------------------------------------------------
// exclusive prefix sums: out[0..n] with out[n] = total
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanItems;

template <class T>
__device__ T block_exclusive_scan(T v, T* total) {
  __shared__ T warp_tot[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    T t = lane < nw ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_tot[lane] = t;
  }
  __syncthreads();
  const T before = w ? warp_tot[w - 1] : T(0);
  *total = warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

template <class Tin, class T>
__global__ void k_scan_tiles(const Tin* in, uint64_t n, T* out, T* tile_sums) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    v[j] = base + j < n ? (T)in[base + j] : T(0);
    s += v[j];
  }
  T total;
  T pre = block_exclusive_scan<T>(s, &total);
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    if (base + j < n) out[base + j] = pre;
    pre += v[j];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

template <class T>
__global__ void k_scan_add(T* out, uint64_t n, const T* tile_pre) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  const T add = tile_pre[blockIdx.x];
  for (uint64_t i = base + threadIdx.x; i < base + kScanTile && i < n; i += blockDim.x) out[i] += add;
}

template <class T>
__global__ void k_scan_total(T* out, uint64_t n, const T* tile_pre, uint64_t tiles) {
  out[n] = tile_pre[tiles];
}

template <class Tin, class T>
shk_status exclusive_scan(Ctx& c, const Tin* in, uint64_t n, T* out) {
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (n == 0) {
    SHK_CUDA(cudaMemsetAsync(out, 0, sizeof(T), c.stream));
    return SHK_OK;
  }
  T* sums;
  T* pre;
  SHK_TRY(c.arena.alloc(&sums, tiles));
  SHK_TRY(c.arena.alloc(&pre, tiles + 1));
  k_scan_tiles<Tin, T><<<(unsigned)tiles, kScanThreads, 0, c.stream>>>(in, n, out, sums);
  c.launches++;
  if (tiles > 1) {
    SHK_TRY((exclusive_scan<T, T>(c, sums, tiles, pre)));
    k_scan_add<T><<<(unsigned)tiles, kScanThreads, 0, c.stream>>>(out, n, pre);
    c.launches++;
  } else {
    SHK_CUDA(cudaMemsetAsync(pre, 0, sizeof(T), c.stream));
    SHK_CUDA(cudaMemcpyAsync(pre + 1, sums, sizeof(T), cudaMemcpyDeviceToDevice, c.stream));
  }
  k_scan_total<T><<<1, 1, 0, c.stream>>>(out, n, pre, tiles);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

template shk_status exclusive_scan<uint32_t, uint32_t>(Ctx&, const uint32_t*, uint64_t, uint32_t*);
template shk_status exclusive_scan<uint64_t, uint64_t>(Ctx&, const uint64_t*, uint64_t, uint64_t*);
template shk_status exclusive_scan<uint32_t, uint64_t>(Ctx&, const uint32_t*, uint64_t, uint64_t*);

// ---------------------------------------------------------------------------
// a2: radix partition into buckets, one or two tile-staged passes.
//
// A pass reads a tile of 2048 16-byte records (coalesced), gives each a digit,
// counts the digits in shared memory, reserves one output range per digit
// and tile with a single global atomic, stages the tile in shared memory in
// digit order and writes each digit's run contiguously.  With B <= 512
// buckets one pass by bucket suffices.  Otherwise pass 1 groups the keys by
// the coarse digit bucket >> s1 (the coarse group's output range is the union
// of its buckets' ranges), and pass 2 sorts each tile of that output by
// bucket: a tile lies in at most two coarse groups, so its buckets are
// within 2^(s1+1) of the first group's first bucket.  Keys outside that window
// (a tile spanning more groups, only when groups are smaller than a tile)
// take a direct atomic slot.  The order inside a bucket is arbitrary here and
// fixed by the in-bucket sort at the start of the splitting kernel.
// ---------------------------------------------------------------------------
constexpr int kRadixThreads = 256;
constexpr int kRadixPerThread = 8;
constexpr uint32_t kRadixTile = kRadixThreads * kRadixPerThread;
constexpr uint32_t kRadixDigits = 512;

// shift: digit = bucket >> shift; window_bits >= 32: digits counted from 0
// (pass 1 or the single pass); otherwise from the tile's first key's bucket
// rounded down to a multiple of 2^window_bits (pass 2).
// Capped at 64 registers (4 blocks per SM): holding the next tile in registers
// must not cost resident blocks.
__global__ void __launch_bounds__(kRadixThreads, 4)
    k_radix_pass(const ulonglong2* __restrict__ in, uint32_t n, uint64_t B, uint32_t shift,
                 uint32_t window_bits, const uint32_t* __restrict__ K, uint32_t* cursor,
                 ulonglong2* __restrict__ out) {
  __shared__ ulonglong2 stage[kRadixTile];
  __shared__ uint32_t hist[kRadixDigits], lstart[kRadixDigits], gstart[kRadixDigits];
  __shared__ uint32_t wsum[kRadixThreads / 32];
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t tiles = (n + kRadixTile - 1) / kRadixTile;
  // The next tile's records are loaded into registers while the current
  // tile's staged runs are written out.
  ulonglong2 v[kRadixPerThread];
  auto load_tile = [&](uint32_t tt) {
    const uint32_t b = tt * kRadixTile;
    const uint32_t c = n - b < kRadixTile ? n - b : kRadixTile;
#pragma unroll
    for (int k = 0; k < kRadixPerThread; k++) {
      const uint32_t i = k * kRadixThreads + tid;
      if (i < c) v[k] = in[b + i];
    }
  };
  if (blockIdx.x < tiles) load_tile(blockIdx.x);
  for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint32_t base = t * kRadixTile;
    const uint32_t cnt = n - base < kRadixTile ? n - base : kRadixTile;
    for (uint32_t d = tid; d < kRadixDigits; d += kRadixThreads) hist[d] = 0;
    const uint64_t dbase =
        window_bits >= 32 ? 0 : ((mulhi64(in[base].y, B) >> window_bits) << window_bits);
    __syncthreads();
    uint32_t dg[kRadixPerThread], rk[kRadixPerThread];
#pragma unroll
    for (int k = 0; k < kRadixPerThread; k++) {
      const uint32_t i = k * kRadixThreads + tid;
      dg[k] = kRadixDigits;
      if (i < cnt) {
        const uint64_t da = mulhi64(v[k].y, B) >> shift;
        if (da - dbase < kRadixDigits) {
          dg[k] = (uint32_t)(da - dbase);
          rk[k] = atomicAdd(&hist[dg[k]], 1u);
        } else {
          // outside the window: a direct slot
          out[K[da << shift] + atomicAdd(&cursor[da], 1u)] = v[k];
        }
      }
    }
    __syncthreads();
    // exclusive scan of the 512 digit counts (2 per thread) and one global
    // reservation per non-empty digit
    const uint32_t c0 = hist[2 * tid], c1 = hist[2 * tid + 1];
    uint32_t x = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (uint32_t w = 0; w < warp; w++) before += wsum[w];
    const uint32_t p0 = before + x - (c0 + c1);
    lstart[2 * tid] = p0;
    lstart[2 * tid + 1] = p0 + c0;
#pragma unroll
    for (int j = 0; j < 2; j++) {
      const uint32_t d = 2 * tid + j, c = j ? c1 : c0;
      if (c) {
        const uint64_t da = dbase + d;
        gstart[d] = K[da << shift] + atomicAdd(&cursor[da], c);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRadixPerThread; k++)
      if (dg[k] < kRadixDigits) stage[lstart[dg[k]] + rk[k]] = v[k];
    __syncthreads();
    if (t + gridDim.x < tiles) load_tile(t + gridDim.x);
    // contiguous runs: consecutive threads write consecutive records
    const uint32_t staged = lstart[kRadixDigits - 1] + hist[kRadixDigits - 1];
    for (uint32_t i = tid; i < staged; i += kRadixThreads) {
      const ulonglong2 w = stage[i];
      const uint32_t d = (uint32_t)((mulhi64(w.y, B) >> shift) - dbase);
      out[gstart[d] + (i - lstart[d])] = w;
    }
    __syncthreads();
  }
}

// Histogram mode and its shared-memory bytes for B buckets.
static int hist_mode(uint64_t B, size_t* bytes) {
  if (B <= 12288) {
    *bytes = B * 4;
    return 1;
  }
  if (B <= 81920) {
    *bytes = ((B + 1) / 2) * 4;
    return 2;
  }
  *bytes = 0;
  return 0;
}

template <class Kern>
static shk_status grid_for(Ctx& c, Kern k, int threads, size_t smem, uint64_t work_blocks,
                           int* blocks) {
  int per_sm = 0;
  SHK_TRY(blocks_per_sm((const void*)k, threads, smem, &per_sm));
  if (per_sm < 1) return fail(SHK_ECUDA, "fingerprint kernel does not fit on an SM");
  const uint64_t cap = (uint64_t)c.num_sms * per_sm;
  *blocks = (int)(work_blocks < cap ? (work_blocks ? work_blocks : 1) : cap);
  return SHK_OK;
}

shk_status launch_fingerprint(Ctx& c, int kind, const void* data, const uint64_t* offs,
                              uint32_t n_keys, uint64_t B, ulonglong2* fp, uint32_t* counts) {
  if (n_keys == 0) return SHK_OK;
  size_t hbytes;
  const int mode = hist_mode(B, &hbytes);
  int blocks;
  if (kind == SHK_KEYS_STR) {
    // one large block per SM when every block holds a large histogram
    const int threads = mode == 2 ? kStrThreadsMax : 256;
    const size_t smem = ((hbytes + 15) & ~(size_t)15) + (size_t)(threads / 32) * kStrBuf;
    SHK_TRY(raise_smem_limit((const void*)k_fingerprint_str, smem));
    SHK_TRY(grid_for(c, k_fingerprint_str, threads, smem, (n_keys + threads - 1) / threads, &blocks));
    k_fingerprint_str<<<blocks, threads, smem, c.stream>>>((const uint8_t*)data, offs, n_keys, B, fp,
                                                           nullptr, nullptr, counts, mode);
  } else {
    const int threads = 512;
    SHK_TRY(raise_smem_limit((const void*)k_fingerprint, hbytes));
    SHK_TRY(grid_for(c, k_fingerprint, threads, hbytes, (n_keys + threads - 1) / threads, &blocks));
    k_fingerprint<<<blocks, threads, hbytes, c.stream>>>(kind, data, offs, n_keys, B, fp, counts,
                                                         mode);
  }
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

shk_status launch_fingerprint_only(Ctx& c, int kind, const void* data, const uint64_t* offs,
                                   uint64_t n_keys, uint64_t* lo, uint64_t* hi) {
  if (n_keys == 0) return SHK_OK;
  int blocks;
  if (kind == SHK_KEYS_STR) {
    const int threads = 256;
    const size_t smem = (size_t)(threads / 32) * kStrBuf;
    SHK_TRY(raise_smem_limit((const void*)k_fingerprint_str, smem));
    SHK_TRY(grid_for(c, k_fingerprint_str, threads, smem, (n_keys + threads - 1) / threads, &blocks));
    k_fingerprint_str<<<blocks, threads, smem, c.stream>>>((const uint8_t*)data, offs, n_keys, 1,
                                                           nullptr, lo, hi, nullptr, 0);
  } else {
    SHK_TRY(grid_for(c, k_fingerprint_only, 256, 0, (n_keys + 255) / 256, &blocks));
    k_fingerprint_only<<<blocks, 256, 0, c.stream>>>(kind, data, offs, n_keys, lo, hi);
  }
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

shk_status launch_scatter(Ctx& c, const ulonglong2* fp, uint32_t n_keys, uint64_t B,
                          const uint32_t* K, ulonglong2* sfp) {
  if (n_keys == 0) return SHK_OK;
  uint32_t bbits = 0;
  while ((1ull << bbits) < B) bbits++;
  const uint32_t tiles = (n_keys + kRadixTile - 1) / kRadixTile;
  int per_sm = 0;
  SHK_TRY(blocks_per_sm((const void*)k_radix_pass, kRadixThreads, 0, &per_sm));
  if (per_sm < 1) per_sm = 1;
  const uint32_t cap = (uint32_t)(c.num_sms * per_sm);
  const uint32_t grid = tiles < cap ? tiles : cap;
  if (B <= kRadixDigits) {
    uint32_t* cursor;
    SHK_TRY(c.arena.alloc(&cursor, B, true));
    k_radix_pass<<<grid, kRadixThreads, 0, c.stream>>>(fp, n_keys, B, 0, 32, K, cursor, sfp);
    c.launches++;
  } else {
    // coarse digit bucket >> s1 with about sqrt(B) groups of 2^s1 buckets
    const uint32_t s1 = (bbits + 1) / 2;
    const uint64_t groups = (B + (1ull << s1) - 1) >> s1;
    if (groups > kRadixDigits) return fail(SHK_EINVAL, "too many buckets for the radix partition");
    uint32_t *gcursor, *cursor;
    ulonglong2* tmp;
    SHK_TRY(c.arena.alloc(&gcursor, groups, true));
    SHK_TRY(c.arena.alloc(&cursor, B, true));
    SHK_TRY(c.arena.alloc(&tmp, n_keys));
    k_radix_pass<<<grid, kRadixThreads, 0, c.stream>>>(fp, n_keys, B, s1, 32, K, gcursor, tmp);
    c.launches++;
    k_radix_pass<<<grid, kRadixThreads, 0, c.stream>>>(tmp, n_keys, B, 0, s1, K, cursor, sfp);
    c.launches++;
  }
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

}  // namespace shk
