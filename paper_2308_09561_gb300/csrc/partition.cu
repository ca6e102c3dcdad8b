// partition.cu -- master hash, bucket histogram, prefix sums, radix
// partition into buckets and the in-bucket sort (paper Sec. 2 RecSplit: keys
// are hashed to buckets; Sec. 8: every key is first reduced to a master hash).
#include "kernels.cuh"

namespace shk {

// ---------------------------------------------------------------------------
// fingerprints
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fp_of_string(const uint8_t* p, uint64_t len, uint64_t* lo,
                                             uint64_t* hi) {
  uint64_t a = mix64(kStrSaltA ^ len);
  uint64_t b = mix64(kStrSaltB + len);
  for (uint64_t j = 0; j < len; j += 8) {
    uint64_t w = 0;
    const uint64_t rem = len - j < 8 ? len - j : 8;
    for (uint64_t t = 0; t < rem; t++) w |= (uint64_t)p[j + t] << (8 * t);
    a = mix64(a ^ w);
    b = mix64(b + w);
  }
  *hi = mix64(a + b);
  *lo = mix64(a ^ ((b << 29) | (b >> 35)));
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

// a1: fingerprint + bucket id + bucket histogram (shared-memory histogram
// when the buckets fit, global atomics otherwise).
__global__ void k_fingerprint(int kind, const void* data, const uint64_t* offs, uint32_t n_keys,
                              uint64_t B, uint64_t* lo, uint64_t* hi, uint32_t* bkt,
                              uint32_t* counts, int smem_hist) {
  extern __shared__ uint32_t hist[];
  if (smem_hist) {
    for (uint32_t i = threadIdx.x; i < B; i += blockDim.x) hist[i] = 0;
    __syncthreads();
  }
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_keys; i += stride) {
    uint64_t l, h;
    key_fp(kind, data, offs, i, &l, &h);
    const uint32_t b = (uint32_t)mulhi64(h, B);
    lo[i] = l;
    hi[i] = h;
    bkt[i] = b;
    if (smem_hist)
      atomicAdd(&hist[b], 1u);
    else
      atomicAdd(&counts[b], 1u);
  }
  if (smem_hist) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < B; i += blockDim.x)
      if (hist[i]) atomicAdd(&counts[i], hist[i]);
  }
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
// a2: scatter into buckets, then sort each bucket in shared memory
// ---------------------------------------------------------------------------
__global__ void k_scatter(const uint64_t* lo, const uint64_t* hi, const uint32_t* bkt,
                          uint32_t n_keys, const uint32_t* K, uint32_t* cursor, uint64_t* slo,
                          uint64_t* shi) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_keys; i += stride) {
    const uint32_t b = bkt[i];
    const uint32_t pos = K[b] + atomicAdd(&cursor[b], 1u);
    slo[pos] = lo[i];
    shi[pos] = hi[i];
  }
}

// Bitonic sort of one bucket by (hi, lo) in shared memory; adjacent equal
// fingerprints are duplicate keys.
__global__ void k_bucket_sort(uint64_t* slo, uint64_t* shi, const uint32_t* K, uint32_t* err) {
  extern __shared__ uint64_t sm[];
  const uint32_t b = blockIdx.x;
  const uint32_t start = K[b], size = K[b + 1] - start;
  if (size <= 1) return;
  if (size > kMaxBucketKeys) {
    if (threadIdx.x == 0) atomicOr(err, kErrBucketOverflow);
    return;
  }
  uint32_t P = 1;
  while (P < size) P <<= 1;
  uint64_t* h = sm;
  uint64_t* l = sm + P;
  for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
    h[i] = i < size ? shi[start + i] : ~0ull;
    l[i] = i < size ? slo[start + i] : ~0ull;
  }
  __syncthreads();
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const uint64_t ha = h[i], hb = h[ixj], la = l[i], lb = l[ixj];
          const bool greater = ha > hb || (ha == hb && la > lb);
          const bool asc = (i & k) == 0;
          if (greater == asc) {
            h[i] = hb;
            h[ixj] = ha;
            l[i] = lb;
            l[ixj] = la;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < size; i += blockDim.x) {
    shi[start + i] = h[i];
    slo[start + i] = l[i];
    if (i + 1 < size && h[i] == h[i + 1] && l[i] == l[i + 1]) atomicOr(err, kErrDup);
  }
}

shk_status launch_fingerprint(Ctx& c, int kind, const void* data, const uint64_t* offs,
                              uint32_t n_keys, uint64_t B, uint64_t* lo, uint64_t* hi,
                              uint32_t* bkt, uint32_t* counts) {
  if (n_keys == 0) return SHK_OK;
  const int threads = 256;
  const int smem_hist = B <= 12288 ? 1 : 0;
  const size_t smem = smem_hist ? B * sizeof(uint32_t) : 0;
  if (smem > 48 * 1024)
    SHK_CUDA(cudaFuncSetAttribute(k_fingerprint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int blocks = (int)((n_keys + threads - 1) / threads);
  const int cap = c.num_sms * 8;
  if (blocks > cap) blocks = cap;
  k_fingerprint<<<blocks, threads, smem, c.stream>>>(kind, data, offs, n_keys, B, lo, hi, bkt,
                                                    counts, smem_hist);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

shk_status launch_fingerprint_only(Ctx& c, int kind, const void* data, const uint64_t* offs,
                                   uint64_t n_keys, uint64_t* lo, uint64_t* hi) {
  if (n_keys == 0) return SHK_OK;
  int blocks = (int)((n_keys + 255) / 256);
  if (blocks > c.num_sms * 8) blocks = c.num_sms * 8;
  k_fingerprint_only<<<blocks, 256, 0, c.stream>>>(kind, data, offs, n_keys, lo, hi);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

shk_status launch_partition(Ctx& c, const uint64_t* lo, const uint64_t* hi, const uint32_t* bkt,
                            uint32_t n_keys, uint64_t B, const uint32_t* K, uint32_t max_bucket,
                            uint64_t* slo, uint64_t* shi, uint32_t* err) {
  if (n_keys == 0) return SHK_OK;
  uint32_t* cursor;
  SHK_TRY(c.arena.alloc(&cursor, B, true));
  int blocks = (int)((n_keys + 255) / 256);
  if (blocks > c.num_sms * 8) blocks = c.num_sms * 8;
  k_scatter<<<blocks, 256, 0, c.stream>>>(lo, hi, bkt, n_keys, K, cursor, slo, shi);
  c.launches++;
  uint32_t P = 1;
  while (P < max_bucket) P <<= 1;
  const size_t smem = (size_t)P * 16;
  SHK_CUDA(cudaFuncSetAttribute(k_bucket_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_bucket_sort<<<(unsigned)B, 1024, smem, c.stream>>>(slo, shi, K, err);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

}  // namespace shk
