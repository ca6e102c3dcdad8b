// encode.cu -- Golomb-Rice code of all seeds (paper Sec. 4: the seed is stored
// with Golomb-Rice codes) and the Elias-Fano bucket index (Sec. 1: prefix sums
// of bucket sizes).  Bit vectors are LSB-first: bit p is bit p%64 of word p/64;
// concurrent writers only ever OR bits into zeroed words.
#include "kernels.cuh"

namespace shk {

// OR the low len (<= 64) bits of v into the bit vector at position pos.
__device__ __forceinline__ void or_bits(uint64_t* w, uint64_t pos, uint64_t v, uint32_t len) {
  if (len == 0) return;
  if (len < 64) v &= (1ull << len) - 1;
  if (v == 0) return;
  const uint64_t i = pos >> 6;
  const uint32_t sh = (uint32_t)(pos & 63);
  atomicOr((unsigned long long*)&w[i], (unsigned long long)(v << sh));
  if (sh && sh + len > 64) atomicOr((unsigned long long*)&w[i + 1], (unsigned long long)(v >> (64 - sh)));
}

__device__ __forceinline__ void or_ones(uint64_t* w, uint64_t pos, uint64_t count) {
  while (count > 0) {
    const uint32_t sh = (uint32_t)(pos & 63);
    const uint64_t t = count < 64 - sh ? count : 64 - sh;
    const uint64_t run = t == 64 ? ~0ull : ((1ull << t) - 1);
    atomicOr((unsigned long long*)&w[pos >> 6], (unsigned long long)(run << sh));
    pos += t;
    count -= t;
  }
}

__device__ __forceinline__ uint64_t rice_len(uint64_t s, uint32_t k) { return k + 1 + (s >> k); }

// Bits of each bucket's stream: one warp per bucket.
__global__ void k_rice_bits(const uint64_t* codes, const uint8_t* code_k, const uint32_t* code_base,
                            uint64_t B, uint64_t* bucket_bits) {
  const uint64_t b = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (b >= B) return;
  const uint32_t c0 = code_base[b], c1 = code_base[b + 1];
  uint64_t bits = 0;
  for (uint32_t j = c0 + lane; j < c1; j += 32) bits += rice_len(codes[j], code_k[j]);
  for (int o = 16; o > 0; o >>= 1) bits += __shfl_down_sync(0xFFFFFFFFu, bits, o);
  if (lane == 0) bucket_bits[b] = bits;
}

// Write each bucket's codes at its offset O[b]: one warp per bucket, codes in
// preorder, positions from a warp scan of the code lengths.
__global__ void k_rice_write(const uint64_t* codes, const uint8_t* code_k, const uint32_t* code_base,
                             uint64_t B, const uint64_t* O, uint64_t* words) {
  const uint64_t b = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (b >= B) return;
  const uint32_t c0 = code_base[b], c1 = code_base[b + 1];
  uint64_t pos0 = O[b];
  for (uint32_t j0 = c0; j0 < c1; j0 += 32) {
    const uint32_t j = j0 + lane;
    uint64_t s = 0, len = 0;
    uint32_t k = 0;
    if (j < c1) {
      s = codes[j];
      k = code_k[j];
      len = rice_len(s, k);
    }
    uint64_t incl = len;
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    if (j < c1) {
      const uint64_t p = pos0 + incl - len;
      or_bits(words, p, s, k);        // k low bits, LSB first
      or_ones(words, p + k, s >> k);  // unary quotient; the stop bit stays 0
    }
    pos0 += __shfl_sync(0xFFFFFFFFu, incl, 31);
  }
}

shk_status launch_rice_bits(Ctx& c, const uint64_t* codes, const uint8_t* code_k,
                            const uint32_t* code_base, uint64_t B, uint64_t* bucket_bits) {
  if (B == 0) return SHK_OK;
  k_rice_bits<<<(unsigned)((B * 32 + 255) / 256), 256, 0, c.stream>>>(codes, code_k, code_base, B,
                                                                       bucket_bits);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

shk_status launch_rice_write(Ctx& c, const uint64_t* codes, const uint8_t* code_k,
                             const uint32_t* code_base, uint64_t B, const uint64_t* O,
                             uint64_t* words) {
  if (B == 0) return SHK_OK;
  k_rice_write<<<(unsigned)((B * 32 + 255) / 256), 256, 0, c.stream>>>(codes, code_k, code_base, B,
                                                                        O, words);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

// Elias-Fano: value i puts its low l bits at i*l and sets bit (v >> l) + i.
template <class T>
__global__ void k_ef_write(const T* v, uint64_t count, uint32_t l, uint64_t* low, uint64_t* high) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint64_t x = v[i];
  if (l) or_bits(low, i * l, x, l);
  const uint64_t p = (x >> l) + i;
  atomicOr((unsigned long long*)&high[p >> 6], 1ull << (p & 63));
}

shk_status launch_ef_write_u32(Ctx& c, const uint32_t* v, uint64_t count, uint32_t l,
                               uint64_t* low, uint64_t* high) {
  k_ef_write<uint32_t><<<(unsigned)((count + 255) / 256), 256, 0, c.stream>>>(v, count, l, low, high);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

shk_status launch_ef_write_u64(Ctx& c, const uint64_t* v, uint64_t count, uint32_t l,
                               uint64_t* low, uint64_t* high) {
  k_ef_write<uint64_t><<<(unsigned)((count + 255) / 256), 256, 0, c.stream>>>(v, count, l, low, high);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

// Decoding (loading a serialized MPHF): rank of each high word's first bit
// from a prefix sum of popcounts, then every set bit p of rank r yields value
// r = ((p - r) << l) | low(r).
__global__ void k_popc_words(const uint64_t* high, uint64_t nwords, uint32_t* pc) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nwords) pc[i] = (uint32_t)__popcll(high[i]);
}

__global__ void k_ef_decode(const uint64_t* low, const uint64_t* high, uint64_t nwords,
                            uint64_t hbits, uint32_t l, uint64_t count, const uint64_t* rank0,
                            uint64_t* out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nwords) return;
  uint64_t w = high[i];
  if ((i + 1) * 64 > hbits) {
    const uint32_t valid = (uint32_t)(hbits - i * 64);
    if (valid < 64) w &= (1ull << valid) - 1;
  }
  uint64_t r = rank0[i];
  while (w && r < count) {
    const uint32_t b = __ffsll((long long)w) - 1;
    w &= w - 1;
    const uint64_t p = i * 64 + b;
    uint64_t lowv = 0;
    if (l) {
      const uint64_t q = r * l;
      const uint32_t sh = (uint32_t)(q & 63);
      lowv = low[q >> 6] >> sh;
      if (sh && sh + l > 64) lowv |= low[(q >> 6) + 1] << (64 - sh);
      lowv &= (l == 64) ? ~0ull : ((1ull << l) - 1);
    }
    out[r] = ((p - r) << l) | lowv;
    r++;
  }
}

// Checks of a decoded index before queries use it: K nondecreasing from 0 to
// N with buckets of at most kMaxBucketKeys keys, O nondecreasing from 0 to the
// Rice length.
__global__ void k_validate_index(const uint32_t* K, const uint64_t* O, uint64_t B, uint64_t N,
                                 uint64_t rice_bits, uint32_t* bad) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > B) return;
  bool ok = true;
  if (i == 0) ok = K[0] == 0 && O[0] == 0 && K[B] == N && O[B] == rice_bits;
  if (i < B) ok = ok && K[i] <= K[i + 1] && K[i + 1] - K[i] <= kMaxBucketKeys && O[i] <= O[i + 1];
  if (!ok) atomicOr(bad, 1u);
}

shk_status launch_validate_index(Ctx& c, const uint32_t* K, const uint64_t* O, uint64_t B,
                                 uint64_t N, uint64_t rice_bits, uint32_t* bad) {
  k_validate_index<<<(unsigned)((B + 1 + 255) / 256), 256, 0, c.stream>>>(K, O, B, N, rice_bits, bad);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

shk_status launch_ef_decode(Ctx& c, const uint64_t* low, const uint64_t* high, uint64_t hbits,
                            uint32_t l, uint64_t count, uint64_t* out) {
  const uint64_t nwords = (hbits + 63) / 64;
  SHK_CUDA(cudaMemsetAsync(out, 0, count * sizeof(uint64_t), c.stream));
  if (nwords == 0) return SHK_OK;
  uint32_t* pc;
  uint64_t* rank0;
  SHK_TRY(c.arena.alloc(&pc, nwords));
  SHK_TRY(c.arena.alloc(&rank0, nwords + 1));
  k_popc_words<<<(unsigned)((nwords + 255) / 256), 256, 0, c.stream>>>(high, nwords, pc);
  c.launches++;
  SHK_TRY((exclusive_scan<uint32_t, uint64_t>(c, pc, nwords, rank0)));
  k_ef_decode<<<(unsigned)((nwords + 255) / 256), 256, 0, c.stream>>>(low, high, nwords, hbits, l,
                                                                      count, rank0, out);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

}  // namespace shk
