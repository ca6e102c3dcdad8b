// shk_internal.cuh -- shared definitions of the GB300 ShockHash-RS library.
//
// Format constants and the arithmetic of the SHKRS002 format as used by the
// kernels.  The definitions follow the paper (ShockHash, Sec. 4; ShockHash-RS,
// Sec. 6) and the project's frozen readings for what the paper leaves open.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <exception>
#include <mutex>
#include <new>
#include <string>

#include "../../include/shk.h"

namespace shk {

// ---------------------------------------------------------------------------
// format constants (hex digits of pi as salts)
// ---------------------------------------------------------------------------
constexpr uint64_t kFpHiSalt = 0x243F6A8885A308D3ull;
constexpr uint64_t kLeafSalt = 0x13198A2E03707344ull;
constexpr uint64_t kSplitSalt = 0xBE5466CF34E90C6Cull;
constexpr uint64_t kRetSalt = 0xC0AC29B7C97C50DDull;
constexpr uint64_t kRetSalt2 = 0x3F84D5B5B5470917ull;
constexpr uint64_t kRetSalt3 = 0xA4093822299F31D0ull;
constexpr uint64_t kStrSaltA = 0x9216D5D98979FB1Bull;
constexpr uint64_t kStrSaltB = 0xD1310BA698DFB5ACull;
constexpr uint64_t kRfSalt = 0x2FFD72DBD01ADFB7ull;  // rotation fitting: set split
constexpr uint64_t kMagic = 0x32303053524B4853ull;  // "SHKRS002"
constexpr uint32_t kHeaderWords = 16;
constexpr uint32_t kMaxLeaf = 64;
constexpr uint32_t kMaxBucketSize = 4096;   // largest accepted b
constexpr uint32_t kMaxBucketKeys = 8192;   // largest bucket the kernels hold
constexpr uint64_t kSeedCap = 1ull << 40;   // seeds searched below this
constexpr uint32_t kRibbonSeeds = 256;      // shard seeds tried
constexpr uint32_t kDefaultEpsNum = 3277;   // eps ~ 5 % (64-bit rows)
constexpr uint32_t kDefaultEpsNum128 = 66;   // eps ~ 0.1 % (128-bit rows)
constexpr uint32_t kNoCode = 0xFFFFFFFFu;

// device error flags (bit set in a u32 word)
constexpr uint32_t kErrDup = 1u << 0;
constexpr uint32_t kErrSeedCap = 1u << 1;
constexpr uint32_t kErrBucketOverflow = 1u << 2;
constexpr uint32_t kErrRibbon = 1u << 3;
constexpr uint32_t kErrLeafSize = 1u << 4;
constexpr uint32_t kErrOrient = 1u << 5;
constexpr uint32_t kErrTimeout = 1u << 6;    // a build's deadline passed
constexpr uint32_t kErrCancelled = 1u << 7;  // the abort flag was set

// Device global timer in ns.
__device__ __forceinline__ uint64_t global_ns() {
#ifdef __CUDA_ARCH__
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
#else
  return 0;
#endif
}

// Rice parameter of a leaf of m keys (frozen literal table of the format):
// floor(log2(ln2 * 0.8 (e/2)^m e / sqrt(pi m))), the trial bound of the
// paper's Thm. shockHashConstruction divided by sqrt(m) (Sec. 8.1).
__host__ __device__ inline uint32_t rice_k_leaf(uint32_t m) {
  constexpr uint8_t t[65] = {0,  0,  0,  0,  0,  0,  1,  1,  1,  2,  2,  2,  3,  3,  4,  4,  4,
                             5,  5,  6,  6,  6,  7,  7,  8,  8,  8,  9,  9,  10, 10, 11, 11, 11,
                             12, 12, 13, 13, 13, 14, 14, 15, 15, 16, 16, 16, 17, 17, 18, 18, 19,
                             19, 19, 20, 20, 21, 21, 22, 22, 22, 23, 23, 24, 24, 25};
  return m <= 64 ? t[m] : 0u;
}

// ---------------------------------------------------------------------------
// arithmetic
// ---------------------------------------------------------------------------
// splitmix64 output function (Steele, Lea, Flood, OOPSLA 2014)
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Tree shape (RecSplit, Sec. 2; fanouts Sec. 6): a node of m keys is a leaf
// when m <= n; otherwise its parts are (fanout - 1) x unit plus the remainder.
struct SplitShape {
  uint32_t unit, fanout;
};

__host__ __device__ __forceinline__ bool split_shape(uint32_t m, uint32_t n, SplitShape* s) {
  const uint32_t a1 = n > 24 ? 4 * n : 2 * n;
  const uint32_t a2 = n > 24 ? 12 * n : 4 * n;
  if (m <= n) return false;
  if (m <= a1) {
    s->unit = n;
    s->fanout = (m + n - 1) / n;
  } else if (m <= a2) {
    s->unit = a1;
    s->fanout = (m + a1 - 1) / a1;
  } else {
    s->unit = a2 * ((m + 2 * a2 - 1) / (2 * a2));
    s->fanout = 2;
  }
  return true;
}

__host__ __device__ __forceinline__ uint32_t part_size(uint32_t m, SplitShape s, uint32_t j) {
  return j + 1 < s.fanout ? s.unit : m - (s.fanout - 1) * s.unit;
}

// Rice parameter of a split node: k = floor(floor(log2 T) / 2) with
// T = floor(c_f prod(parts) / m), c_f = 3, 19, 119 for fanouts 2, 3, 4.
__host__ __device__ inline uint32_t rice_k_split(uint32_t m, uint32_t n) {
  SplitShape s;
  if (!split_shape(m, n, &s)) return 0;
  const uint64_t cf = s.fanout == 2 ? 3 : (s.fanout == 3 ? 19 : 119);
  uint64_t prod = 1;
  for (uint32_t j = 0; j < s.fanout; j++) prod *= part_size(m, s, j);
  const uint64_t t = cf * prod / m;
  if (t == 0) return 0;
#ifdef __CUDA_ARCH__
  const uint32_t lg = 63 - __clzll((long long)t);
#else
  const uint32_t lg = 63 - __builtin_clzll(t);
#endif
  return lg / 2;
}

// Leaf hash (Sec. 4; self-loops avoided): the two candidate cells of key x
// under seed constant c = mix(kLeafSalt + s) in a leaf of m >= 2 cells.
// a = (lo32(x) ^ lo32(c)) * (hi32(x) | 1) + hi32(c) mod 2^32; a * m gives h0
// (high word) and, from its low word r, t = floor(r (m-1) / 2^32) and
// h1 = t + (t >= h0).
__host__ __device__ __forceinline__ void leaf_cells(uint64_t x, uint64_t c, uint32_t m,
                                                    uint32_t* h0, uint32_t* h1) {
  const uint32_t a = ((uint32_t)x ^ (uint32_t)c) * ((uint32_t)(x >> 32) | 1u) + (uint32_t)(c >> 32);
  const uint64_t w = (uint64_t)a * m;
  const uint32_t u = (uint32_t)(w >> 32);
  const uint32_t t = (uint32_t)(((uint64_t)(uint32_t)w * (m - 1)) >> 32);
  *h0 = u;
  *h1 = t + (t >= u ? 1u : 0u);
}

// Rotation fitting (Sec. 4; partial hash calculation, App. A.2): the cells of
// key x under candidate v = s*m + r.  Keys of set A (top bit of
// mix(x ^ kRfSalt) clear) take the cells of seed s - (s mod 8) when m > 32, of
// seed s otherwise; keys of set B the cells of seed s moved by r (mod m).
__host__ __device__ __forceinline__ void rf_cells(uint64_t x, uint64_t v, uint32_t m,
                                                  uint32_t* h0, uint32_t* h1) {
  const uint64_t s = v / m;
  const uint32_t r = (uint32_t)(v - s * m);
  if ((mix64(x ^ kRfSalt) >> 63) == 0) {
    const uint64_t sa = m > 32 ? s - s % 8 : s;
    leaf_cells(x, mix64(kLeafSalt + sa), m, h0, h1);
  } else {
    leaf_cells(x, mix64(kLeafSalt + s), m, h0, h1);
    *h0 = *h0 + r >= m ? *h0 + r - m : *h0 + r;
    *h1 = *h1 + r >= m ? *h1 + r - m : *h1 + r;
  }
}

// Cells of a leaf key under its stored value (a seed, or v with rotation
// fitting).
__host__ __device__ __forceinline__ void value_cells(uint32_t leaf_mode, uint64_t x, uint64_t value,
                                                     uint32_t m, uint32_t* h0, uint32_t* h1) {
  if (leaf_mode)
    rf_cells(x, value, m, h0, h1);
  else
    leaf_cells(x, mix64(kLeafSalt + value), m, h0, h1);
}

// Retrieval row width w (paper Sec. 8.2: 128-bit words, 64 bits for n <= 24).
__host__ __device__ __forceinline__ uint32_t ribbon_width(uint32_t n) { return n > 24 ? 128u : 64u; }

// Defaults per width: shards of about 8,192 keys and eps = 5 % (w = 64),
// 12,288 keys and eps = 0.1 % (w = 128; the largest shards whose band fits a
// CTA's shared memory).
__host__ __device__ __forceinline__ uint32_t default_shard_buckets(uint32_t b, uint32_t w) {
  const uint32_t s = (w == 128 ? 12288u : 8192u) / b;
  return s ? s : 1u;
}

__host__ __device__ __forceinline__ uint32_t default_eps_num(uint32_t w) {
  return w == 128 ? kDefaultEpsNum128 : kDefaultEpsNum;
}

// Retrieval row of one key in a shard of m slots of width w with shard seed
// r: band start in [0, m - w] and the coefficient bits 0..63 (c0, bit 0 set)
// and 64..127 (c1; 0 for w = 64).
__host__ __device__ __forceinline__ void ribbon_row(uint64_t lo, uint64_t hi, uint32_t r,
                                                    uint64_t m, uint32_t w, uint64_t* start,
                                                    uint64_t* c0, uint64_t* c1) {
  const uint64_t t = mix64(hi ^ (kRetSalt + r));
  const uint64_t u = mix64(lo ^ t);
  *start = mulhi64(u, m - (w - 1));
  *c0 = mix64(u ^ kRetSalt2) | 1ull;
  *c1 = w == 128 ? mix64(u ^ kRetSalt3) : 0ull;
}

__host__ __device__ __forceinline__ uint64_t shard_slots(uint64_t keys, uint32_t eps_num, uint32_t w) {
  return keys ? keys + (keys * eps_num + 65535) / 65536 + (w - 1) : 0;
}

__host__ __device__ __forceinline__ uint32_t ef_low_bits(uint64_t U, uint64_t c) {
  const uint64_t q = U / c;
  if (q == 0) return 0;
#ifdef __CUDA_ARCH__
  return 63 - __clzll((long long)q);
#else
  return 63 - __builtin_clzll(q);
#endif
}

// ---------------------------------------------------------------------------
// leaf work description
// ---------------------------------------------------------------------------
struct LeafDesc {
  uint32_t key_off;   // first key of the leaf in leaf order
  uint32_t m;         // keys in the leaf (2..64 for searched leaves)
  uint32_t code_idx;  // slot of its seed in the code array (kNoCode if none)
  uint32_t bucket;
};

// ---------------------------------------------------------------------------
// host-side plumbing
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
shk_status fail(shk_status st, const std::string& msg);

// Runs f, turning a host-side exception (a failed host allocation, a thread
// that cannot start) into a status: no exception crosses the C ABI.
template <class F>
shk_status no_throw(F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return fail(SHK_ENOMEM, "host memory allocation failed");
  } catch (const std::exception& e) {
    return fail(SHK_ENOMEM, e.what());
  }
}

#define SHK_CUDA(call)                                                          \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess)                                                      \
      return ::shk::fail(SHK_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define SHK_TRY(expr)                    \
  do {                                   \
    shk_status s_ = (expr);              \
    if (s_ != SHK_OK) return s_;         \
  } while (0)

// Stream-ordered allocation from the library's memory pool of the current
// device (created on first use; it keeps freed memory for later calls).
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s);

// Stream-ordered device allocations that are released together.  It tracks
// at most kCap allocations; one more fails with SHK_ENOMEM (after returning
// the block it just took), so no allocation is ever left untracked.
struct Arena {
  static constexpr int kCap = 256;
  cudaStream_t stream;
  void* ptrs[kCap];
  int n = 0;
  explicit Arena(cudaStream_t s) : stream(s) {}
  ~Arena() {
    for (int i = 0; i < n; i++) cudaFreeAsync(ptrs[i], stream);
  }
  template <class T>
  shk_status alloc(T** p, size_t count, bool zero = false) {
    void* q = nullptr;
    size_t bytes = count ? count * sizeof(T) : 16;
    cudaError_t e = pool_malloc(&q, bytes, stream);
    if (e != cudaSuccess) return fail(SHK_ENOMEM, std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(e));
    if (n == kCap) {
      cudaFreeAsync(q, stream);
      return fail(SHK_ENOMEM, "internal: more than 256 working allocations in one call");
    }
    ptrs[n++] = q;
    if (zero) {
      e = cudaMemsetAsync(q, 0, bytes, stream);
      if (e != cudaSuccess) return fail(SHK_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    }
    *p = (T*)q;
    return SHK_OK;
  }
};

}  // namespace shk

// The MPHF object: the encoded words on the device plus decoded index arrays
// used by queries (not part of the encoded bits).
namespace shk {
// Query index: one record per code in preorder -- the code's value and, for a
// split node, the distance from its record to the first record of children
// 1..3 (child 0 follows at +1).
struct __align__(16) QNode {
  uint64_t seed;
  uint16_t child[3];
  uint16_t pad;
};
}  // namespace shk

struct shk_mphf {
  uint64_t hdr[shk::kHeaderWords];
  uint64_t words = 0;          // total u64 words of the encoded form
  uint64_t* d_blob = nullptr;  // device copy of the encoded form
  // section offsets in words
  uint64_t off_rice = 0, off_kl = 0, off_kh = 0, off_ol = 0, off_oh = 0, off_seed = 0,
           off_rib = 0;
  // decoded query support (device)
  uint32_t* d_K = nullptr;          // B + 1 key prefix sums
  uint64_t* d_O = nullptr;          // B + 1 Rice bit offsets
  uint64_t* d_shard_off = nullptr;  // num_shards + 1 slot offsets
  // query index, built by the first query (not part of the encoded form)
  shk::QNode* d_qnode = nullptr;  // one record per code
  uint32_t* d_qbase = nullptr;    // B + 1: first record of each bucket
  std::mutex qmu;
  shk_stats stats{};
  int device = 0;
};
