/*
 * shk_oracle.c -- CPU oracle for ShockHash-RS construction.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct CPU
 * implementation of what the paper's construction computes, written from its
 * definitions.  Only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  The CUDA library neither includes, links nor calls
 * anything here, and nothing here comes from the CUDA library.
 *
 * Paper: "ShockHash: Towards Optimal-Space Minimal Perfect Hashing Beyond
 * Brute-Force" (Lehmann, Sanders, Walzer).
 *
 * Where the paper fixes the result it is written out as that definition:
 *   - the leaf seed is the minimum seed whose 2-choice graph admits a
 *     1-orientation (Sec. 4, Eq. ShockHash), tested as "every connected
 *     component has at most as many edges as nodes" (Sec. 2, Pseudoforests);
 *   - the bit-mask filter is "every table cell is a candidate of some key"
 *     (Sec. 4, Filter by Bit Mask), a necessary condition only;
 *   - a split seed is the minimum seed giving the prescribed part sizes
 *     (Sec. 2, RecSplit);
 *   - rank(x) = prefix(bucket) + offset of the leaf + h_{s,f(x)}(x)
 *     (Sec. 1 prefix-sum form; Sec. 4 query).
 * Where the paper is silent (hash functions, tree shape above the two lowest
 * levels, Rice parameters, bit order, Elias-Fano layout, the retrieval
 * structure, which of the 2^c orientations to keep) the code follows the
 * project's frozen format readings; each function names its reading.
 *
 * Pins (tests/test_oracle_*.py): brute force over all graphs for m <= 6,
 * exact coverage probability (m up to 64), Fig. 2 trial counts (every row,
 * n = 6 .. 40), brute-force orientation, brute-force ribbon solutions, the
 * ribbon's success rate against random bands, Rice/EF round trips, bijection
 * of every build.  The hash functions are readings (the paper defines none);
 * each is pinned to something outside itself: the mixer to splitmix64's
 * published outputs, the string fingerprint to SipHash-2-4's published test
 * vector, and the leaf, split and retrieval hashes to the exact statistics of
 * the ideal random model they stand for.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

enum {
  ORC_OK = 0,
  ORC_EINVAL = 1,
  ORC_EDUPKEY = 2,
  ORC_ENOMEM = 3,
  ORC_ESEEDCAP = 5,
  ORC_EFORMAT = 7
};

enum { ORC_KEYS_U64 = 0, ORC_KEYS_STR = 1, ORC_KEYS_FP128 = 2 };

#define ORC_MAX_LEAF 64u
#define ORC_MAX_BUCKET_KEYS 8192u
#define ORC_MAX_BUCKET_SIZE 4096u
#define ORC_SEED_CAP (1ull << 40)
#define ORC_RIBBON_SEEDS 256u
#define ORC_HEADER_WORDS 16u
#define ORC_MAGIC 0x32303053524B4853ull /* "SHKRS002" */

/* Format constants: salts (hex digits of pi). */
#define FP_HI_SALT 0x243F6A8885A308D3ull
#define LEAF_SALT 0x13198A2E03707344ull
#define SPLIT_SALT 0xBE5466CF34E90C6Cull
#define RET_SALT 0xC0AC29B7C97C50DDull
#define RET_SALT2 0x3F84D5B5B5470917ull
#define RET_SALT3 0xA4093822299F31D0ull
#define STR_SALT_A 0x9216D5D98979FB1Bull
#define STR_SALT_B 0xD1310BA698DFB5ACull
#define RF_SALT 0x2FFD72DBD01ADFB7ull
#define RF_PARTIAL_K 8u  /* App. A.2: the first set keeps seed x - (x mod k), k = 8 */

/* Rice parameter of a leaf of m keys: floor(log2(ln2 * mu(m))) with mu(m) the
 * mean number of seeds tried, mu ~ 0.8 (e/2)^m e / sqrt(pi m) (the paper's
 * trial bound of Thm. shockHashConstruction divided by sqrt(m), as Sec. 8.1
 * observes).  Frozen as a literal format table; index 0 and 1 unused. */
static const uint8_t K_LEAF[65] = {
    0,  0,  0,  0,  0,  0,  1,  1,  1,  2,  2,  2,  3,  3,  4,  4,  4,
    5,  5,  6,  6,  6,  7,  7,  8,  8,  8,  9,  9,  10, 10, 11, 11, 11,
    12, 12, 13, 13, 13, 14, 14, 15, 15, 16, 16, 16, 17, 17, 18, 18, 19,
    19, 19, 20, 20, 21, 21, 22, 22, 22, 23, 23, 24, 24, 25};

/* ------------------------------------------------------------------------ */
/* Mixer: the splitmix64 output function (Steele, Lea, Flood, "Fast          */
/* splittable pseudorandom number generators", OOPSLA 2014).                 */
/* ------------------------------------------------------------------------ */
uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint64_t rotl64(uint64_t v, unsigned r) { return (v << r) | (v >> (64 - r)); }

/* ------------------------------------------------------------------------ */
/* Master hash code (Sec. 8: every key is first reduced to one high-quality  */
/* hash; all later hashes are functions of it).  128-bit fingerprint.        */
/* Reading: u64 key k -> (lo, hi) = (mix(k), mix(k ^ FP_HI_SALT)); mix is a   */
/* bijection, so distinct integer keys never share lo.                        */
/* ------------------------------------------------------------------------ */
void orc_fp_u64(const uint64_t* keys, uint64_t n, uint64_t* lo, uint64_t* hi) {
  for (uint64_t i = 0; i < n; i++) {
    lo[i] = orc_mix64(keys[i]);
    hi[i] = orc_mix64(keys[i] ^ FP_HI_SALT);
  }
}

/* ------------------------------------------------------------------------ */
/* SipHash-2-4 (Aumasson, Bernstein, "SipHash: a fast short-input PRF",      */
/* INDOCRYPT 2012): 64-bit output under the 128-bit key (k0, k1); the message */
/* is read as 8-byte little-endian words, the last block holding the tail     */
/* bytes and the length mod 256 in its top byte; 2 rounds per block, 4 to     */
/* finalize.  Written from the algorithm's description.                       */
/* ------------------------------------------------------------------------ */
static void sip_round(uint64_t v[4]) {
  v[0] += v[1]; v[1] = rotl64(v[1], 13); v[1] ^= v[0]; v[0] = rotl64(v[0], 32);
  v[2] += v[3]; v[3] = rotl64(v[3], 16); v[3] ^= v[2];
  v[0] += v[3]; v[3] = rotl64(v[3], 21); v[3] ^= v[0];
  v[2] += v[1]; v[1] = rotl64(v[1], 17); v[1] ^= v[2]; v[2] = rotl64(v[2], 32);
}

uint64_t orc_siphash24(uint64_t k0, uint64_t k1, const uint8_t* p, uint64_t len) {
  uint64_t v[4] = {k0 ^ 0x736f6d6570736575ull, k1 ^ 0x646f72616e646f6dull,
                   k0 ^ 0x6c7967656e657261ull, k1 ^ 0x7465646279746573ull};
  const uint64_t full = len / 8;
  for (uint64_t j = 0; j < full; j++) {
    uint64_t w = 0;
    for (unsigned t = 0; t < 8; t++) w |= (uint64_t)p[8 * j + t] << (8 * t);
    v[3] ^= w;
    sip_round(v);
    sip_round(v);
    v[0] ^= w;
  }
  uint64_t b = (len & 0xFF) << 56;
  for (uint64_t t = 0; t < len - 8 * full; t++) b |= (uint64_t)p[8 * full + t] << (8 * t);
  v[3] ^= b;
  sip_round(v);
  sip_round(v);
  v[0] ^= b;
  v[2] ^= 0xFF;
  for (int r = 0; r < 4; r++) sip_round(v);
  return v[0] ^ v[1] ^ v[2] ^ v[3];
}

/* Reading for byte-string keys: the two 64-bit halves of the fingerprint are
 * SipHash-2-4 of the key's bytes under two fixed keys,
 * lo = SipHash(STR_SALT_A, STR_SALT_B), hi = SipHash(STR_SALT_B, STR_SALT_A). */
void orc_fp_str(const uint8_t* bytes, const uint64_t* offs, uint64_t n, uint64_t* lo,
                uint64_t* hi) {
#pragma omp parallel for schedule(static)
  for (uint64_t i = 0; i < n; i++) {
    const uint8_t* p = bytes + offs[i];
    const uint64_t len = offs[i + 1] - offs[i];
    lo[i] = orc_siphash24(STR_SALT_A, STR_SALT_B, p, len);
    hi[i] = orc_siphash24(STR_SALT_B, STR_SALT_A, p, len);
  }
}

/* Bucket of a key (Sec. 2, RecSplit: keys are hashed to buckets of expected
 * size b).  Reading: B = ceil(N/b) buckets, bucket = floor(hi * B / 2^64). */
uint64_t orc_bucket(uint64_t hi, uint64_t B) { return (uint64_t)(((u128)hi * B) >> 64); }

/* The bucket of each of n keys (for tests of large builds). */
void orc_buckets(const uint64_t* hi, uint64_t n, uint64_t B, uint32_t* out) {
#pragma omp parallel for schedule(static)
  for (uint64_t i = 0; i < n; i++) out[i] = (uint32_t)orc_bucket(hi[i], B);
}

/* ------------------------------------------------------------------------ */
/* Splitting-tree shape (Sec. 2 RecSplit: the shape depends only on the      */
/* node size; Sec. 6 Fanouts: lowest split level 4, next 3 for n > 24, all 2 */
/* for n <= 24).  Reading for the remaining levels: binary splits whose left */
/* part is a multiple of the second-level size.                              */
/* Returns 0 for a leaf, else 1 with unit and fanout set; part j < fanout-1  */
/* has unit keys and the last part takes the remainder.                      */
/* ------------------------------------------------------------------------ */
int orc_split_shape(uint32_t m, uint32_t n, uint32_t* unit, uint32_t* fanout) {
  uint32_t a1 = n > 24 ? 4 * n : 2 * n;
  uint32_t a2 = n > 24 ? 12 * n : 4 * n;
  if (m <= n) return 0;
  if (m <= a1) {
    *unit = n;
    *fanout = (m + n - 1) / n;
  } else if (m <= a2) {
    *unit = a1;
    *fanout = (m + a1 - 1) / a1;
  } else {
    *unit = a2 * ((m + 2 * a2 - 1) / (2 * a2));
    *fanout = 2;
  }
  return 1;
}

static uint32_t part_size(uint32_t m, uint32_t unit, uint32_t fanout, uint32_t j) {
  return j + 1 < fanout ? unit : m - (fanout - 1) * unit;
}

/* Split hash (reading): g = mix(SPLIT_SALT + m), d = mix(g + s),
 * a = (hi32(x) ^ lo32(d)) * (lo32(x) | 1) + hi32(d) mod 2^32,
 * v = floor(a * m / 2^32); the child is the number of part boundaries
 * j*unit (1 <= j < fanout) that v has reached. */
uint32_t orc_split_child(uint64_t x, uint64_t seed, uint32_t m, uint32_t unit,
                         uint32_t fanout) {
  uint64_t g = orc_mix64(SPLIT_SALT + m);
  uint64_t d = orc_mix64(g + seed);
  uint32_t a = ((uint32_t)(x >> 32) ^ (uint32_t)d) * ((uint32_t)x | 1u) + (uint32_t)(d >> 32);
  uint32_t v = (uint32_t)(((uint64_t)a * m) >> 32);
  uint32_t child = 0;
  for (uint32_t j = 1; j < fanout; j++)
    if (v >= j * unit) child++;
  return child;
}

/* Split seed: the smallest seed whose split hash sends exactly the prescribed
 * number of keys to every child (Sec. 2, RecSplit). */
int orc_split_seed(const uint64_t* x, uint32_t m, uint32_t n, uint64_t* seed_out) {
  uint32_t unit, fan;
  if (!orc_split_shape(m, n, &unit, &fan)) return ORC_EINVAL;
  for (uint64_t s = 0; s < ORC_SEED_CAP; s++) {
    uint32_t cnt[4] = {0, 0, 0, 0};
    for (uint32_t i = 0; i < m; i++) cnt[orc_split_child(x[i], s, m, unit, fan)]++;
    int ok = 1;
    for (uint32_t j = 0; j < fan; j++)
      if (cnt[j] != part_size(m, unit, fan, j)) ok = 0;
    if (ok) {
      *seed_out = s;
      return ORC_OK;
    }
  }
  return ORC_ESEEDCAP;
}

/* Rice parameter of a split node (reading): the expected number of trials of
 * a split into parts p_j is about sqrt((2 pi)^(f-1) prod p_j / m) (Stirling on
 * the multinomial success probability); k = floor(log2(ln2 * trials)) is taken
 * as floor(floor(log2 T) / 2) with the integer T = floor(c_f prod p_j / m) and
 * c_f = round((2 pi)^(f-1) ln^2 2) = 3, 19, 119 for f = 2, 3, 4. */
uint32_t orc_rice_k_split(uint32_t m, uint32_t n) {
  uint32_t unit, fan;
  if (!orc_split_shape(m, n, &unit, &fan)) return 0;
  static const uint64_t cf[5] = {0, 0, 3, 19, 119};
  uint64_t prod = 1;
  for (uint32_t j = 0; j < fan; j++) prod *= part_size(m, unit, fan, j);
  uint64_t t = cf[fan] * prod / m;
  if (t == 0) return 0;
  uint32_t lg = 63 - (uint32_t)__builtin_clzll(t);
  return lg / 2;
}

uint32_t orc_rice_k_leaf(uint32_t m) { return m >= 2 && m <= 64 ? K_LEAF[m] : 0; }

/* ------------------------------------------------------------------------ */
/* Leaf hash (Sec. 4: key x gets candidate cells h_{s,0}(x), h_{s,1}(x) in   */
/* [m]; footnote in Sec. 5: self-loops are avoided).  Reading:               */
/*   c = mix(LEAF_SALT + s);                                                  */
/*   a = (lo32(x) ^ lo32(c)) * (hi32(x) | 1) + hi32(c)  mod 2^32;              */
/*   h0 = floor(a * m / 2^32);  r = a * m mod 2^32;                            */
/*   t = floor(r * (m-1) / 2^32);  h1 = t + (t >= h0)                          */
/* -- h0 uniform over [m], h1 uniform over the other m-1 cells.               */
/* ------------------------------------------------------------------------ */
void orc_leaf_hash(uint64_t x, uint64_t seed, uint32_t m, uint32_t* h0, uint32_t* h1) {
  uint64_t c = orc_mix64(LEAF_SALT + seed);
  uint32_t y = (uint32_t)x ^ (uint32_t)c;
  uint32_t mult = (uint32_t)(x >> 32) | 1u;
  uint32_t a = y * mult + (uint32_t)(c >> 32);
  uint64_t w = (uint64_t)a * m;
  uint32_t u = (uint32_t)(w >> 32);
  uint32_t t = (uint32_t)(((uint64_t)(uint32_t)w * (m - 1)) >> 32);
  *h0 = u;
  *h1 = t + (t >= u ? 1u : 0u);
}

/* Pseudoforest test (Sec. 2, Pseudoforests: a 1-orientation exists iff every
 * connected component has at most as many edges as nodes).  Components are
 * found by relaxing labels along edges until every edge joins equal labels. */
int orc_is_pseudoforest(const uint32_t* h0, const uint32_t* h1, uint32_t m) {
  uint32_t label[ORC_MAX_LEAF], nodes[ORC_MAX_LEAF], edges[ORC_MAX_LEAF];
  for (uint32_t v = 0; v < m; v++) label[v] = v;
  int changed = 1;
  while (changed) {
    changed = 0;
    for (uint32_t e = 0; e < m; e++) {
      uint32_t a = label[h0[e]], b = label[h1[e]];
      if (a != b) {
        uint32_t lo = a < b ? a : b;
        label[h0[e]] = lo;
        label[h1[e]] = lo;
        changed = 1;
      }
    }
  }
  for (uint32_t v = 0; v < m; v++) nodes[v] = edges[v] = 0;
  for (uint32_t v = 0; v < m; v++) nodes[label[v]]++;
  for (uint32_t e = 0; e < m; e++) edges[label[h0[e]]]++;
  for (uint32_t v = 0; v < m; v++)
    if (edges[v] > nodes[v]) return 0;
  return 1;
}

/* Bit-mask filter (Sec. 4, Filter by Bit Mask): every cell is a candidate of
 * some key. */
int orc_covers_all(const uint32_t* h0, const uint32_t* h1, uint32_t m) {
  uint64_t mask = 0;
  for (uint32_t e = 0; e < m; e++) mask |= (1ull << h0[e]) | (1ull << h1[e]);
  uint64_t full = m == 64 ? ~0ull : ((1ull << m) - 1);
  return mask == full;
}

/* Batch form of the two tests above for enumerations in the pins: graph g
 * has edges {h0[g*m+e], h1[g*m+e]}, e < m. */
void orc_pf_batch(const uint32_t* h0, const uint32_t* h1, uint64_t count, uint32_t m,
                  uint8_t* pf, uint8_t* cov) {
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < (int64_t)count; g++) {
    pf[g] = (uint8_t)orc_is_pseudoforest(h0 + g * m, h1 + g * m, m);
    cov[g] = (uint8_t)orc_covers_all(h0 + g * m, h1 + g * m, m);
  }
}

/* Leaf seed (Sec. 4, Eq. ShockHash): the smallest s >= start such that some
 * f makes x -> h_{s,f(x)}(x) a bijection onto [m], i.e. the graph
 * ([m], {{h0(x), h1(x)}}) is a pseudoforest.  The filter only skips seeds
 * that cannot pass; use_filter = 0 tests every seed in full. */
int orc_leaf_seed(const uint64_t* x, uint32_t m, uint64_t start, uint64_t cap, int use_filter,
                  uint64_t* seed_out) {
  uint32_t h0[ORC_MAX_LEAF], h1[ORC_MAX_LEAF];
  if (m < 2 || m > ORC_MAX_LEAF) return ORC_EINVAL;
  for (uint64_t s = start; s < cap; s++) {
    for (uint32_t i = 0; i < m; i++) orc_leaf_hash(x[i], s, m, &h0[i], &h1[i]);
    if (use_filter && !orc_covers_all(h0, h1, m)) continue;
    if (orc_is_pseudoforest(h0, h1, m)) {
      *seed_out = s;
      return ORC_OK;
    }
  }
  return ORC_ESEEDCAP;
}

/* ------------------------------------------------------------------------ */
/* Rotation fitting (Sec. 4, Rotation Fitting) with partial hash calculation */
/* (App. A.2).  Reading: a fixed 1-bit hash puts key x in set B when        */
/* mix(x ^ RF_SALT) has its top bit set, else in set A.  Candidate v = s*m+r */
/* (seed s, rotation r in [0, m)): keys of A take the cells of seed s_A,     */
/* keys of B the cells of seed s moved by r (mod m) -- the cyclic rotation  */
/* of B's bit mask.  s_A = s - (s mod 8) for leaves of more than 32 keys    */
/* (the first set is hashed with a seed fixed over 8 consecutive seeds),    */
/* s_A = s otherwise.  The leaf value is the smallest pseudoforest v.       */
/* ------------------------------------------------------------------------ */
int orc_rf_set(uint64_t x) { return (int)(orc_mix64(x ^ RF_SALT) >> 63); }

void orc_rf_cells(uint64_t x, uint64_t v, uint32_t m, uint32_t* h0, uint32_t* h1) {
  uint64_t s = v / m, r = v % m;
  if (!orc_rf_set(x)) {
    uint64_t sa = m > 32 ? s - s % RF_PARTIAL_K : s;
    orc_leaf_hash(x, sa, m, h0, h1);
  } else {
    orc_leaf_hash(x, s, m, h0, h1);
    *h0 = (uint32_t)((*h0 + r) % m);
    *h1 = (uint32_t)((*h1 + r) % m);
  }
}

/* The rotation-fitting search in the paper's order (Sec. 4, Rotation
 * Fitting): the keys are split into the two sets once; for each seed s both
 * sets are hashed (set A with its partial seed, App. A.2); then for each
 * rotation r = 0 .. m-1 the cells of set B are moved by r and the candidate
 * v = s*m + r is tested (filter, then pseudoforest).  Candidates are visited
 * in increasing v, so the first that passes is the minimum; the cells of
 * every candidate are those orc_rf_cells gives. */
int orc_rf_value(const uint64_t* x, uint32_t m, uint64_t start, uint64_t cap, int use_filter,
                 uint64_t* v_out) {
  uint32_t a0[ORC_MAX_LEAF], a1[ORC_MAX_LEAF], h0[ORC_MAX_LEAF], h1[ORC_MAX_LEAF];
  int in_b[ORC_MAX_LEAF];
  if (m < 2 || m > ORC_MAX_LEAF) return ORC_EINVAL;
  for (uint32_t i = 0; i < m; i++) in_b[i] = orc_rf_set(x[i]);
  for (uint64_t s = start / m; s * m < cap; s++) {
    const uint64_t sa = m > 32 ? s - s % RF_PARTIAL_K : s;
    for (uint32_t i = 0; i < m; i++) orc_leaf_hash(x[i], in_b[i] ? s : sa, m, &a0[i], &a1[i]);
    for (uint32_t r = 0; r < m; r++) {
      const uint64_t v = s * m + r;
      if (v < start) continue;
      if (v >= cap) break;
      for (uint32_t i = 0; i < m; i++) {  /* B's cells moved by r, mod m */
        h0[i] = in_b[i] ? (a0[i] + r >= m ? a0[i] + r - m : a0[i] + r) : a0[i];
        h1[i] = in_b[i] ? (a1[i] + r >= m ? a1[i] + r - m : a1[i] + r) : a1[i];
      }
      if (use_filter && !orc_covers_all(h0, h1, m)) continue;
      if (orc_is_pseudoforest(h0, h1, m)) {
        *v_out = v;
        return ORC_OK;
      }
    }
  }
  return ORC_ESEEDCAP;
}

/* Over seeds s0 .. s0+count-1 of one leaf: how many pass the filter and how
 * many give a pseudoforest (for the filter-rate and trial-count pins). */
void orc_leaf_seed_stats(const uint64_t* x, uint32_t m, uint64_t s0, uint64_t count,
                         uint64_t* n_cov, uint64_t* n_pf) {
  uint32_t h0[ORC_MAX_LEAF], h1[ORC_MAX_LEAF];
  uint64_t c = 0, p = 0;
  for (uint64_t s = s0; s < s0 + count; s++) {
    for (uint32_t i = 0; i < m; i++) orc_leaf_hash(x[i], s, m, &h0[i], &h1[i]);
    if (orc_covers_all(h0, h1, m)) {
      c++;
      p += (uint64_t)orc_is_pseudoforest(h0, h1, m);
    }
  }
  *n_cov = c;
  *n_pf = p;
}

/* ------------------------------------------------------------------------ */
/* Orientation.  A pseudoforest has 2^c 1-orientations (Sec. 5, Eq.          */
/* orientations-cycles).  Reading: keep the lexicographically smallest f     */
/* (key 0 first, f = 0 meaning cell h0).  Written as the definition: fix     */
/* f(0), f(1), ... greedily to 0 whenever a bijection still exists, checked  */
/* by bipartite matching with augmenting paths.                              */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t m;
  const uint32_t* h0;
  const uint32_t* h1;
  const int* fixed; /* -1 free, 0 or 1 fixed */
  int owner[ORC_MAX_LEAF];
  uint8_t seen[ORC_MAX_LEAF];
} matching_t;

static int try_key(matching_t* mt, uint32_t key) {
  uint32_t cand[2];
  int nc = 0;
  if (mt->fixed[key] != 1) cand[nc++] = mt->h0[key];
  if (mt->fixed[key] != 0) cand[nc++] = mt->h1[key];
  for (int i = 0; i < nc; i++) {
    uint32_t c = cand[i];
    if (mt->seen[c]) continue;
    mt->seen[c] = 1;
    if (mt->owner[c] < 0 || try_key(mt, (uint32_t)mt->owner[c])) {
      mt->owner[c] = (int)key;
      return 1;
    }
  }
  return 0;
}

static int bijection_exists(uint32_t m, const uint32_t* h0, const uint32_t* h1, const int* fixed) {
  matching_t mt;
  mt.m = m;
  mt.h0 = h0;
  mt.h1 = h1;
  mt.fixed = fixed;
  for (uint32_t c = 0; c < m; c++) mt.owner[c] = -1;
  for (uint32_t k = 0; k < m; k++) {
    memset(mt.seen, 0, sizeof mt.seen);
    if (!try_key(&mt, k)) return 0;
  }
  return 1;
}

static int orient_cells(const uint32_t* h0, const uint32_t* h1, uint32_t m, uint8_t* f) {
  int fixed[ORC_MAX_LEAF];
  for (uint32_t i = 0; i < m; i++) fixed[i] = -1;
  if (!bijection_exists(m, h0, h1, fixed)) return ORC_EINVAL;
  for (uint32_t i = 0; i < m; i++) {
    fixed[i] = 0;
    if (!bijection_exists(m, h0, h1, fixed)) fixed[i] = 1;
    f[i] = (uint8_t)fixed[i];
  }
  return ORC_OK;
}

/* The leaf's cells under its stored value: a seed (plain) or v (rotation
 * fitting). */
static void leaf_cells_mode(int rf, uint64_t x, uint64_t value, uint32_t m, uint32_t* h0,
                            uint32_t* h1) {
  if (rf)
    orc_rf_cells(x, value, m, h0, h1);
  else
    orc_leaf_hash(x, value, m, h0, h1);
}

int orc_orient_mode(int rf, const uint64_t* x, uint32_t m, uint64_t value, uint8_t* f) {
  uint32_t h0[ORC_MAX_LEAF], h1[ORC_MAX_LEAF];
  if (m == 1) {
    f[0] = 0;
    return ORC_OK;
  }
  if (m < 2 || m > ORC_MAX_LEAF) return ORC_EINVAL;
  for (uint32_t i = 0; i < m; i++) leaf_cells_mode(rf, x[i], value, m, &h0[i], &h1[i]);
  return orient_cells(h0, h1, m, f);
}

int orc_orient(const uint64_t* x, uint32_t m, uint64_t seed, uint8_t* f) {
  return orc_orient_mode(0, x, m, seed, f);
}

/* Batched leaf search over independent leaves (same definitions as above):
 * leaf i holds x[leaf_off[i] .. leaf_off[i+1]).  f_mask bit j = f of key j. */
int orc_leaf_search_batch(const uint64_t* x, const uint32_t* leaf_off, uint32_t n_leaves,
                          uint64_t seed_start, uint64_t* seeds_out, uint64_t* f_mask,
                          int nthreads, int rf) {
  int status = ORC_OK;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < (int64_t)n_leaves; i++) {
    uint32_t m = leaf_off[i + 1] - leaf_off[i];
    uint64_t s = 0;
    uint8_t f[ORC_MAX_LEAF];
    int st = ORC_OK;
    if (m == 0 || m > ORC_MAX_LEAF) {
      st = ORC_EINVAL;
    } else if (m == 1) { /* one key: no hash, any seed works; the first is seed_start */
      s = seed_start;
      f[0] = 0;
    } else {
      if (rf)
        st = orc_rf_value(x + leaf_off[i], m, seed_start, ORC_SEED_CAP, 1, &s);
      else
        st = orc_leaf_seed(x + leaf_off[i], m, seed_start, ORC_SEED_CAP, 1, &s);
      if (st == ORC_OK) st = orc_orient_mode(rf, x + leaf_off[i], m, s, f);
    }
    if (st != ORC_OK) {
#pragma omp critical
      status = st;
      continue;
    }
    seeds_out[i] = s;
    if (f_mask) {
      uint64_t mk = 0;
      for (uint32_t j = 0; j < m; j++) mk |= (uint64_t)f[j] << j;
      f_mask[i] = mk;
    }
  }
  return status;
}

/* ------------------------------------------------------------------------ */
/* Bit vectors, LSB-first: bit p lives in bit (p mod 64) of word p / 64.      */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint64_t* w;
  uint64_t nbits;
  uint64_t cap; /* words */
} bitvec_t;

static int bv_reserve(bitvec_t* bv, uint64_t nbits) {
  uint64_t need = (nbits + 63) / 64 + 1;
  if (need <= bv->cap) return 1;
  uint64_t cap = bv->cap ? bv->cap : 16;
  while (cap < need) cap *= 2;
  uint64_t* w = (uint64_t*)realloc(bv->w, cap * 8);
  if (!w) return 0;
  memset(w + bv->cap, 0, (cap - bv->cap) * 8);
  bv->w = w;
  bv->cap = cap;
  return 1;
}

static int bv_push_bit(bitvec_t* bv, int bit) {
  if (!bv_reserve(bv, bv->nbits + 1)) return 0;
  if (bit) bv->w[bv->nbits / 64] |= 1ull << (bv->nbits % 64);
  bv->nbits++;
  return 1;
}

static int bv_push_bits(bitvec_t* bv, uint64_t v, uint32_t nbits) {
  for (uint32_t j = 0; j < nbits; j++)
    if (!bv_push_bit(bv, (int)((v >> j) & 1))) return 0;
  return 1;
}

static int get_bit(const uint64_t* w, uint64_t p) { return (int)((w[p / 64] >> (p % 64)) & 1); }

static uint64_t get_bits(const uint64_t* w, uint64_t p, uint32_t nbits) {
  uint64_t v = 0;
  for (uint32_t j = 0; j < nbits; j++) v |= (uint64_t)get_bit(w, p + j) << j;
  return v;
}

/* Golomb-Rice code (Sec. 4: the seed is stored with Golomb-Rice codes).
 * Reading: the k low bits of s LSB-first, then q = s >> k one-bits and a
 * terminating zero-bit. */
static int rice_put(bitvec_t* bv, uint64_t s, uint32_t k) {
  if (!bv_push_bits(bv, s, k)) return 0;
  for (uint64_t q = s >> k; q > 0; q--)
    if (!bv_push_bit(bv, 1)) return 0;
  return bv_push_bit(bv, 0);
}

static uint64_t rice_get(const uint64_t* w, uint64_t* pos, uint32_t k) {
  uint64_t low = get_bits(w, *pos, k);
  *pos += k;
  uint64_t q = 0;
  while (get_bit(w, *pos)) {
    q++;
    (*pos)++;
  }
  (*pos)++;
  return (q << k) | low;
}

/* ------------------------------------------------------------------------ */
/* One bucket: the splitting tree in depth-first preorder (Sec. 2 RecSplit). */
/* Keys are (lo, hi) fingerprints in ascending order; children take their    */
/* keys by stable partition so every leaf stays in ascending order.          */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint64_t* seed;
  uint8_t* k;
  uint32_t n, cap;
} codes_t;

static int codes_push(codes_t* c, uint64_t seed, uint32_t k) {
  if (c->n == c->cap) {
    uint32_t cap = c->cap ? 2 * c->cap : 64;
    uint64_t* s = (uint64_t*)realloc(c->seed, cap * 8);
    if (!s) return 0;
    c->seed = s;
    uint8_t* kk = (uint8_t*)realloc(c->k, cap);
    if (!kk) return 0;
    c->k = kk;
    c->cap = cap;
  }
  c->seed[c->n] = seed;
  c->k[c->n] = (uint8_t)k;
  c->n++;
  return 1;
}

/* Leaves of a bucket, recorded instead of searched (splits-only mode). */
typedef struct {
  uint32_t* off;
  uint32_t* m;
  uint32_t cap, n;
} leafrec_t;

static int build_node(uint64_t* lo, uint64_t* hi, uint8_t* f, uint32_t m, uint32_t n,
                      codes_t* codes, uint64_t* tlo, uint64_t* thi, int rf, leafrec_t* lr,
                      uint32_t base) {
  uint32_t unit, fan;
  if (!orc_split_shape(m, n, &unit, &fan)) {
    if (m == 1) {
      f[0] = 0;
      return ORC_OK;
    }
    if (lr) {
      /* splits only: the leaf's code slot holds a marker, its keys stay put */
      if (lr->n >= lr->cap) return ORC_EINVAL;
      lr->off[lr->n] = base;
      lr->m[lr->n] = m;
      lr->n++;
      return codes_push(codes, ~0ull, orc_rice_k_leaf(m)) ? ORC_OK : ORC_ENOMEM;
    }
    uint64_t s;
    int st = rf ? orc_rf_value(lo, m, 0, ORC_SEED_CAP, 1, &s)
                : orc_leaf_seed(lo, m, 0, ORC_SEED_CAP, 1, &s);
    if (st != ORC_OK) return st;
    if (!codes_push(codes, s, orc_rice_k_leaf(m))) return ORC_ENOMEM;
    return orc_orient_mode(rf, lo, m, s, f);
  }
  uint64_t s;
  int st = orc_split_seed(lo, m, n, &s);
  if (st != ORC_OK) return st;
  if (!codes_push(codes, s, orc_rice_k_split(m, n))) return ORC_ENOMEM;
  /* stable partition by child */
  uint32_t pos = 0;
  for (uint32_t j = 0; j < fan; j++)
    for (uint32_t i = 0; i < m; i++)
      if (orc_split_child(lo[i], s, m, unit, fan) == j) {
        tlo[pos] = lo[i];
        thi[pos] = hi[i];
        pos++;
      }
  memcpy(lo, tlo, (size_t)m * 8);
  memcpy(hi, thi, (size_t)m * 8);
  uint32_t off = 0;
  for (uint32_t j = 0; j < fan; j++) {
    uint32_t p = part_size(m, unit, fan, j);
    st = build_node(lo + off, hi + off, f + off, p, n, codes, tlo, thi, rf, lr, base + off);
    if (st != ORC_OK) return st;
    off += p;
  }
  return ORC_OK;
}

/* Bucket-level entry point for sampled parity: keys sorted ascending on
 * input, reordered into leaf order on output; codes in preorder. */
int orc_bucket_build(uint64_t* lo, uint64_t* hi, uint32_t size, uint32_t n, uint64_t* seeds,
                     uint8_t* ks, uint32_t cap, uint32_t* ncodes, uint8_t* f, int rf) {
  if (size == 0) {
    *ncodes = 0;
    return ORC_OK;
  }
  codes_t c = {0};
  uint64_t* tlo = (uint64_t*)malloc((size_t)size * 8);
  uint64_t* thi = (uint64_t*)malloc((size_t)size * 8);
  int st = (tlo && thi) ? build_node(lo, hi, f, size, n, &c, tlo, thi, rf, NULL, 0) : ORC_ENOMEM;
  if (st == ORC_OK) {
    if (c.n > cap) st = ORC_EINVAL;
    else {
      memcpy(seeds, c.seed, (size_t)c.n * 8);
      memcpy(ks, c.k, c.n);
      *ncodes = c.n;
    }
  }
  free(tlo);
  free(thi);
  free(c.seed);
  free(c.k);
  return st;
}

/* The splitting tree of one bucket without the leaf searches: codes in
 * preorder with all-ones in the leaf slots, keys reordered into leaf order,
 * and each leaf's (offset, size) for leaves of two or more keys, in order. */
int orc_bucket_splits(uint64_t* lo, uint64_t* hi, uint32_t size, uint32_t n, uint64_t* seeds,
                      uint8_t* ks, uint32_t cap, uint32_t* ncodes, uint32_t* leaf_off,
                      uint32_t* leaf_m, uint32_t leaf_cap, uint32_t* nleaves) {
  *ncodes = 0;
  *nleaves = 0;
  if (size == 0) return ORC_OK;
  codes_t c = {0};
  leafrec_t lr = {leaf_off, leaf_m, leaf_cap, 0};
  uint8_t* f = (uint8_t*)malloc(size);
  uint64_t* tlo = (uint64_t*)malloc((size_t)size * 8);
  uint64_t* thi = (uint64_t*)malloc((size_t)size * 8);
  int st = (f && tlo && thi) ? build_node(lo, hi, f, size, n, &c, tlo, thi, 0, &lr, 0) : ORC_ENOMEM;
  if (st == ORC_OK) {
    if (c.n > cap) st = ORC_EINVAL;
    else {
      memcpy(seeds, c.seed, (size_t)c.n * 8);
      memcpy(ks, c.k, c.n);
      *ncodes = c.n;
      *nleaves = lr.n;
    }
  }
  free(f);
  free(tlo);
  free(thi);
  free(c.seed);
  free(c.k);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Elias-Fano (reading of the prefix-sum index of Sec. 1): for v_0..v_{c-1}  */
/* nondecreasing with U = v_{c-1}: l = floor(log2(U / c)) (0 if U < c); low  */
/* part = c fields of l bits; high part sets bit (v_i >> l) + i in a vector  */
/* of (U >> l) + c bits.                                                     */
/* ------------------------------------------------------------------------ */
static uint32_t ef_l(uint64_t U, uint64_t c) {
  uint64_t q = U / c;
  if (q == 0) return 0;
  return 63 - (uint32_t)__builtin_clzll(q);
}

static int ef_encode(const uint64_t* v, uint64_t c, bitvec_t* low, bitvec_t* high, uint32_t* l_out) {
  uint64_t U = v[c - 1];
  uint32_t l = ef_l(U, c);
  for (uint64_t i = 0; i < c; i++)
    if (!bv_push_bits(low, v[i], l)) return 0;
  uint64_t hb = (U >> l) + c;
  if (!bv_reserve(high, hb)) return 0;
  high->nbits = hb;
  for (uint64_t i = 0; i < c; i++) {
    uint64_t p = (v[i] >> l) + i;
    high->w[p / 64] |= 1ull << (p % 64);
  }
  *l_out = l;
  return 1;
}

static void ef_decode_all(const uint64_t* low, const uint64_t* high, uint64_t hbits, uint32_t l,
                          uint64_t c, uint64_t* v) {
  uint64_t i = 0;
  for (uint64_t p = 0; p < hbits && i < c; p++)
    if (get_bit(high, p)) {
      v[i] = ((p - i) << l) | get_bits(low, i * l, l);
      i++;
    }
}

/* ------------------------------------------------------------------------ */
/* 1-bit retrieval (Sec. 2 Retrieval; Sec. 6: all f bits go into one          */
/* retrieval structure; Sec. 8.2: 128-bit words, 64 bits for n <= 24).       */
/* Reading: a standard ribbon of width w (128 for n > 24, else 64), sharded  */
/* by runs of shard_buckets buckets.  Shard slots m = keys + ceil(keys * eps */
/* / 2^16) + w - 1 (0 for an empty shard).  Key equation with shard seed r:  */
/*   t = mix(hi ^ (RET_SALT + r)), u = mix(lo ^ t),                          */
/*   start = floor(u * (m - w + 1) / 2^64), coeff bits 0..63 =               */
/*   mix(u ^ RET_SALT2) | 1, bits 64..127 = mix(u ^ RET_SALT3) (w = 128),     */
/*   parity(coeff & sol[start .. start + w - 1]) = f(x).                      */
/* r is the smallest seed in [0, 256) giving a consistent system; the stored */
/* solution is the unique one that is zero on every non-pivot column, pivots */
/* being the lowest set column of each echelon row.                          */
/* ------------------------------------------------------------------------ */
/* Ribbon width (Sec. 8.2: BuRR with 128-bit words, 64 bits for n <= 24). */
uint32_t orc_ribbon_width(uint32_t n) { return n > 24 ? 128u : 64u; }

static uint64_t shard_slots(uint64_t keys, uint32_t eps_num, uint32_t w) {
  if (keys == 0) return 0;
  return keys + (keys * eps_num + 65535) / 65536 + (w - 1);
}

/* Row of one key: band start in [0, m - w] and a w-bit coefficient with bit
 * 0 set (w = 64: the low word only). */
static void ribbon_row(uint64_t lo, uint64_t hi, uint32_t r, uint64_t m, uint32_t w,
                       uint64_t* start, u128* coeff) {
  uint64_t t = orc_mix64(hi ^ (RET_SALT + r));
  uint64_t u = orc_mix64(lo ^ t);
  *start = (uint64_t)(((u128)u * (m - (w - 1))) >> 64);
  uint64_t c0 = orc_mix64(u ^ RET_SALT2) | 1ull;
  uint64_t c1 = w == 128 ? orc_mix64(u ^ RET_SALT3) : 0;
  *coeff = ((u128)c1 << 64) | c0;
}

/* The rows of n keys under shard seed r in a shard of m slots (for tests). */
void orc_ribbon_rows(const uint64_t* lo, const uint64_t* hi, uint64_t n, uint32_t r, uint64_t m,
                     uint32_t w, uint64_t* start, uint64_t* coeff_lo, uint64_t* coeff_hi) {
  for (uint64_t i = 0; i < n; i++) {
    u128 c;
    ribbon_row(lo[i], hi[i], r, m, w, &start[i], &c);
    coeff_lo[i] = (uint64_t)c;
    coeff_hi[i] = (uint64_t)(c >> 64);
  }
}

static unsigned ctz128(u128 v) {
  uint64_t lo = (uint64_t)v;
  return lo ? (unsigned)__builtin_ctzll(lo) : 64u + (unsigned)__builtin_ctzll((uint64_t)(v >> 64));
}

/* Gaussian elimination restricted to the band: a row is reduced by the row
 * stored at its lowest set column until it finds a free column (new pivot) or
 * vanishes (consistent if its right-hand side vanishes too).  Back
 * substitution then fills pivot columns from the top, free columns = 0. */
static int ribbon_solve_shard(const uint64_t* lo, const uint64_t* hi, const uint8_t* f,
                              uint64_t keys, uint64_t m, uint32_t w, uint32_t r, u128* rows,
                              uint8_t* rhs, uint8_t* sol) {
  memset(rows, 0, (size_t)m * sizeof(u128));
  memset(rhs, 0, (size_t)m);
  for (uint64_t i = 0; i < keys; i++) {
    uint64_t st;
    u128 c;
    ribbon_row(lo[i], hi[i], r, m, w, &st, &c);
    uint8_t b = f[i];
    for (;;) {
      if (rows[st] == 0) {
        rows[st] = c;
        rhs[st] = b;
        break;
      }
      c ^= rows[st];
      b ^= rhs[st];
      if (c == 0) {
        if (b) return 0;
        break;
      }
      unsigned tz = ctz128(c);
      c >>= tz;
      st += tz;
    }
  }
  for (uint64_t ii = m; ii-- > 0;) {
    if (rows[ii] == 0) {
      sol[ii] = 0;
      continue;
    }
    uint8_t b = rhs[ii];
    for (uint32_t j = 1; j < w; j++)
      if ((rows[ii] >> j) & 1) b ^= sol[ii + j];
    sol[ii] = b;
  }
  return 1;
}

/* Solve one shard: smallest consistent seed, canonical solution bits. */
int orc_ribbon_shard(const uint64_t* lo, const uint64_t* hi, const uint8_t* f, uint64_t keys,
                     uint32_t eps_num, uint32_t w, uint32_t* seed_out, uint8_t* sol /* shard_slots */) {
  uint64_t m = shard_slots(keys, eps_num, w);
  if (m == 0) {
    *seed_out = 0;
    return ORC_OK;
  }
  u128* rows = (u128*)malloc((size_t)m * sizeof(u128));
  uint8_t* rhs = (uint8_t*)malloc((size_t)m);
  if (!rows || !rhs) {
    free(rows);
    free(rhs);
    return ORC_ENOMEM;
  }
  int st = ORC_ESEEDCAP;
  for (uint32_t r = 0; r < ORC_RIBBON_SEEDS; r++)
    if (ribbon_solve_shard(lo, hi, f, keys, m, w, r, rows, rhs, sol)) {
      *seed_out = r;
      st = ORC_OK;
      break;
    }
  free(rows);
  free(rhs);
  return st;
}

uint64_t orc_shard_slots(uint64_t keys, uint32_t eps_num, uint32_t w) {
  return shard_slots(keys, eps_num, w);
}

/* ------------------------------------------------------------------------ */
/* Whole build.                                                              */
/* ------------------------------------------------------------------------ */
static int cmp_fp(const void* a, const void* b) {
  const uint64_t* x = (const uint64_t*)a;
  const uint64_t* y = (const uint64_t*)b;
  if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1; /* hi first */
  if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
  return 0;
}

static void put_words(uint8_t* out, uint64_t* pos_words, const uint64_t* w, uint64_t nwords) {
  if (nwords) memcpy(out + *pos_words * 8, w, (size_t)nwords * 8);
  *pos_words += nwords;
}

/* Retrieval defaults per ribbon width: shards of about 8,192 keys and
 * eps = 5 % (w = 64), 12,288 keys and eps = 0.1 % (w = 128). */
uint32_t orc_default_shard_buckets(uint32_t b, uint32_t w) {
  uint32_t s = (w == 128 ? 12288u : 8192u) / b;
  return s ? s : 1u;
}

uint32_t orc_default_eps_num(uint32_t w) { return w == 128 ? 66u : 3277u; }

int orc_build(int kind, const void* data, const uint64_t* offs, uint64_t N, uint32_t n,
              uint32_t b, uint32_t shard_buckets, uint32_t eps_num, int nthreads, int leaf_mode,
              uint8_t** out, uint64_t* out_len) {
  *out = NULL;
  *out_len = 0;
  if (n < 2 || n > ORC_MAX_LEAF || b < n || b > ORC_MAX_BUCKET_SIZE || N >= (1ull << 32) ||
      (leaf_mode != 0 && leaf_mode != 1))
    return ORC_EINVAL;
  const uint32_t rw_bits = orc_ribbon_width(n);
  if (shard_buckets == 0) shard_buckets = orc_default_shard_buckets(b, rw_bits);
  if (eps_num == 0) eps_num = orc_default_eps_num(rw_bits);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  int status = ORC_OK;
  uint64_t B = N ? (N + b - 1) / b : 0;
  uint64_t* fp = (uint64_t*)malloc((size_t)(N ? N : 1) * 16); /* (lo, hi) pairs */
  uint64_t* lo = (uint64_t*)malloc((size_t)(N ? N : 1) * 8);
  uint64_t* hi = (uint64_t*)malloc((size_t)(N ? N : 1) * 8);
  uint8_t* f = (uint8_t*)malloc((size_t)(N ? N : 1));
  uint64_t* K = (uint64_t*)calloc((size_t)B + 1, 8);
  uint64_t* O = (uint64_t*)calloc((size_t)B + 1, 8);
  codes_t* bc = (codes_t*)calloc((size_t)(B ? B : 1), sizeof(codes_t));
  bitvec_t rice = {0}, kl = {0}, kh = {0}, ol = {0}, oh = {0};
  uint64_t num_shards = (B + shard_buckets - 1) / shard_buckets;
  uint32_t* shard_seed = (uint32_t*)calloc((size_t)(num_shards ? num_shards : 1), 4);
  uint64_t* shard_off = (uint64_t*)calloc((size_t)num_shards + 1, 8);
  uint8_t* solbits = NULL;
  uint8_t* blob = NULL;
  if (!fp || !lo || !hi || !f || !K || !O || !bc || !shard_seed || !shard_off) {
    status = ORC_ENOMEM;
    goto done;
  }
  /* master hash */
  if (kind == ORC_KEYS_U64) {
    orc_fp_u64((const uint64_t*)data, N, lo, hi);
  } else if (kind == ORC_KEYS_STR) {
    orc_fp_str((const uint8_t*)data, offs, N, lo, hi);
  } else if (kind == ORC_KEYS_FP128) {
    const uint64_t* d = (const uint64_t*)data;
    for (uint64_t i = 0; i < N; i++) {
      lo[i] = d[2 * i];
      hi[i] = d[2 * i + 1];
    }
  } else {
    status = ORC_EINVAL;
    goto done;
  }
  /* bucket partition = sort by (hi, lo): the bucket is monotone in hi */
  for (uint64_t i = 0; i < N; i++) {
    fp[2 * i] = lo[i];
    fp[2 * i + 1] = hi[i];
  }
  qsort(fp, (size_t)N, 16, cmp_fp);
  for (uint64_t i = 0; i < N; i++) {
    lo[i] = fp[2 * i];
    hi[i] = fp[2 * i + 1];
    if (i && lo[i] == lo[i - 1] && hi[i] == hi[i - 1]) {
      status = ORC_EDUPKEY;
      goto done;
    }
  }
  for (uint64_t i = 0; i < N; i++) K[orc_bucket(hi[i], B) + 1]++;
  for (uint64_t i = 0; i < B; i++) {
    if (K[i + 1] > ORC_MAX_BUCKET_KEYS) {
      status = ORC_EINVAL;
      goto done;
    }
    K[i + 1] += K[i];
  }
  /* splitting trees, leaf seeds and orientations, one bucket at a time */
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < (int64_t)B; i++) {
    uint32_t size = (uint32_t)(K[i + 1] - K[i]);
    if (size == 0) continue;
    uint64_t* tlo = (uint64_t*)malloc((size_t)size * 8);
    uint64_t* thi = (uint64_t*)malloc((size_t)size * 8);
    int st = (tlo && thi)
                 ? build_node(lo + K[i], hi + K[i], f + K[i], size, n, &bc[i], tlo, thi, leaf_mode, NULL, 0)
                 : ORC_ENOMEM;
    free(tlo);
    free(thi);
    if (st != ORC_OK) {
#pragma omp critical
      status = st;
    }
  }
  if (status != ORC_OK) goto done;
  /* Rice stream, buckets in order */
  for (uint64_t i = 0; i < B; i++) {
    O[i] = rice.nbits;
    for (uint32_t j = 0; j < bc[i].n; j++)
      if (!rice_put(&rice, bc[i].seed[j], bc[i].k[j])) {
        status = ORC_ENOMEM;
        goto done;
      }
  }
  O[B] = rice.nbits;
  uint32_t lK, lO;
  if (!ef_encode(K, B + 1, &kl, &kh, &lK) || !ef_encode(O, B + 1, &ol, &oh, &lO)) {
    status = ORC_ENOMEM;
    goto done;
  }
  /* retrieval shards */
  for (uint64_t s = 0; s < num_shards; s++) {
    uint64_t b0 = s * shard_buckets, b1 = b0 + shard_buckets < B ? b0 + shard_buckets : B;
    shard_off[s + 1] = shard_off[s] + shard_slots(K[b1] - K[b0], eps_num, rw_bits);
  }
  solbits = (uint8_t*)calloc((size_t)shard_off[num_shards] + 1, 1);
  if (!solbits) {
    status = ORC_ENOMEM;
    goto done;
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t s = 0; s < (int64_t)num_shards; s++) {
    uint64_t b0 = (uint64_t)s * shard_buckets;
    uint64_t b1 = b0 + shard_buckets < B ? b0 + shard_buckets : B;
    uint64_t k0 = K[b0], keys = K[b1] - K[b0];
    int st = orc_ribbon_shard(lo + k0, hi + k0, f + k0, keys, eps_num, rw_bits, &shard_seed[s],
                              solbits + shard_off[s]);
    if (st != ORC_OK) {
#pragma omp critical
      status = st;
    }
  }
  if (status != ORC_OK) goto done;
  {
    uint64_t rib_bits = shard_off[num_shards];
    uint64_t w_rice = (rice.nbits + 63) / 64, w_kl = (kl.nbits + 63) / 64,
             w_kh = (kh.nbits + 63) / 64, w_ol = (ol.nbits + 63) / 64, w_oh = (oh.nbits + 63) / 64,
             w_seed = (num_shards + 7) / 8, w_rib = (rib_bits + 63) / 64;
    uint64_t words = ORC_HEADER_WORDS + w_rice + w_kl + w_kh + w_ol + w_oh + w_seed + w_rib;
    blob = (uint8_t*)calloc((size_t)words, 8);
    if (!blob) {
      status = ORC_ENOMEM;
      goto done;
    }
    uint64_t hdr[ORC_HEADER_WORDS] = {ORC_MAGIC, N, n, b, B, shard_buckets, eps_num, num_shards,
                                      rice.nbits, lK, kh.nbits, lO, oh.nbits, rib_bits,
                                      (uint64_t)leaf_mode, rw_bits};
    uint64_t pw = 0;
    put_words(blob, &pw, hdr, ORC_HEADER_WORDS);
    put_words(blob, &pw, rice.w, w_rice);
    put_words(blob, &pw, kl.w, w_kl);
    put_words(blob, &pw, kh.w, w_kh);
    put_words(blob, &pw, ol.w, w_ol);
    put_words(blob, &pw, oh.w, w_oh);
    for (uint64_t s = 0; s < num_shards; s++) blob[pw * 8 + s] = (uint8_t)shard_seed[s];
    pw += w_seed;
    uint64_t* rw = (uint64_t*)(blob + pw * 8);
    for (uint64_t p = 0; p < rib_bits; p++)
      if (solbits[p]) rw[p / 64] |= 1ull << (p % 64);
    pw += w_rib;
    *out = blob;
    *out_len = words * 8;
    blob = NULL;
  }
done:
  free(fp);
  free(lo);
  free(hi);
  free(f);
  free(K);
  free(O);
  if (bc) {
    for (uint64_t i = 0; i < B; i++) {
      free(bc[i].seed);
      free(bc[i].k);
    }
    free(bc);
  }
  free(rice.w);
  free(kl.w);
  free(kh.w);
  free(ol.w);
  free(oh.w);
  free(shard_seed);
  free(shard_off);
  free(solbits);
  free(blob);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Query (Sec. 1: x -> p_{g(x)} + h_{g(x)}(x); Sec. 4: retrieve f(x), return */
/* h_{s,f(x)}(x)).  Decodes the tree from the bucket's Rice stream.          */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint64_t N, n, b, B, shard_buckets, eps_num, num_shards, leaf_mode, width;
  const uint64_t* rice;
  const uint8_t* seeds;
  const uint64_t* rib;
  uint64_t* K;
  uint64_t* O;
  uint64_t* shard_off;
} mphf_view_t;

static void skip_subtree(const mphf_view_t* v, uint64_t* pos, uint32_t m) {
  uint32_t unit, fan;
  if (!orc_split_shape(m, (uint32_t)v->n, &unit, &fan)) {
    if (m >= 2) (void)rice_get(v->rice, pos, orc_rice_k_leaf(m));
    return;
  }
  (void)rice_get(v->rice, pos, orc_rice_k_split(m, (uint32_t)v->n));
  for (uint32_t j = 0; j < fan; j++) skip_subtree(v, pos, part_size(m, unit, fan, j));
}

static uint64_t query_one(const mphf_view_t* v, uint64_t lo, uint64_t hi) {
  uint64_t bkt = orc_bucket(hi, v->B);
  uint32_t m = (uint32_t)(v->K[bkt + 1] - v->K[bkt]);
  uint64_t pos = v->O[bkt], offset = 0;
  uint32_t n = (uint32_t)v->n;
  for (;;) {
    uint32_t unit, fan;
    if (!orc_split_shape(m, n, &unit, &fan)) break;
    uint64_t s = rice_get(v->rice, &pos, orc_rice_k_split(m, n));
    uint32_t child = orc_split_child(lo, s, m, unit, fan);
    for (uint32_t j = 0; j < child; j++) {
      uint32_t p = part_size(m, unit, fan, j);
      skip_subtree(v, &pos, p);
      offset += p;
    }
    m = part_size(m, unit, fan, child);
  }
  uint32_t local = 0;
  if (m >= 2) {
    uint64_t s = rice_get(v->rice, &pos, orc_rice_k_leaf(m));
    uint32_t h0, h1;
    leaf_cells_mode((int)v->leaf_mode, lo, s, m, &h0, &h1);
    uint64_t sh = bkt / v->shard_buckets;
    uint64_t b0 = sh * v->shard_buckets;
    uint64_t b1 = b0 + v->shard_buckets < v->B ? b0 + v->shard_buckets : v->B;
    uint64_t ms = shard_slots(v->K[b1] - v->K[b0], (uint32_t)v->eps_num, (uint32_t)v->width);
    uint64_t st;
    u128 c;
    ribbon_row(lo, hi, v->seeds[sh], ms, (uint32_t)v->width, &st, &c);
    int bit = 0;
    for (uint32_t j = 0; j < v->width; j++)
      if ((c >> j) & 1) bit ^= get_bit(v->rib, v->shard_off[sh] + st + j);
    local = bit ? h1 : h0;
  }
  return v->K[bkt] + offset + local;
}

int orc_query(const uint8_t* blob, uint64_t len, const uint64_t* lo, const uint64_t* hi,
              uint64_t nq, uint64_t* ranks) {
  if (len < ORC_HEADER_WORDS * 8 || (len % 8)) return ORC_EFORMAT;
  const uint64_t* h = (const uint64_t*)blob;
  if (h[0] != ORC_MAGIC) return ORC_EFORMAT;
  mphf_view_t v;
  v.N = h[1];
  v.n = h[2];
  v.b = h[3];
  v.B = h[4];
  v.shard_buckets = h[5];
  v.eps_num = h[6];
  v.num_shards = h[7];
  v.leaf_mode = h[14];
  v.width = h[15];
  if (v.leaf_mode > 1 || v.n < 2 || v.n > ORC_MAX_LEAF || v.width != orc_ribbon_width((uint32_t)v.n))
    return ORC_EFORMAT;
  uint64_t rice_bits = h[8], lK = h[9], khb = h[10], lO = h[11], ohb = h[12], rib = h[13];
  if (v.N == 0) return nq == 0 ? ORC_OK : ORC_EINVAL;
  uint64_t pw = ORC_HEADER_WORDS;
  const uint64_t* w = (const uint64_t*)blob;
  v.rice = w + pw;
  pw += (rice_bits + 63) / 64;
  const uint64_t* kl = w + pw;
  pw += ((v.B + 1) * lK + 63) / 64;
  const uint64_t* kh = w + pw;
  pw += (khb + 63) / 64;
  const uint64_t* ol = w + pw;
  pw += ((v.B + 1) * lO + 63) / 64;
  const uint64_t* oh = w + pw;
  pw += (ohb + 63) / 64;
  v.seeds = blob + pw * 8;
  pw += (v.num_shards + 7) / 8;
  v.rib = w + pw;
  pw += (rib + 63) / 64;
  if (pw * 8 != len) return ORC_EFORMAT;
  v.K = (uint64_t*)malloc((size_t)(v.B + 1) * 8);
  v.O = (uint64_t*)malloc((size_t)(v.B + 1) * 8);
  v.shard_off = (uint64_t*)calloc((size_t)v.num_shards + 1, 8);
  if (!v.K || !v.O || !v.shard_off) {
    free(v.K);
    free(v.O);
    free(v.shard_off);
    return ORC_ENOMEM;
  }
  ef_decode_all(kl, kh, khb, (uint32_t)lK, v.B + 1, v.K);
  ef_decode_all(ol, oh, ohb, (uint32_t)lO, v.B + 1, v.O);
  for (uint64_t s = 0; s < v.num_shards; s++) {
    uint64_t b0 = s * v.shard_buckets;
    uint64_t b1 = b0 + v.shard_buckets < v.B ? b0 + v.shard_buckets : v.B;
    v.shard_off[s + 1] =
        v.shard_off[s] + shard_slots(v.K[b1] - v.K[b0], (uint32_t)v.eps_num, (uint32_t)v.width);
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)nq; i++) ranks[i] = query_one(&v, lo[i], hi[i]);
  free(v.K);
  free(v.O);
  free(v.shard_off);
  return ORC_OK;
}

void orc_free(void* p) { free(p); }
