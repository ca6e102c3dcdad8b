// query.cu -- rank of a key (paper Sec. 1: x -> p_{g(x)} + h_{g(x)}(x); Sec. 4:
// a ShockHash leaf returns h_{s,f(x)}(x) with f(x) from the retrieval
// structure).  One thread per key: bucket from the fingerprint, tree descent
// by decoding the bucket's Rice stream, leaf cell, retrieval parity.
#include "kernels.cuh"

namespace shk {

struct QueryView {
  const uint64_t* rice;
  uint64_t rice_words;
  const uint8_t* seeds;
  const uint64_t* rib;
  uint64_t rib_words;
  const uint32_t* K;
  const uint64_t* O;
  const uint64_t* shard_off;
  uint64_t B;
  uint32_t n, S, eps_num, leaf_mode, w;
};

__device__ __forceinline__ uint64_t window64(const uint64_t* w, uint64_t nwords, uint64_t p) {
  const uint64_t i = p >> 6;
  const uint32_t sh = (uint32_t)(p & 63);
  uint64_t v = i < nwords ? w[i] >> sh : 0;
  if (sh && i + 1 < nwords) v |= w[i + 1] << (64 - sh);
  return v;
}

// Retrieval parity of a key: coefficient & solution window (w bits from
// start) over GF(2).
__device__ __forceinline__ uint32_t retrieve_bit(const QueryView& q, uint64_t b, uint64_t lo,
                                                 uint64_t hi) {
  const uint64_t sh = b / q.S;
  const uint64_t b0 = sh * q.S, b1 = b0 + q.S < q.B ? b0 + q.S : q.B;
  const uint64_t ms = shard_slots(q.K[b1] - q.K[b0], q.eps_num, q.w);
  uint64_t st, c0, c1;
  ribbon_row(lo, hi, q.seeds[sh], ms, q.w, &st, &c0, &c1);
  const uint64_t p = q.shard_off[sh] + st;
  uint32_t par = __popcll(window64(q.rib, q.rib_words, p) & c0);
  if (q.w == 128) par += __popcll(window64(q.rib, q.rib_words, p + 64) & c1);
  return par & 1u;
}

__device__ __forceinline__ uint64_t rice_next(const QueryView& q, uint64_t* pos, uint32_t k) {
  uint64_t low = 0;
  if (k) {
    low = window64(q.rice, q.rice_words, *pos) & ((1ull << k) - 1);
    *pos += k;
  }
  uint64_t quo = 0;
  for (;;) {
    const uint64_t w = window64(q.rice, q.rice_words, *pos);
    const uint64_t zeros = ~w;
    if (zeros) {
      const uint32_t ones = __ffsll((long long)zeros) - 1;
      quo += ones;
      *pos += ones + 1;
      break;
    }
    quo += 64;
    *pos += 64;
  }
  return (quo << k) | low;
}

__device__ void skip_subtree(const QueryView& q, uint64_t* pos, uint32_t m0) {
  uint32_t stack[64];
  int sp = 0;
  stack[sp++] = m0;
  while (sp > 0) {
    const uint32_t m = stack[--sp];
    SplitShape s;
    if (split_shape(m, q.n, &s)) {
      (void)rice_next(q, pos, rice_k_split(m, q.n));
      for (int j = (int)s.fanout - 1; j >= 0 && sp < 64; j--) stack[sp++] = part_size(m, s, (uint32_t)j);
    } else if (m >= 2) {
      (void)rice_next(q, pos, rice_k_leaf(m));
    }
  }
}

__device__ uint64_t query_one(const QueryView& q, uint64_t lo, uint64_t hi) {
  const uint64_t b = mulhi64(hi, q.B);
  uint32_t m = q.K[b + 1] - q.K[b];
  uint64_t pos = q.O[b];
  uint64_t offset = 0;
  SplitShape s;
  while (split_shape(m, q.n, &s)) {
    const uint64_t seed = rice_next(q, &pos, rice_k_split(m, q.n));
    const uint64_t d = mix64(mix64(kSplitSalt + m) + seed);
    const uint32_t a = ((uint32_t)(lo >> 32) ^ (uint32_t)d) * ((uint32_t)lo | 1u) + (uint32_t)(d >> 32);
    const uint32_t v = __umulhi(a, m);
    uint32_t child = 0;
    for (uint32_t j = 1; j < s.fanout; j++) child += v >= j * s.unit;
    for (uint32_t j = 0; j < child; j++) {
      skip_subtree(q, &pos, s.unit);
      offset += s.unit;
    }
    m = part_size(m, s, child);
  }
  uint32_t local = 0;
  if (m >= 2) {
    const uint64_t seed = rice_next(q, &pos, rice_k_leaf(m));
    uint32_t h0, h1;
    value_cells(q.leaf_mode, lo, seed, m, &h0, &h1);
    local = retrieve_bit(q, b, lo, hi) ? h1 : h0;
  }
  return q.K[b] + offset + local;
}

__global__ void k_query(QueryView q, const uint64_t* lo, const uint64_t* hi, uint64_t n,
                        uint64_t* ranks) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    ranks[i] = query_one(q, lo[i], hi[i]);
}

// Query index: one thread per bucket decodes the bucket's Rice stream once, in
// the preorder in which it was written, into one record per code; a split
// node's record gets the distance to each later child's first record.
__global__ void k_qindex_build(QueryView q, const uint32_t* __restrict__ qbase, QNode* out) {
  const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= q.B) return;
  const uint32_t m0 = q.K[b + 1] - q.K[b];
  if (m0 < 2 || m0 > kMaxBucketKeys) return;  // no records (as counted by the tree bookkeeping)
  uint64_t pos = q.O[b];
  uint32_t next = qbase[b];
  uint32_t st_m[64], st_parent[64], st_j[64];
  int sp = 0;
  st_m[0] = m0;
  st_parent[0] = 0;
  st_j[0] = 0;
  sp = 1;
  while (sp > 0) {
    sp--;
    const uint32_t m = st_m[sp], parent = st_parent[sp], j = st_j[sp];
    if (j > 0) out[parent].child[j - 1] = (uint16_t)(next - parent);
    SplitShape s;
    if (split_shape(m, q.n, &s)) {
      const uint32_t idx = next++;
      out[idx].seed = rice_next(q, &pos, rice_k_split(m, q.n));
      for (int c = (int)s.fanout - 1; c >= 0 && sp < 64; c--) {
        st_m[sp] = part_size(m, s, (uint32_t)c);
        st_parent[sp] = idx;
        st_j[sp] = (uint32_t)c;
        sp++;
      }
    } else if (m >= 2) {
      out[next++].seed = rice_next(q, &pos, rice_k_leaf(m));
    }
  }
}

// Rank of a key through the query index: one 16-byte record per tree level.
__device__ uint64_t query_one_indexed(const QueryView& q, const QNode* __restrict__ nodes,
                                      const uint32_t* __restrict__ qbase, uint64_t lo,
                                      uint64_t hi) {
  const uint64_t b = mulhi64(hi, q.B);
  uint32_t m = q.K[b + 1] - q.K[b];
  if (m > kMaxBucketKeys) return query_one(q, lo, hi);  // a bucket without records
  uint32_t node = qbase[b];
  uint64_t offset = 0;
  SplitShape s;
  while (split_shape(m, q.n, &s)) {
    const QNode r = nodes[node];
    const uint64_t d = mix64(mix64(kSplitSalt + m) + r.seed);
    const uint32_t a = ((uint32_t)(lo >> 32) ^ (uint32_t)d) * ((uint32_t)lo | 1u) + (uint32_t)(d >> 32);
    const uint32_t v = __umulhi(a, m);
    uint32_t child = 0;
    for (uint32_t j = 1; j < s.fanout; j++) child += v >= j * s.unit;
    offset += (uint64_t)child * s.unit;
    node += child ? r.child[child - 1] : 1u;
    m = part_size(m, s, child);
  }
  uint32_t local = 0;
  if (m >= 2) {
    uint32_t h0, h1;
    value_cells(q.leaf_mode, lo, nodes[node].seed, m, &h0, &h1);
    local = retrieve_bit(q, b, lo, hi) ? h1 : h0;
  }
  return q.K[b] + offset + local;
}

__global__ void k_query_indexed(QueryView q, const QNode* nodes, const uint32_t* qbase,
                                const uint64_t* lo, const uint64_t* hi, uint64_t n,
                                uint64_t* ranks) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    ranks[i] = query_one_indexed(q, nodes, qbase, lo[i], hi[i]);
}

static QueryView query_view(const shk_mphf* mp) {
  QueryView q;
  q.rice = mp->d_blob + mp->off_rice;
  q.rice_words = mp->off_kl - mp->off_rice;
  q.seeds = (const uint8_t*)(mp->d_blob + mp->off_seed);
  q.rib = mp->d_blob + mp->off_rib;
  q.rib_words = mp->words - mp->off_rib;
  q.K = mp->d_K;
  q.O = mp->d_O;
  q.shard_off = mp->d_shard_off;
  q.B = mp->hdr[4];
  q.n = (uint32_t)mp->hdr[2];
  q.S = (uint32_t)mp->hdr[5];
  q.eps_num = (uint32_t)mp->hdr[6];
  q.leaf_mode = (uint32_t)mp->hdr[14];
  q.w = (uint32_t)mp->hdr[15];
  return q;
}

shk_status launch_query(Ctx& c, const shk_mphf* mp, const uint64_t* lo, const uint64_t* hi,
                        uint64_t n, uint64_t* ranks) {
  if (n == 0) return SHK_OK;
  const QueryView q = query_view(mp);
  uint64_t blocks = (n + 255) / 256;
  if (blocks > (uint64_t)c.num_sms * 16) blocks = (uint64_t)c.num_sms * 16;
  if (mp->d_qnode)
    k_query_indexed<<<(unsigned)blocks, 256, 0, c.stream>>>(q, mp->d_qnode, mp->d_qbase, lo, hi, n,
                                                             ranks);
  else
    k_query<<<(unsigned)blocks, 256, 0, c.stream>>>(q, lo, hi, n, ranks);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

shk_status launch_qindex_build(Ctx& c, const shk_mphf* mp, const uint32_t* qbase, QNode* nodes) {
  const QueryView q = query_view(mp);
  if (q.B == 0) return SHK_OK;
  k_qindex_build<<<(unsigned)((q.B + 127) / 128), 128, 0, c.stream>>>(q, qbase, nodes);
  c.launches++;
  SHK_CUDA(cudaGetLastError());
  return SHK_OK;
}

}  // namespace shk
