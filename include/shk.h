/*
 * shk.h -- C ABI of the GB300 ShockHash-RS construction library (libshk_gpu.so).
 *
 * The library builds minimal perfect hash functions (MPHFs): bijections from a
 * set of N distinct keys onto [0, N) (paper Sec. 1), with the ShockHash-RS
 * construction: keys hashed to buckets and split recursively (RecSplit, Sec. 2;
 * fanouts Sec. 6), each leaf solved by the ShockHash seed search (Sec. 4, Eq.
 * ShockHash: the smallest seed whose 2-choice graph is a pseudoforest, with the
 * bit-mask filter of Sec. 4), the orientation bits of all keys stored in one
 * 1-bit retrieval structure (Sec. 2 Retrieval, Sec. 6).  Every step runs in CUDA
 * kernels on the calling device; the result is bit-identical to the format
 * defined by the project (version SHKRS002).
 *
 * Conventions
 *   - Every function returns an shk_status and never aborts.  On failure a
 *     message is available from shk_last_error() (thread-local, valid until
 *     the next call on the same thread).
 *   - Input buffers are borrowed for the duration of the call.  Objects that
 *     the library returns (shk_mphf) are owned by the caller and released with
 *     shk_free().
 *   - "Device" pointers are CUDA global-memory addresses of the current
 *     device; "host" pointers are ordinary (pageable or pinned) host memory.
 *   - cuda_stream is a cudaStream_t (NULL = the legacy default stream).  The
 *     functions enqueue their work on that stream and return after it has
 *     completed (they synchronise it), except where stated.
 *   - The current CUDA device at call time is the device that is used.
 */
#ifndef SHK_H
#define SHK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SHK_OK = 0,
  SHK_EINVAL = 1,     /* bad argument (sizes, limits, null pointers)            */
  SHK_EDUPKEY = 2,    /* two keys have the same 128-bit fingerprint             */
  SHK_ENOMEM = 3,     /* a host or device allocation failed                     */
  SHK_ECUDA = 4,      /* a CUDA call failed; the message names it              */
  SHK_ESEEDCAP = 5,   /* a seed search reached its cap (never in practice)      */
  SHK_ETIMEOUT = 6,   /* a build's time budget (deadline_ms) ran out            */
  SHK_EFORMAT = 7,    /* a serialized MPHF is malformed                         */
  SHK_ECANCELLED = 8  /* a served request was cancelled (shk_server_cancel)     */
} shk_status;

typedef enum {
  SHK_KEYS_U64 = 0,   /* data: uint64_t[n_keys]                                 */
  SHK_KEYS_STR = 1,   /* data: uint8_t bytes; str_offsets: uint64_t[n_keys + 1] */
  SHK_KEYS_FP128 = 2  /* data: uint64_t[2 * n_keys], (lo, hi) per key, used as   */
                      /*       the 128-bit fingerprint directly                 */
} shk_key_kind;

/* A borrowed set of keys.  If on_device is non-zero, data (and str_offsets)
 * are device pointers, otherwise host pointers. */
typedef struct {
  int32_t kind;                 /* shk_key_kind                                */
  int32_t on_device;            /* 0 = host buffers, 1 = device buffers        */
  const void* data;
  const uint64_t* str_offsets;  /* SHK_KEYS_STR only, else NULL                */
  uint64_t n_keys;
} shk_keys;

/* Leaf-search scheduling (both give identical results). */
typedef enum {
  SHK_SCHED_PERSISTENT = 0,     /* one persistent launch over all leaves, work  */
                                /* stealing over (leaf, seed-chunk) items       */
  SHK_SCHED_PER_BUCKET = 1,     /* one launch per bucket, one warp per leaf     */
  SHK_SCHED_SINGLE_LAUNCH = 2   /* one launch over all leaves, one warp per     */
                                /* leaf, no work sharing                        */
} shk_sched;

/* How leaves are solved (both are ShockHash: the smallest value whose graph
 * is a pseudoforest). */
typedef enum {
  SHK_LEAF_PLAIN = 0,    /* value = seed s (Sec. 4, Eq. ShockHash)                  */
  SHK_LEAF_ROTATION = 1  /* value = s*m + r: rotation fitting with partial hash     */
                         /* calculation (Sec. 4 Rotation Fitting, App. A.2)       */
} shk_leaf_mode;

/* Build options.  Zero-initialise and set leaf_size and bucket_size; zero in
 * any other field selects its default. */
typedef struct {
  uint32_t leaf_size;        /* n, 2..64 (leaf bit mask is one 64-bit word)      */
  uint32_t bucket_size;      /* b, n..4096: expected keys per bucket            */
  uint32_t shard_buckets;    /* retrieval shard = this many buckets; 0 = the     */
                             /* default: 12288/b (leaf size > 24: 128-bit rows), */
                             /* 8192/b (64-bit rows), at least 1                 */
  uint32_t eps_num;          /* retrieval overhead eps = eps_num/65536; 0 = the  */
                             /* default: 66 (128-bit rows), 3277 (64-bit rows)   */
  uint32_t sched;            /* shk_sched                                        */
  uint32_t seeds_per_lane;   /* leaf kernel: seeds per lane per pass (1, 2, 4);  */
                             /* 0 = the autotuner's choice for this leaf size     */
  uint32_t chunk_passes;     /* leaf kernel: passes per work item, 0 = default    */
  uint32_t profile;          /* 1: time each phase with CUDA events              */
  uint32_t warps_per_block;  /* with seeds_per_lane != 0: 4, 8 or 16; 0 = 8      */
  uint32_t key_unroll;       /* with seeds_per_lane != 0: 1, 2 or 4; 0 = 2       */
  uint32_t leaf_mode;        /* shk_leaf_mode; recorded in the encoded header     */
  uint32_t deadline_ms;      /* 0 = none; else the leaf search stops once this    */
                             /* many ms have passed since the build started on    */
                             /* the device (checked once per work item, about    */
                             /* every 0.1 ms) and the build fails with           */
                             /* SHK_ETIMEOUT                                      */
} shk_build_opts;

/* Statistics of the build that produced an MPHF (shk_build_stats). */
typedef struct {
  uint64_t n_keys, n_buckets, n_leaves, n_search_leaves, n_split_nodes;
  uint64_t leaf_seeds_min;      /* sum over leaves of (seed + 1): the seeds a    */
                                /* sequential search tests                      */
  uint64_t leaf_seeds_executed; /* seeds the leaf kernel actually evaluated      */
  uint64_t leaf_key_evals;      /* sum over leaves of (seed + 1) * m             */
  uint64_t kernel_launches;     /* library kernels launched by the build         */
  uint64_t size_bits;           /* shk_size_bits                                 */
  /* phase times in milliseconds (profile = 1), CUDA events on the stream:  */
  /* fingerprint = key staging, fingerprints and the bucket histogram;       */
  /* partition = bucket offsets and the scatter into buckets; split = the    */
  /* in-bucket sort and the splitting trees; leaf; orient; encode = Rice and */
  /* Elias-Fano; ribbon = retrieval; total also holds the tree bookkeeping   */
  /* and its host synchronisation.                                           */
  double ms_fingerprint, ms_partition, ms_split, ms_leaf, ms_orient, ms_encode,
      ms_ribbon, ms_total;
  uint64_t leaf_launches;       /* launches of the leaf-search kernel           */
  uint32_t leaf_cfg[4];         /* seeds per lane, warps per block, key unroll,  */
                                /* passes per work item of the leaf kernel      */
  /* Work a sequential search over the same leaves does (the roofline's      */
  /* numerator), counted from the results:                                   */
  uint64_t leaf_hash_evals;     /* key hash evaluations: (seed + 1) * m per      */
                                /* plain leaf; with rotation fitting, seeds      */
                                /* tested T = floor(v/m) + 1 and, for m > 32,    */
                                /* |B| T + |A| ceil(T/8) (set A hashed once per  */
                                /* 8 seeds, App. A.2), else m T                  */
  double leaf_rf_cells;         /* rotation fitting, m > 32: (seed, missed cell) */
                                /* steps of the bit-parallel rotation filter,    */
                                /* 8 ceil(T/8) x E[min(cells A misses, 24 (m =   */
                                /* 64) or 20)] given |A| (exact expectation for  */
                                /* ideal hashing); 0 otherwise                  */
  uint64_t leaf_seeds_tested;   /* seeds a sequential search tests: sum of seed  */
                                /* + 1 (plain) or floor(v/m) + 1 (rotation       */
                                /* fitting) over leaves                         */
  uint64_t leaf_t0_ns, leaf_t1_ns; /* device global timer (ns) when the first    */
                                /* leaf-search block started and the last one   */
                                /* ended (persistent schedule): lets concurrent */
                                /* builds' kernels be compared on one clock     */
  uint64_t device_bytes_peak;   /* high watermark of the library's device memory */
                                /* pool during the build, plus the result; only  */
                                /* a build that runs alone reads its own peak    */
} shk_stats;

typedef struct shk_mphf shk_mphf;

/* shk_build -- construct an MPHF over keys (paper Sec. 6, ShockHash-RS).
 *   keys:   borrowed; host or device buffers (keys->on_device).
 *   opts:   leaf_size n in [2, 64]; bucket_size b in [n, 4096].
 *   out:    receives a new object owned by the caller (shk_free).
 * Errors: SHK_EINVAL (limits, N >= 2^32, a bucket above 8192 keys),
 * SHK_EDUPKEY, SHK_ENOMEM, SHK_ECUDA, SHK_ESEEDCAP.  The result is resident on
 * the current device and also serialisable with shk_serialize. */
shk_status shk_build(const shk_keys* keys, const shk_build_opts* opts, void* cuda_stream,
                     shk_mphf** out);

/* shk_build_stats -- statistics of the build that produced mphf. */
shk_status shk_build_stats(const shk_mphf* mphf, shk_stats* out);

/* shk_query -- ranks of keys (paper Sec. 1: x -> p_{g(x)} + h_{g(x)}(x); Sec. 4:
 * the leaf part is h_{s,f(x)}(x) with f(x) from the retrieval structure).
 *   ranks_out: uint64_t[keys->n_keys], device memory if out_on_device, else host.
 * For keys of the build set the ranks are a permutation of [0, N); for other
 * keys the result is some value in [0, N) (retrieval semantics, Sec. 2).
 * The first query on an object decodes its tree codes once into a device-side
 * query index (16 bytes per code, about 0.5 bytes per key at leaf size 48;
 * freed by shk_free) and waits for it; later queries, also from other host
 * threads, use it.  Queries on one object may run concurrently. */
shk_status shk_query(const shk_mphf* mphf, const shk_keys* keys, uint64_t* ranks_out,
                     int out_on_device, void* cuda_stream);

/* shk_serialize -- copy the encoded MPHF (format SHKRS002) into buf (host).
 * With buf == NULL or cap too small, only *len is set (and SHK_EINVAL is
 * returned if buf was given but too small). */
shk_status shk_serialize(const shk_mphf* mphf, uint8_t* buf, size_t cap, size_t* len);

/* shk_deserialize -- load a serialized MPHF (host bytes) onto the current
 * device.  SHK_EFORMAT if the bytes are not a well-formed SHKRS002 object. */
shk_status shk_deserialize(const uint8_t* buf, size_t len, shk_mphf** out);

/* shk_size_bits -- size of the encoded MPHF in bits (header included). */
uint64_t shk_size_bits(const shk_mphf* mphf);

/* shk_free -- release an MPHF and its device memory.  NULL is ignored. */
void shk_free(shk_mphf* mphf);

/* shk_last_error -- message of the last failure on this thread ("" if none). */
const char* shk_last_error(void);

/* shk_leaf_search -- batched ShockHash leaf search over independent leaves
 * (paper Sec. 4: for each leaf the smallest seed >= seed_start whose graph
 * ([m], {{h0(x), h1(x)}}) is a pseudoforest, found with the bit-mask filter
 * and a union-find test of survivors; f = the lexicographically smallest
 * 1-orientation).
 *   leaf_keys: device uint64_t[leaf_off[n_leaves]]: the 64-bit leaf inputs x.
 *   leaf_off:  device uint32_t[n_leaves + 1]; leaf i holds
 *              leaf_keys[leaf_off[i] .. leaf_off[i+1]), 1 <= size <= 64.
 *   seeds_out: device uint64_t[n_leaves].
 *   f_out:     device uint64_t[n_leaves] or NULL; bit j = f of key j.
 * The persistent launch is captured in a CUDA graph and replayed.  Errors:
 * SHK_EINVAL (a leaf of size 0 or above 64), SHK_ESEEDCAP, SHK_ECUDA. */
shk_status shk_leaf_search(const uint64_t* leaf_keys, const uint32_t* leaf_off,
                           uint32_t n_leaves, uint64_t seed_start, uint64_t* seeds_out,
                           uint64_t* f_out, void* cuda_stream);

/* shk_leaf_search_noalloc -- shk_leaf_search without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they run -- a process whose GPU memory
 * is owned by another memory manager, or a serving loop with a fixed memory
 * budget that must not meet an out-of-memory error or the device-wide
 * synchronisation of cudaMalloc/cudaFree mid-request.  Arguments, results and
 * errors are those of shk_leaf_search; the caller still provides every input
 * and output buffer.  Working memory comes from one fixed array in the
 * library's device image (about 1.3 MB, held by every GPU that loads the
 * library until the process exits), so n_leaves is limited to 65536
 * (SHK_EINVAL beyond, with a message).  Each call looks up the array's
 * device address on the current device (no allocation), reads the device
 * error flag back and synchronises cuda_stream, so it cannot be called inside
 * a stream capture.  All calls share the array: calls that overlap on the GPU
 * race and must be serialised by the caller. */
shk_status shk_leaf_search_noalloc(const uint64_t* leaf_keys, const uint32_t* leaf_off,
                                   uint32_t n_leaves, uint64_t seed_start, uint64_t* seeds_out,
                                   uint64_t* f_out, void* cuda_stream);

/* shk_leaf_tune -- the leaf kernel configuration the autotuner picks for
 * leaves of leaf_size keys on the current device (timed once per device and
 * leaf-size bin, then cached).  cfg_out[4] = seeds per lane, warps per
 * block, key-loop unroll, passes per work item; evals_per_s (nullable) = its
 * measured key-seed evaluations per second.  With probe_all, every supported
 * configuration is timed into all_evals_per_s[shk_leaf_configs()].  The
 * configuration never changes results. */
shk_status shk_leaf_tune(uint32_t leaf_size, uint32_t* cfg_out, double* evals_per_s,
                         int probe_all, double* all_evals_per_s);

/* shk_leaf_configs -- the supported leaf kernel configurations, 4 words each
 * (as in shk_leaf_tune; passes 0); returns their number. */
uint32_t shk_leaf_configs(uint32_t* cfgs, uint32_t cap);

/* shk_leaf_search_rf -- the batched leaf search with rotation fitting and
 * partial hash calculation (paper Sec. 4 Rotation Fitting, App. A.2): per
 * leaf the smallest v = s*m + r whose graph is a pseudoforest, where set A's
 * keys take the cells of seed s - (s mod 8) (m > 32; s otherwise) and set B's
 * the cells of seed s moved by r (mod m); f as in shk_leaf_search.  Buffers
 * and errors as for shk_leaf_search (no seed start: values start at 0). */
shk_status shk_leaf_search_rf(const uint64_t* leaf_keys, const uint32_t* leaf_off,
                              uint32_t n_leaves, uint64_t* values_out, uint64_t* f_out,
                              void* cuda_stream);

/* shk_leaf_graph_replays -- how many times this host thread has launched the
 * captured leaf-search graph (each shk_leaf_search call launches it once;
 * calls with unchanged pointers and sizes reuse the instantiated graph). */
uint64_t shk_leaf_graph_replays(void);

/* ---- Serving: a request loop over builds of different sizes ----------------
 * A server owns a queue of build requests and a pool of workers, each with its
 * own CUDA stream on the device current at creation.  A request is admitted
 * (first in, first out) as soon as a worker is free and its estimated device
 * footprint fits in what the budget leaves (a request larger than the whole
 * budget runs alone).  Admitted builds run concurrently, so the kernels of
 * different requests overlap on the GPU, and requests arriving while others
 * run are admitted as slots and memory free up.  Each result is the same MPHF
 * that shk_build returns for the same keys and options. */
typedef struct shk_server shk_server;

typedef struct {
  int32_t done;               /* 1 when finished (successfully or not)      */
  int32_t status;             /* the build's status once done               */
  uint64_t n_keys;
  uint64_t footprint_bytes;   /* device memory reserved by admission        */
  uint64_t submit_ns, start_ns, finish_ns; /* steady-clock timestamps       */
} shk_request_info;

typedef struct {
  uint64_t submitted, completed, queued, running;
  uint64_t budget_bytes, in_use_bytes, peak_in_use_bytes;
  uint32_t workers;
} shk_server_stats;

/* shk_server_create -- hbm_budget_bytes: device memory the server may reserve
 * for running builds (0 = 80 % of the free memory); workers: builds in flight
 * (0 = 4). */
shk_status shk_server_create(uint64_t hbm_budget_bytes, uint32_t workers, shk_server** out);

/* shk_server_submit -- queue a build.  keys are copied before the call returns:
 * host keys into host memory, device keys into the library's device memory
 * pool on the server's device (they never pass through the host); opts as for
 * shk_build.  *req_id identifies it. */
shk_status shk_server_submit(shk_server* srv, const shk_keys* keys, const shk_build_opts* opts,
                             uint64_t* req_id);

/* shk_server_poll -- non-blocking.  While the request runs or waits, *out is
 * NULL and info->done is 0.  Once done, *out receives the MPHF (owned by the
 * caller; NULL if the build failed, with info->status its error) and the
 * request is forgotten.  SHK_EINVAL for an unknown request id. */
shk_status shk_server_poll(shk_server* srv, uint64_t req_id, shk_mphf** out,
                           shk_request_info* info);

/* shk_server_wait -- as shk_server_poll, blocking until the request is done.
 * If another thread collects the same request first, SHK_EINVAL (unknown
 * request id). */
shk_status shk_server_wait(shk_server* srv, uint64_t req_id, shk_mphf** out,
                           shk_request_info* info);

/* shk_server_cancel -- cancel a request.  A queued request never runs; a
 * running one stops its leaf search at its next work item (the build's
 * kernels poll a host-mapped flag).  Either way the request completes with
 * status SHK_ECANCELLED and no MPHF (also if its build had already finished
 * but was not yet collected).  A finished request is left as it is.
 * SHK_EINVAL for an unknown request id. */
shk_status shk_server_cancel(shk_server* srv, uint64_t req_id);

/* shk_build_footprint -- the device bytes the server reserves for a build of
 * these keys with these options (the admission estimate): the keys as
 * staged, 96 bytes per key, 96 per bucket and 8 MiB; with leaf size above 24
 * also the 128-bit retrieval solver's scratch (37 bytes per slot of a shard
 * of 1.25 times the average shard's keys plus 512, for each of its persistent
 * warps: those resident on the device, at most 8 per shard).  A build that runs
 * alone reports its measured peak in shk_stats.device_bytes_peak. */
shk_status shk_build_footprint(const shk_keys* keys, const shk_build_opts* opts, uint64_t* bytes);

/* shk_server_get_stats -- counters and the device-memory reservation. */
shk_status shk_server_get_stats(shk_server* srv, shk_server_stats* out);

/* shk_server_destroy -- finish running builds, drop queued ones, free results
 * never polled.  No other call on srv may be in progress or follow.  NULL is
 * ignored. */
void shk_server_destroy(shk_server* srv);

/* shk_int_issue_rate -- integer-issue microbenchmark of the current device.
 * The paper has no counterpart: it measures the ceiling the leaf search's
 * roofline is quoted against (the leaf kernels are bound by integer issue,
 * Sec. 4's filter being a few 32-bit operations per key and seed).  One
 * persistent launch (SMs x resident 256-thread blocks), each thread running
 * 8 independent chains for iters iterations; best of 3 timed launches after
 * a warm-up.
 *   mix 0: 3-input logic + funnel shift; 1: 32-bit multiply-add; 2: both, 1:1;
 *          3: the leaf hash and 64-bit coverage-mask update for 8 seeds x 16
 *          keys held in registers.
 *   *rate: lane operations per second (mix 3: key-seed evaluations per second).
 *   *ms:   (nullable) duration of the best launch.
 * Errors: SHK_EINVAL (mix > 3, iters = 0, rate NULL), SHK_ENOMEM, SHK_ECUDA. */
shk_status shk_int_issue_rate(uint32_t mix, uint32_t iters, double* rate, double* ms,
                              void* cuda_stream);

/* shk_version -- format version string ("SHKRS002"). */
const char* shk_version(void);

/* shk_release_memory -- return to the device the working memory the library
 * keeps between calls.  Builds and queries take their temporary device memory
 * from a memory pool per device that the library owns; memory freed at the end
 * of a call stays in that pool (up to the largest call's working set) so that
 * the next call does not map it again.  Safe while other calls run: only memory
 * no call holds is released.  MPHF objects are not affected. */
void shk_release_memory(void);

#ifdef __cplusplus
}
#endif

#endif /* SHK_H */
