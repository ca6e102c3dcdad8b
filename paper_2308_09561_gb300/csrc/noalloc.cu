// noalloc.cu -- shk_leaf_search_noalloc: the batched leaf search without any
// device allocation.
//
// Some callers cannot allocate device memory while they run: a process whose
// device memory is entirely owned by another memory manager (a framework's
// caching allocator that has reserved the GPU), or a serving loop that has
// fixed its memory budget up front and must not see an out-of-memory error
// or the device-wide synchronisation of cudaMalloc/cudaFree in the middle of
// a request.  For them this entry point takes its working memory from one
// fixed array that lives in the library's device image instead of from the
// allocator.  The caller still provides the inputs and the outputs.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kNoAllocScratchBytes, about 1.3 MB) until the process
// exits.  Host code cannot use the symbol as a device address, so every call
// looks the address up with cudaGetSymbolAddress on the current device (an
// allocation-free lookup; no address is cached, so a context that was reset
// and rebuilt is looked up afresh).  All calls share the one array and it
// keeps the previous call's contents, so each call clears the parts that
// must start at zero.  Calls whose work overlaps on the GPU (on different
// streams, or from different host threads) race on the array and must be
// serialised by the caller.  Each call reads the device error flag back and
// synchronises its stream, so it cannot be issued inside a stream capture.
#include "kernels.cuh"

namespace shk {

// Largest batch the fixed scratch holds.
constexpr uint32_t kNoAllocMaxLeaves = 65536;

// scratch layout (bytes): leaf descriptors | work state | error flag |
// seed counter
constexpr size_t kNaDescBytes = (size_t)kNoAllocMaxLeaves * sizeof(LeafDesc);
constexpr size_t kNaStateWords = (size_t)kNoAllocMaxLeaves + (kNoAllocMaxLeaves + 31) / 32 + 1;
constexpr size_t kNaStateBytes = ((kNaStateWords * 4 + 255) / 256) * 256;
constexpr size_t kNaErrOff = kNaDescBytes + kNaStateBytes;
constexpr size_t kNaCountOff = kNaErrOff + 256;
constexpr size_t kNoAllocScratchBytes = kNaCountOff + 256;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device (host code may
// not use the symbol itself as an address).
static shk_status noalloc_scratch(uint8_t** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr)
    return fail(SHK_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = (uint8_t*)p;
  return SHK_OK;
}

__global__ void k_na_leaf_descs(const uint32_t* off, uint32_t n_leaves, LeafDesc* d) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_leaves) return;
  LeafDesc v;
  v.key_off = off[i];
  v.m = off[i + 1] - off[i];
  v.code_idx = kNoCode;
  v.bucket = 0;
  d[i] = v;
}

}  // namespace shk

using namespace shk;

extern "C" shk_status shk_leaf_search_noalloc(const uint64_t* leaf_keys, const uint32_t* leaf_off,
                                              uint32_t n_leaves, uint64_t seed_start,
                                              uint64_t* seeds_out, uint64_t* f_out,
                                              void* cuda_stream) {
  if (n_leaves > kNoAllocMaxLeaves)
    return fail(SHK_EINVAL, "shk_leaf_search_noalloc: n_leaves exceeds the fixed scratch limit of 65536");
  if (n_leaves && (!leaf_keys || !leaf_off || !seeds_out)) return fail(SHK_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Ctx c(st);
  SHK_TRY(init_ctx(c));
  uint8_t* scratch = nullptr;
  SHK_TRY(noalloc_scratch(&scratch));
  if (n_leaves == 0) return SHK_OK;
  LeafDesc* d = (LeafDesc*)scratch;
  uint32_t* state = (uint32_t*)(scratch + kNaDescBytes);
  uint32_t* err = (uint32_t*)(scratch + kNaErrOff);
  unsigned long long* counter = (unsigned long long*)(scratch + kNaCountOff);
  auto run = [&]() -> shk_status {
    SHK_CUDA(cudaMemsetAsync(err, 0, 256 + 8, st));  // error flag and counter start at zero
    k_na_leaf_descs<<<(n_leaves + 255) / 256, 256, 0, st>>>(leaf_off, n_leaves, d);
    c.launches++;
    SHK_CUDA(cudaGetLastError());
    SHK_CUDA(cudaMemsetAsync(seeds_out, 0xFF, (size_t)n_leaves * 8, st));
    LeafSearchArgs a{d, n_leaves, leaf_keys, seed_start, (unsigned long long*)seeds_out, err,
                     counter, LeafCfg{4, 8, 2, 8}};
    SHK_TRY(launch_leaf_persistent_state(c, a, state));
    SHK_TRY(launch_orient(c, d, n_leaves, leaf_keys, (unsigned long long*)seeds_out, nullptr,
                          nullptr, f_out, err));
    uint32_t h_err = 0;
    SHK_CUDA(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, st));
    SHK_CUDA(cudaStreamSynchronize(st));
    if (h_err & kErrLeafSize) return fail(SHK_EINVAL, "a leaf has 0 or more than 64 keys");
    if (h_err & kErrSeedCap) return fail(SHK_ESEEDCAP, "a seed search reached 2^40");
    if (h_err) return fail(SHK_ECUDA, "internal: orientation of a leaf failed");
    return SHK_OK;
  };
  const shk_status s = run();
  if (s != SHK_OK) cudaStreamSynchronize(st);
  return s;
}
