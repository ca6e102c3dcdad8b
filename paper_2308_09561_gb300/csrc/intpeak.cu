// intpeak.cu -- integer-issue microbenchmark: the lane-operation rate this GPU
// sustains for the instruction classes the leaf search is made of.
//
// The leaf kernels are bound by integer issue, not by memory: one key-seed
// evaluation is a handful of 32-bit logic, shift and multiply operations.  The
// nominal ceiling is one warp instruction per scheduler and cycle (SMs x 4 x
// 32 lanes x clock).  These kernels measure what is reached in practice with
// dependent-chain-free code: every thread advances 8 independent chains, so
// issue, not latency, is the limit.
//   mix 0: 3-input logic op + funnel shift (the ALU pipe alone)
//   mix 1: 32-bit multiply-add (the FMA pipe alone)
//   mix 2: multiply-add + 3-input logic op, 1:1 (both pipes)
//   mix 3: the plain leaf hash and 64-bit coverage-mask update (paper Sec. 4,
//          Filter by Bit Mask) for 8 seeds x 16 keys held in registers; the
//          count is key-seed evaluations instead of operations.
// Inline PTX pins the operation of mixes 0-2 so that the compiler can neither
// fold nor reorder them away.
#include "kernels.cuh"

namespace shk {

__device__ __forceinline__ uint32_t lop3_xor(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__device__ __forceinline__ uint32_t shf_l(uint32_t a, uint32_t b) {
  uint32_t d;
  asm volatile("shf.l.wrap.b32 %0, %1, %2, 5;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

constexpr int kChains = 8;
constexpr int kMixKeys = 16;

template <int MIX>
__global__ void __launch_bounds__(256) k_int_peak(uint32_t iters, uint32_t salt, uint32_t* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t v[kChains], u[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) {
    v[c] = (uint32_t)mix64(salt + tid * 8u + c);
    u[c] = (uint32_t)mix64(~(salt + tid * 8u + c)) | 1u;
  }
  if (MIX <= 2) {
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
      for (int c = 0; c < kChains; c++) {
        if (MIX == 0) {
          v[c] = lop3_xor(v[c], u[c], it);
          v[c] = shf_l(v[c], u[c]);
        } else if (MIX == 1) {
          v[c] = imad(v[c], u[c], it);
          v[c] = imad(v[c], u[c], tid);
        } else {
          v[c] = imad(v[c], u[c], it);
          v[c] = lop3_xor(v[c], u[c], tid);
        }
      }
    }
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) r ^= v[c];
    if (r == 0x9E3779B9u) sink[tid] = r;  // keeps the chains live
  } else {
    // 16 leaf keys in registers (xor input, multiplier), 8 seed constants;
    // m = 64 cells, 64-bit coverage masks as in the leaf kernel
    uint32_t xl[kMixKeys], mu[kMixKeys];
#pragma unroll
    for (int k = 0; k < kMixKeys; k++) {
      const uint64_t x = mix64(salt * 977u + tid * 16u + k);
      xl[k] = (uint32_t)x;
      mu[k] = (uint32_t)(x >> 32) | 1u;
    }
    const uint32_t m = 48 + (salt & 15u), m1 = m - 1;  // runtime leaf size, as in the kernel
    uint64_t acc = 0;
    for (uint32_t it = 0; it < iters; it++) {
      uint64_t mask[kChains];
#pragma unroll
      for (int c = 0; c < kChains; c++) mask[c] = 0;
#pragma unroll
      for (int k = 0; k < kMixKeys; k++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) {
          const uint32_t a = (xl[k] ^ v[c]) * mu[k] + u[c];
          const uint64_t w = (uint64_t)a * m;
          const uint32_t h0 = (uint32_t)(w >> 32);
          const uint32_t t = __umulhi((uint32_t)w, m1);
          const uint32_t h1 = t + (t >= h0 ? 1u : 0u);
          mask[c] |= (1ull << h0) | (1ull << h1);
        }
      }
#pragma unroll
      for (int c = 0; c < kChains; c++) {
        v[c] += (uint32_t)mask[c];  // next "seed" depends on this one's mask
        acc ^= mask[c];
      }
    }
    if (acc == 0x9E3779B97F4A7C15ull) sink[tid] = (uint32_t)acc;
  }
}

// lane operations (mix 3: key-seed evaluations) per thread and iteration
static double units_per_iter(uint32_t mix) {
  return mix <= 2 ? 2.0 * kChains : (double)kChains * kMixKeys;
}

static shk_status int_peak_impl(uint32_t mix, uint32_t iters, double* rate, double* ms_out,
                                cudaStream_t st) {
  if (mix > 3 || iters == 0 || !rate) return fail(SHK_EINVAL, "bad argument");
  Ctx c(st);
  SHK_TRY(init_ctx(c));
  void (*kern)(uint32_t, uint32_t, uint32_t*) =
      mix == 0 ? k_int_peak<0> : (mix == 1 ? k_int_peak<1> : (mix == 2 ? k_int_peak<2> : k_int_peak<3>));
  int per_sm = 0;
  SHK_TRY(blocks_per_sm((const void*)kern, 256, 0, &per_sm));
  if (per_sm < 1) per_sm = 1;
  const uint32_t blocks = (uint32_t)(c.num_sms * per_sm);
  uint32_t* sink;
  SHK_TRY(c.arena.alloc(&sink, (size_t)blocks * 256));
  cudaEvent_t e0, e1;
  SHK_CUDA(cudaEventCreate(&e0));
  SHK_CUDA(cudaEventCreate(&e1));
  float best = 0;
  for (int run = -1; run < 3; run++) {  // run -1: warm-up
    SHK_CUDA(cudaEventRecord(e0, st));
    kern<<<blocks, 256, 0, st>>>(iters, 0x5EEDu + (uint32_t)run, sink);
    SHK_CUDA(cudaEventRecord(e1, st));
    SHK_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    SHK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (run >= 0 && (best == 0 || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SHK_CUDA(cudaGetLastError());
  const double units = (double)blocks * 256 * iters * units_per_iter(mix);
  *rate = best > 0 ? units / (best * 1e-3) : 0;
  if (ms_out) *ms_out = best;
  return SHK_OK;
}

}  // namespace shk

extern "C" shk_status shk_int_issue_rate(uint32_t mix, uint32_t iters, double* rate,
                                         double* ms, void* cuda_stream) {
  return shk::no_throw(
      [&] { return shk::int_peak_impl(mix, iters, rate, ms, (cudaStream_t)cuda_stream); });
}
