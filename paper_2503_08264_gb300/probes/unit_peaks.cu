// Per-SM issue rates of the units the contraction kernels' rooflines use,
// measured on the GPU they run on (a standalone program; not part of libqem):
//   ex2.approx.ftz.f32 (the exponential unit), fma.rn.f32 and fma.rn.f32x2
//   (the FP32 pipe), and tcgen05.mma (M = 128, K = 16 BF16 / K = 8 TF32,
//   N = 128 and 256) from one issuing thread.
// Method: every SM runs the same fixed work; a block's clock64 span gives SM
// cycles (independent of the clock frequency), so rate = operations per SM /
// cycles of the slowest block.  The ALU probes run 8 blocks x 256 threads
// per SM (full occupancy) with 8 independent dependency chains per thread;
// the MMA probe issues 4096 MMAs per SM, unrolled in groups of 8, from
// zero-filled shared operands into TMEM, and times them to the commit of the
// last one.  Prints one JSON object.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256, 8) k_ex2(float* out, long long* cyc, int nit) {
  float x[kChains];
  for (int c = 0; c < kChains; ++c) x[c] = 0.01f * (threadIdx.x + c);
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < nit; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(-x[c]));
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(256, 8) k_fma(float* out, long long* cyc, int nit) {
  float x[kChains];
  for (int c = 0; c < kChains; ++c) x[c] = 0.01f * (threadIdx.x + c);
  const float a = 0.999f, b = 0.001f;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < nit; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(a), "f"(b));
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(256, 8) k_fma2(float* out, long long* cyc, int nit) {
  float x[2 * kChains];
  for (int c = 0; c < 2 * kChains; ++c) x[c] = 0.01f * (threadIdx.x + c);
  const float a = 0.999f, b = 0.001f;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < nit; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c)
      asm volatile(
          "{\n .reg .b64 p, q, r;\n mov.b64 p, {%0, %1};\n mov.b64 q, {%2, %2};\n mov.b64 r, {%3, %3};\n"
          " fma.rn.f32x2 p, p, q, r;\n mov.b64 {%0, %1}, p;\n}\n"
          : "+f"(x[2 * c]), "+f"(x[2 * c + 1])
          : "f"(a), "f"(b));
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
  for (int c = 0; c < 2 * kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t ph, long long lim) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(ph)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > lim) return false;
  }
}

__device__ __forceinline__ uint64_t sdesc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint32_t a = smem_u32(p);
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

template <bool TF32>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (TF32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

// One CTA per SM (120 KB of shared memory); operands 128 x 128 B (A) and
// 256 x 128 B (B) rows, canonical K-major no-swizzle layout, zero-filled.
template <bool TF32>
__global__ void __launch_bounds__(128, 1) k_mma(int n, int nm, long long* cyc, int* err, long long lim) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* base = (uint8_t*)(((uintptr_t)sm + 1023) & ~(uintptr_t)1023);
  uint8_t* A = base;
  uint8_t* B = base + 16384;
  uint64_t* bar = (uint64_t*)(base + 16384 + 32768);
  uint32_t* tslot = (uint32_t*)(bar + 1);
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (16384 + 32768) / 16; i += blockDim.x) ((uint4*)base)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  if (threadIdx.x == 0) {
    const uint32_t fmt = TF32 ? 2u : 1u;
    const uint32_t id = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint64_t ad = sdesc(A, 128, 1024), bd = sdesc(B, 128, 1024);
    const long long t0 = clock64();
    for (int g = 0; g < nm / 8; ++g) {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        mma<TF32>(tmem, ad + (uint64_t)((j & 3) * 16), bd + (uint64_t)((j & 3) * 16), id, (g > 0 || j > 0) ? 1u : 0u);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
    const bool ok = mbar_wait(bar, 0, lim);
    cyc[blockIdx.x] = clock64() - t0;
    if (!ok) atomicOr(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

long long max_cycles(const long long* d, int n, long long* host) {
  cudaMemcpy(host, d, sizeof(long long) * n, cudaMemcpyDeviceToHost);
  long long mx = 0;
  for (int i = 0; i < n; ++i) mx = host[i] > mx ? host[i] : mx;
  return mx;
}

}  // namespace

int main() {
  int dev = 0, sms = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  const int threads = 256, per_sm = 8, blocks = sms * per_sm, nit = 20000;
  float* out = nullptr;
  long long* cyc = nullptr;
  int* err = nullptr;
  if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess ||
      cudaMalloc(&cyc, sizeof(long long) * blocks) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess)
    return 1;
  cudaMemset(err, 0, sizeof(int));
  long long* host = new long long[blocks];
  const double ops_sm = (double)per_sm * threads * nit * kChains;  // lane-ops per SM (x2 for f32x2)
  double rate[3];
  for (int kind = 0; kind < 3; ++kind) {
    double best = 0.0;
    for (int rep = 0; rep < 3; ++rep) {
      if (kind == 0) k_ex2<<<blocks, threads>>>(out, cyc, nit);
      else if (kind == 1) k_fma<<<blocks, threads>>>(out, cyc, nit);
      else k_fma2<<<blocks, threads>>>(out, cyc, nit);
      if (cudaDeviceSynchronize() != cudaSuccess) return 2;
      const double r = ops_sm * (kind == 2 ? 2.0 : 1.0) / (double)max_cycles(cyc, blocks, host);
      best = r > best ? r : best;
    }
    rate[kind] = best;
  }
  cudaFuncSetAttribute(k_mma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 120 * 1024);
  cudaFuncSetAttribute(k_mma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 120 * 1024);
  const int nm = 4096;
  double mma_cyc[2][2];
  for (int tf = 0; tf < 2; ++tf)
    for (int ni = 0; ni < 2; ++ni) {
      const int n = ni ? 256 : 128;
      if (tf) k_mma<true><<<sms, 128, 120 * 1024>>>(n, nm, cyc, err, (long long)khz * 2000);
      else k_mma<false><<<sms, 128, 120 * 1024>>>(n, nm, cyc, err, (long long)khz * 2000);
      if (cudaDeviceSynchronize() != cudaSuccess) return 2;
      mma_cyc[tf][ni] = (double)max_cycles(cyc, sms, host) / nm;
    }
  int e = 0;
  cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost);
  printf("{\"sms\": %d, \"clock_attr_mhz\": %.0f, \"ex2_per_clk_sm\": %.2f, \"fma_f32_lanes_per_clk_sm\": %.2f, "
         "\"fma_f32x2_lanes_per_clk_sm\": %.2f, \"mma_bf16_m128_k16_cycles\": {\"n128\": %.1f, \"n256\": %.1f}, "
         "\"mma_tf32_m128_k8_cycles\": {\"n128\": %.1f, \"n256\": %.1f}, \"mma_wait_expired\": %d}\n",
         sms, khz / 1000.0, rate[0], rate[1], rate[2], mma_cyc[0][0], mma_cyc[0][1], mma_cyc[1][0], mma_cyc[1][1], e);
  return e ? 3 : 0;
}
