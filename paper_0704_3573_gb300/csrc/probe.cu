// probe.cu -- integer-throughput probe (libianus_probe.so); see
// include/ianus_probe.h.  Each thread runs eight independent dependency
// chains so that latency is hidden and the issue rate of the probed
// instruction is what limits the loop.
#include <algorithm>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ianus_probe.h"
#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kIters = 4096;

__device__ __forceinline__ uint32_t lop3_xor(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__device__ __forceinline__ uint64_t mad_wide(uint32_t a, uint32_t b, uint64_t c) {
  uint64_t d;
  asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

__device__ __forceinline__ uint32_t smid() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// rec[3*block] = smid, rec[3*block+1] = start cycle, rec[3*block+2] = end cycle
__global__ void __launch_bounds__(kThreads) k_probe(int kind, uint32_t seed, uint64_t* rec, uint32_t* sink,
                                                   ianus::PhiloxKeys keys) {
  uint32_t x[8];
  uint64_t w[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    x[j] = seed * (threadIdx.x + 1u) + 0x9E3779B9u * (uint32_t)j;
    w[j] = x[j];
  }
  __syncthreads();
  const uint64_t t0 = clock64();
  if (kind == 0) {
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = lop3_xor(x[j], x[(j + 1) & 7], x[(j + 3) & 7]);
    }
  } else if (kind == 1) {
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) w[j] = mad_wide(x[j], 0xD2511F53u, w[j]);
    }
  } else if (kind == 2) {
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        w[j] = mad_wide(x[j], 0xCD9E8D57u, w[j]);
        x[j] = lop3_xor(x[j], (uint32_t)w[j], 0x12345u);
        x[j] = lop3_xor(x[j], (uint32_t)(w[j] >> 32), 0x6789u);
      }
    }
  } else {
    for (int i = 0; i < kIters / 16; ++i) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const uint4 r = ianus::philox10(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3], keys);
        x[4 * j] = r.x;
        x[4 * j + 1] = r.y;
        x[4 * j + 2] = r.z;
        x[4 * j + 3] = r.w;
      }
    }
  }
  const uint64_t t1 = clock64();
  __syncthreads();
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) acc ^= x[j] ^ (uint32_t)w[j] ^ (uint32_t)(w[j] >> 32);
  if (acc == 0x5eed5eedu) sink[0] = acc;  // keeps the chains alive
  if (threadIdx.x == 0) {
    rec[3 * blockIdx.x] = smid();
    rec[3 * blockIdx.x + 1] = t0;
    rec[3 * blockIdx.x + 2] = t1;
  }
}

}  // namespace

extern "C" int ianus_probe_int(int kind, int blocks_per_sm, double* out) {
  if (kind < 0 || kind > 3 || blocks_per_sm < 1 || blocks_per_sm > 8 || !out) return 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 3;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 3;
  const int blocks = sms * blocks_per_sm;
  uint64_t* rec = nullptr;
  uint32_t* sink = nullptr;
  if (cudaMalloc(&rec, 3 * blocks * sizeof(uint64_t)) != cudaSuccess) return 3;
  if (cudaMalloc(&sink, sizeof(uint32_t)) != cudaSuccess) {
    cudaFree(rec);
    return 3;
  }
  const ianus::PhiloxKeys keys = ianus::make_keys(0x1234abcdull);
  k_probe<<<blocks, kThreads>>>(kind, 7u, rec, sink, keys);  // warm-up
  k_probe<<<blocks, kThreads>>>(kind, 11u, rec, sink, keys);
  std::vector<uint64_t> h(3 * (size_t)blocks);
  cudaError_t e = cudaMemcpy(h.data(), rec, h.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost);
  cudaFree(rec);
  cudaFree(sink);
  if (e != cudaSuccess) return 3;
  double ops_per_block;
  if (kind == 0 || kind == 1)
    ops_per_block = (double)kThreads * kIters * 8;
  else if (kind == 2)
    ops_per_block = (double)kThreads * kIters * 8 * 3;
  else
    ops_per_block = (double)kThreads * (kIters / 16) * 2;
  // per SM: all its blocks' work over (last end - first start) on its own clock
  std::vector<uint64_t> t0(1024, ~0ull), t1(1024, 0ull);
  std::vector<int> nb(1024, 0);
  for (int b = 0; b < blocks; ++b) {
    const uint64_t sm = h[3 * b] & 1023u;
    t0[sm] = std::min(t0[sm], h[3 * b + 1]);
    t1[sm] = std::max(t1[sm], h[3 * b + 2]);
    nb[sm] += 1;
  }
  std::vector<double> rate;
  for (int sm = 0; sm < 1024; ++sm)
    if (nb[sm] > 0 && t1[sm] > t0[sm]) rate.push_back(nb[sm] * ops_per_block / (double)(t1[sm] - t0[sm]));
  if (rate.empty()) return 3;
  std::sort(rate.begin(), rate.end());
  *out = rate[rate.size() / 2];
  return 0;
}
