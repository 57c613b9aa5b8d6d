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

__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__device__ __forceinline__ uint32_t mul_hi(uint32_t a, uint32_t b) {
  uint32_t d;
  asm volatile("mul.hi.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

__device__ __forceinline__ uint32_t mul_lo(uint32_t a, uint32_t b) {
  uint32_t d;
  asm volatile("mul.lo.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

__device__ __forceinline__ uint32_t add3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("{ .reg .u32 t; add.u32 t, %1, %2; add.u32 %0, t, %3; }" : "=r"(d) : "r"(a), "r"(b), "r"(c));
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
  } else if (kind == 4) {  // independent lop3 and mad.wide chains side by side
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x[j] = lop3_xor(x[j], x[(j + 1) & 3], 0x5A5A5A5Au);
        w[4 + j] = mad_wide(x[4 + j], 0xD2511F53u, w[4 + j]);
      }
    }
  } else if (kind == 5) {  // 32-bit multiply-add
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = mad_lo(x[j], 0x9E3779B1u, x[(j + 1) & 7]);
    }
  } else if (kind == 6) {  // three-input add
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = add3(x[j], x[(j + 1) & 7], x[(j + 3) & 7]);
    }
  } else if (kind == 7) {  // independent lop3 and 32-bit multiply-add chains side by side
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x[j] = lop3_xor(x[j], x[(j + 1) & 3], 0x5A5A5A5Au);
        x[4 + j] = mad_lo(x[4 + j], 0x9E3779B1u, x[4 + ((j + 1) & 3)]);
      }
    }
  } else if (kind == 8) {  // 32-bit high product chains
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = mul_hi(x[j], 0xD2511F53u);
    }
  } else if (kind == 9) {  // independent lop3 and 32-bit high-product chains side by side
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x[j] = lop3_xor(x[j], x[(j + 1) & 3], 0x5A5A5A5Au);
        x[4 + j] = mul_hi(x[4 + j], 0xD2511F53u);
      }
    }
  } else if (kind == 10) {  // Philox blocks with the products as separate high and low halves
    for (int i = 0; i < kIters / 16; ++i) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        uint32_t c0 = x[4 * j], c1 = x[4 * j + 1], c2 = x[4 * j + 2], c3 = x[4 * j + 3];
#pragma unroll
        for (int r = 0; r < 10; ++r) {
          const uint32_t h0 = mul_hi(c0, 0xD2511F53u), l0 = mul_lo(c0, 0xD2511F53u);
          const uint32_t h1 = mul_hi(c2, 0xCD9E8D57u), l1 = mul_lo(c2, 0xCD9E8D57u);
          c0 = lop3_xor(h1, c1, keys.k0[r]);
          c2 = lop3_xor(h0, c3, keys.k1[r]);
          c1 = l1;
          c3 = l0;
        }
        x[4 * j] = c0;
        x[4 * j + 1] = c1;
        x[4 * j + 2] = c2;
        x[4 * j + 3] = c3;
      }
    }
  } else if (kind >= 11) {
    // Philox blocks with each product (11, 13) or the first product of a
    // round (14) as a separate high multiply and a low multiply-add that
    // cannot be merged with it (lo(a M) = a (M - 1) + a), or both as
    // 64-bit products (12); 12..14 also run 24 lop3.b32 of an independent
    // chain per block, as a sweep does besides its random numbers.
    uint32_t y0 = x[0] ^ 0x1234u, y1 = x[1] ^ 0x5678u;
    for (int i = 0; i < kIters / 16; ++i) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        uint32_t c0 = x[4 * j], c1 = x[4 * j + 1], c2 = x[4 * j + 2], c3 = x[4 * j + 3];
#pragma unroll
        for (int r = 0; r < 10; ++r) {
          uint32_t h0, l0, h1, l1;
          if (kind == 12) {
            const uint64_t p0 = mad_wide(c0, 0xD2511F53u, 0ull), p1 = mad_wide(c2, 0xCD9E8D57u, 0ull);
            h0 = (uint32_t)(p0 >> 32);
            l0 = (uint32_t)p0;
            h1 = (uint32_t)(p1 >> 32);
            l1 = (uint32_t)p1;
          } else if (kind == 14) {
            const uint64_t p1 = mad_wide(c2, 0xCD9E8D57u, 0ull);
            h0 = mul_hi(c0, 0xD2511F53u);
            l0 = mad_lo(c0, 0xD2511F52u, c0);
            h1 = (uint32_t)(p1 >> 32);
            l1 = (uint32_t)p1;
          } else {
            h0 = mul_hi(c0, 0xD2511F53u);
            l0 = mad_lo(c0, 0xD2511F52u, c0);
            h1 = mul_hi(c2, 0xCD9E8D57u);
            l1 = mad_lo(c2, 0xCD9E8D56u, c2);
          }
          c0 = lop3_xor(h1, c1, keys.k0[r]);
          c2 = lop3_xor(h0, c3, keys.k1[r]);
          c1 = l1;
          c3 = l0;
          if (kind != 11 && (r & 3) != 3) {  // 24 lop3 per block beside the block's own
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              y0 = lop3_xor(y0, y1, 0x0F0F0F0Fu);
              y1 = lop3_xor(y1, y0, 0x33333333u);
            }
          }
        }
        x[4 * j] = c0;
        x[4 * j + 1] = c1;
        x[4 * j + 2] = c2;
        x[4 * j + 3] = c3;
      }
    }
    x[5] ^= y0 ^ y1;
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
  if (kind < 0 || kind > 14 || blocks_per_sm < 1 || blocks_per_sm > 8 || !out) return 1;
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
  if (kind == 0 || kind == 1 || (kind >= 4 && kind <= 9))
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
