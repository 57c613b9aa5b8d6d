// jit_sweep.cuh -- bit-sliced sweep specialised at run time for one set of
// lane-uniform acceptance thresholds (every lane of every slot at the same
// temperature).  Compiled by jit.cu with NVRTC for sm_103a after a preamble
// that defines:
//   IANUS_JIT_D, IANUS_JIT_ALGO (0 Metropolis, 1 heat bath), IANUS_JIT_R,
//   IANUS_JIT_P2 (L a power of two), IANUS_JIT_LUTS (32 truth tables),
//   IANUS_JIT_ALWAYS, IANUS_JIT_NEED.
//
// The update is the look-up-table compare of Sec. 3.2 in bit-sliced form (see
// k_msc.cu).  With thresholds fixed at compile time, the threshold bit of
// plane p for a lane of class u = (u2 u1 u0) is bit u of an 8-bit truth
// table, which is exactly one lop3 with that table as immediate per 32 bits,
// instead of seven AND-ORs with per-class masks.  Plane pairs 0..7 are
// unrolled with their tables as immediates; the rare pairs 8..15 (a word is
// still undecided after 16 planes with probability < 64 * 2^-16) use the
// per-class masks and the tables from shared memory.
#include "common.cuh"

namespace ianus {
namespace jit {

constexpr int D = IANUS_JIT_D;
constexpr int ALGO = IANUS_JIT_ALGO;
constexpr int R = IANUS_JIT_R;
constexpr bool P2 = IANUS_JIT_P2 != 0;
constexpr uint32_t kLut[32] = {IANUS_JIT_LUTS};
constexpr uint32_t kAlways = IANUS_JIT_ALWAYS;
constexpr uint32_t kNeed = IANUS_JIT_NEED;
constexpr int kBlock = 256;
constexpr int kUnrolled = 8;

template <uint32_t LUT>
__device__ __forceinline__ uint64_t lop3c(uint64_t a, uint64_t b, uint64_t c) {
  uint32_t lo, hi;
  asm("lop3.b32 %0, %1, %2, %3, %4;"
      : "=r"(lo)
      : "r"((uint32_t)a), "r"((uint32_t)b), "r"((uint32_t)c), "n"(LUT & 0xFFu));
  asm("lop3.b32 %0, %1, %2, %3, %4;"
      : "=r"(hi)
      : "r"((uint32_t)(a >> 32)), "r"((uint32_t)(b >> 32)), "r"((uint32_t)(c >> 32)), "n"(LUT & 0xFFu));
  return (uint64_t)lo | ((uint64_t)hi << 32);
}

struct Word {
  uint64_t u0, u1, u2, und, lt;
};

// One plane pair with compile-time tables: planes 2M and 2M+1.
template <int M>
__device__ __forceinline__ void pair(Word& w, const BitsParams& p, uint32_t site, uint32_t c2) {
  const uint4 x = philox10(site, p.t_lo, c2 | ((uint32_t)M << 24), p.t_hi, p.keys);
  const uint64_t r0 = (uint64_t)x.x | ((uint64_t)x.y << 32);
  const uint64_t r1 = (uint64_t)x.z | ((uint64_t)x.w << 32);
  const uint64_t t0 = lop3c<kLut[2 * M]>(w.u2, w.u1, w.u0);
  const uint64_t c0 = w.und & t0 & ~r0;  // decided at plane 2M with r < T
  w.und &= ~(r0 ^ t0);
  const uint64_t t1 = lop3c<kLut[2 * M + 1]>(w.u2, w.u1, w.u0);
  const uint64_t c1 = w.und & t1 & ~r1;
  w.und &= ~(r1 ^ t1);
  w.lt |= c0 | c1;
}

template <int M>
__device__ __forceinline__ void pairs(Word& w, const BitsParams& p, uint32_t site, uint32_t c2) {
  if constexpr (M < kUnrolled) {
    if (w.und == 0ull) return;
    pair<M>(w, p, site, c2);
    pairs<M + 1>(w, p, site, c2);
  }
}

// Pairs kUnrolled..15 with runtime tables (lut from shared memory).
__device__ __noinline__ void tail(Word& w, const BitsParams& p, uint32_t site, uint32_t c2, const uint8_t* lut) {
  uint64_t m[8];
#pragma unroll
  for (int u = 0; u < 8; ++u)
    m[u] = ((u & 4) ? w.u2 : ~w.u2) & ((u & 2) ? w.u1 : ~w.u1) & ((u & 1) ? w.u0 : ~w.u0);
  for (uint32_t mm = kUnrolled; mm < 16u && w.und != 0ull; ++mm) {
    const uint4 x = philox10(site, p.t_lo, c2 | (mm << 24), p.t_hi, p.keys);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint64_t r = q == 0 ? ((uint64_t)x.x | ((uint64_t)x.y << 32)) : ((uint64_t)x.z | ((uint64_t)x.w << 32));
      const uint32_t tab = lut[2u * mm + (uint32_t)q];
      uint64_t tb = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) tb |= m[u] & (0ull - (uint64_t)((tab >> u) & 1u));
      w.lt |= w.und & tb & ~r;
      w.und &= ~(r ^ tb);
    }
  }
}

}  // namespace jit
}  // namespace ianus

extern "C" __global__ void __launch_bounds__(ianus::jit::kBlock)
    ianus_jit_sweep(const ianus::BitsParams p, const uint8_t* __restrict__ lut_t) {
  using namespace ianus;
  using namespace ianus::jit;
  __shared__ uint8_t s_lut[32];
  if (threadIdx.x < 32) s_lut[threadIdx.x] = lut_t[threadIdx.x];
  __syncthreads();
  const int gt = blockIdx.y;  // g * K + tslot
  const int g = gt / p.K, tslot = gt - g * p.K;
  const Geom geom = p.geom;
  const uint32_t N = geom.N;
  const uint64_t* Jg = p.J + (uint64_t)g * D * N;
  const uint32_t w_begin = blockIdx.x * p.words_per_block;
  const uint32_t w_end = min(w_begin + p.words_per_block, geom.half);
  for (uint32_t wi = w_begin + threadIdx.x; wi < w_end; wi += kBlock) {
    const Nbr n = split_neighbours_t<P2>(geom, p.colour, wi);
    uint64_t jw[2 * D];
    jw[0] = __ldg(Jg + n.self);
    jw[1] = __ldg(Jg + n.xm);
    jw[2] = __ldg(Jg + N + n.self);
    jw[3] = __ldg(Jg + N + n.ym);
    if (D == 3) {
      jw[4] = __ldg(Jg + 2u * N + n.self);
      jw[5] = __ldg(Jg + 2u * N + n.zm);
    }
#pragma unroll
    for (int a = 0; a < R; ++a) {
      const int sigma = tslot * R + a;
      uint64_t* sp = p.spins + ((uint64_t)g * p.slots + sigma) * N;
      const uint64_t b = sp[n.self];
      uint64_t e[2 * D];
      e[0] = b ^ sp[n.xp] ^ jw[0];
      e[1] = b ^ sp[n.xm] ^ jw[1];
      e[2] = b ^ sp[n.yp] ^ jw[2];
      e[3] = b ^ sp[n.ym] ^ jw[3];
      if (D == 3) {
        e[4] = b ^ sp[n.zp] ^ jw[4];
        e[5] = b ^ sp[n.zm] ^ jw[5];
      }
      Word w;
      count_unsat<D>(e, w.u0, w.u1, w.u2);
      w.lt = kAlways ? lop3c<kAlways>(w.u2, w.u1, w.u0) : 0ull;
      w.und = lop3c<kNeed>(w.u2, w.u1, w.u0);
      const uint32_t c2 = (TAG_SPIN << 28) | ((uint32_t)sigma << 12) | (uint32_t)g;
      pairs<0>(w, p, n.site, c2);
      if (w.und != 0ull) tail(w, p, n.site, c2, s_lut);
      const uint64_t flip = (ALGO == 0) ? w.lt : ~w.lt;
      if (flip) sp[n.self] = b ^ flip;
    }
  }
}
