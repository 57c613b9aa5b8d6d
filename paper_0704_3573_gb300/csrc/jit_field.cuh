// jit_field.cuh -- bit-sliced sweep of the random-field model (Eq. 2 with
// h_i = +-|h|, x_i = 1) specialised at run time for lane-uniform thresholds
// (one temperature).  Compiled by jit.cu with NVRTC after a preamble that
// defines IANUS_JIT_D, IANUS_JIT_ALGO, IANUS_JIT_R, IANUS_JIT_P2,
// IANUS_JIT_MINB and the truth tables:
//   IANUS_JIT_LUT0 / IANUS_JIT_LUT1: 32 bytes each, bit u of byte p = bit
//     (31 - p) of the threshold of class (u, f) for f = 0 / 1;
//   IANUS_JIT_ALWAYS0/1: bit u set where T(u, f) = 2^32;
//   IANUS_JIT_NEED0/1: bit u set where the class compares a random number.
//
// A lane's class is (u, f): u = unsatisfied bonds (3 bit-planes from the
// adder tree), f = [s_i h_i > 0] = ~(b ^ hb) with hb the lane bit of h_i < 0.
// The threshold bit of plane p is then one lop3 per f value (the table as
// immediate) and one lop3 select by f.  Plane pairs 0..7 use immediates,
// two Philox blocks in flight; pairs 8..15 (rare) read the tables from
// shared memory.  The class planes of every replica are computed first, so
// that all loads of a site are in flight together.
#include "common.cuh"

namespace ianus {
namespace jitf {

constexpr int D = IANUS_JIT_D;
constexpr int ALGO = IANUS_JIT_ALGO;
constexpr int R = IANUS_JIT_R;
constexpr bool P2 = IANUS_JIT_P2 != 0;
constexpr uint32_t kLut0[32] = {IANUS_JIT_LUT0};
constexpr uint32_t kLut1[32] = {IANUS_JIT_LUT1};
constexpr uint32_t kAlways0 = IANUS_JIT_ALWAYS0, kAlways1 = IANUS_JIT_ALWAYS1;
constexpr uint32_t kNeed0 = IANUS_JIT_NEED0, kNeed1 = IANUS_JIT_NEED1;
constexpr int kBlock = 256;

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

// f ? a : b, lane by lane
__device__ __forceinline__ uint64_t sel(uint64_t f, uint64_t a, uint64_t b) { return lop3c<0xCAu>(f, a, b); }

// threshold bit-plane of class (u, f) from two tables
template <uint32_t L0, uint32_t L1>
__device__ __forceinline__ uint64_t tab2(uint64_t u2, uint64_t u1, uint64_t u0, uint64_t f) {
  return sel(f, lop3c<L1>(u2, u1, u0), lop3c<L0>(u2, u1, u0));
}

struct Word {
  uint64_t u0, u1, u2, f, und, lt;
};

template <int M>
__device__ __forceinline__ void planes(Word& w, const uint4& x) {
  const uint64_t r0 = (uint64_t)x.x | ((uint64_t)x.y << 32);
  const uint64_t r1 = (uint64_t)x.z | ((uint64_t)x.w << 32);
  const uint64_t t0 = tab2<kLut0[2 * M], kLut1[2 * M]>(w.u2, w.u1, w.u0, w.f);
  const uint64_t c0 = w.und & t0 & ~r0;
  w.und &= ~(r0 ^ t0);
  const uint64_t t1 = tab2<kLut0[2 * M + 1], kLut1[2 * M + 1]>(w.u2, w.u1, w.u0, w.f);
  const uint64_t c1 = w.und & t1 & ~r1;
  w.und &= ~(r1 ^ t1);
  w.lt |= c0 | c1;
}

// pairs M..7, two Philox blocks at a time
template <int M>
__device__ __forceinline__ void pairs(Word& w, const BitsParams& p, const Tick& tk, uint32_t site, uint32_t c2) {
  if constexpr (M < 8) {
    if (w.und == 0ull) return;
    const uint4 xa = philox10(site, tk.lo, c2 | ((uint32_t)M << 24), tk.hi, p.keys);
    const uint4 xb = philox10(site, tk.lo, c2 | ((uint32_t)(M + 1) << 24), tk.hi, p.keys);
    planes<M>(w, xa);
    planes<M + 1>(w, xb);
    pairs<M + 2>(w, p, tk, site, c2);
  }
}

struct Decided {
  uint64_t und, lt;
};

// pairs 8..15 with the tables from shared memory (lut[0..31] for f = 0,
// lut[32..63] for f = 1)
__device__ __noinline__ Decided tail(uint64_t u0, uint64_t u1, uint64_t u2, uint64_t f, uint64_t und, uint64_t lt,
                                     const BitsParams& p, const Tick tk, uint32_t site, uint32_t c2,
                                     const uint8_t* lut) {
  uint64_t m[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) m[u] = ((u & 4) ? u2 : ~u2) & ((u & 2) ? u1 : ~u1) & ((u & 1) ? u0 : ~u0);
  for (uint32_t mm = 8; mm < 16u && und != 0ull; ++mm) {
    const uint4 x = philox10(site, tk.lo, c2 | (mm << 24), tk.hi, p.keys);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint64_t r = q == 0 ? ((uint64_t)x.x | ((uint64_t)x.y << 32)) : ((uint64_t)x.z | ((uint64_t)x.w << 32));
      const uint32_t t0 = lut[2u * mm + (uint32_t)q], t1 = lut[32u + 2u * mm + (uint32_t)q];
      uint64_t tb = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const uint64_t b0 = 0ull - (uint64_t)((t0 >> u) & 1u), b1 = 0ull - (uint64_t)((t1 >> u) & 1u);
        tb |= m[u] & ((f & b1) | (~f & b0));
      }
      lt |= und & tb & ~r;
      und &= ~(r ^ tb);
    }
  }
  return Decided{und, lt};
}

}  // namespace jitf
}  // namespace ianus

extern "C" __global__ void __launch_bounds__(ianus::jitf::kBlock, IANUS_JIT_MINB)
    ianus_jit_field_sweep(const ianus::BitsParams p, const uint64_t* __restrict__ hbits,
                          const uint8_t* __restrict__ lut_t) {
  using namespace ianus;
  using namespace ianus::jitf;
  __shared__ uint8_t s_lut[64];
  if (threadIdx.x < 64) s_lut[threadIdx.x] = lut_t[threadIdx.x];
  __syncthreads();
  const int gt = blockIdx.y;  // g * K + tslot (K = 1)
  const int g = gt / p.K, tslot = gt - g * p.K;
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  const Geom geom = p.geom;
  const uint32_t N = geom.N;
  const uint64_t* Jg = p.J + (uint64_t)g * D * N;
  const uint64_t* Hg = hbits + (uint64_t)g * N;
  uint64_t* s0 = p.spins + ((uint64_t)g * p.slots + (uint64_t)(tslot * R)) * N;
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
    const uint64_t hb = __ldg(Hg + n.self);
    Word w[R];
#pragma unroll
    for (int a = 0; a < R; ++a) {
      const uint64_t* sp = s0 + (uint64_t)a * N;
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
      count_unsat<D>(e, w[a].u0, w[a].u1, w[a].u2);
      w[a].f = ~(b ^ hb);
    }
#pragma unroll
    for (int a = 0; a < R; ++a) {
      Word& x = w[a];
      x.lt = tab2<kAlways0, kAlways1>(x.u2, x.u1, x.u0, x.f);
      x.und = tab2<kNeed0, kNeed1>(x.u2, x.u1, x.u0, x.f);
      const uint32_t c2 = (TAG_SPIN << 28) | ((uint32_t)(tslot * R + a) << 12) | (uint32_t)g;
      pairs<0>(x, p, tk, n.site, c2);
      if (x.und != 0ull) {
        const Decided d = tail(x.u0, x.u1, x.u2, x.f, x.und, x.lt, p, tk, n.site, c2, s_lut);
        x.lt = d.lt;
      }
      const uint64_t flip = (ALGO == 0) ? x.lt : ~x.lt;
      if (flip) s0[(uint64_t)a * N + n.self] ^= flip;
    }
  }
}
