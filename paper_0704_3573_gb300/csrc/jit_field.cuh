// jit_field.cuh -- bit-sliced sweep of the Ising-like models with fields
// (Eq. 2): the random-field model (h_i = +-|h|, x_i = 1) and, with
// IANUS_JIT_DILUTE, the diluted antiferromagnet in a field (x_i in {0,1}),
// specialised at run time for lane-uniform thresholds (one temperature).
// Compiled by jit.cu with NVRTC after a preamble that defines IANUS_JIT_D,
// IANUS_JIT_ALGO, IANUS_JIT_R, IANUS_JIT_P2, IANUS_JIT_MINB, IANUS_JIT_DILUTE
// and the truth tables IANUS_JIT_LUT<f><h> (32 bytes each), IANUS_JIT_ALWAYS<f><h>
// and IANUS_JIT_NEED<f><h> for f = [s_i h_i > 0] in {0,1} and h in {0,1}:
//   without dilution the class is (u, f), u = unsatisfied bonds (3 planes),
//     bit u of LUT<f>0 byte p = bit (31 - p) of T(u, f) (h = 1 unused);
//   with dilution it is (t, f), t = v + 2D = 8 h + k in 0..4D (4 planes),
//     bit k of LUT<f><h> byte p = bit (31 - p) of T(t, f).
// ALWAYS: T = 2^32; NEED: the class compares a random number.
//
// The threshold bit of plane p is a lop3 table per (f, h) and lop3 selects;
// plane pairs 0..7 use immediates with two Philox blocks in flight, pairs
// 8..15 (rare) read the tables from shared memory.  The class planes of every
// replica are computed first, so that all loads of a site are in flight
// together.  With dilution the local field is t = 2 sum(hi_j) + sum(lo_j),
// hi_j = x_j & ~e_j, lo_j = ~x_j (c_j + 1 = 2 hi_j + lo_j), and empty sites
// are never updated.
#include "common.cuh"

namespace ianus {
namespace jitf {

constexpr int D = IANUS_JIT_D;
constexpr int ALGO = IANUS_JIT_ALGO;
constexpr int R = IANUS_JIT_R;
constexpr bool P2 = IANUS_JIT_P2 != 0;
constexpr bool kDilute = IANUS_JIT_DILUTE != 0;
constexpr uint32_t kLut00[32] = {IANUS_JIT_LUT00};
constexpr uint32_t kLut01[32] = {IANUS_JIT_LUT01};
constexpr uint32_t kLut10[32] = {IANUS_JIT_LUT10};
constexpr uint32_t kLut11[32] = {IANUS_JIT_LUT11};
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

// s ? a : b, lane by lane
__device__ __forceinline__ uint64_t sel(uint64_t s, uint64_t a, uint64_t b) { return lop3c<0xCAu>(s, a, b); }

struct Word {
  uint64_t c0, c1, c2, c3, f, und, lt;  // class planes (u or t), t3 only with dilution
};

// threshold bit-plane of the class from the four tables
template <uint32_t L00, uint32_t L01, uint32_t L10, uint32_t L11>
__device__ __forceinline__ uint64_t tab(const Word& w) {
  if constexpr (kDilute) {
    const uint64_t a0 = sel(w.c3, lop3c<L01>(w.c2, w.c1, w.c0), lop3c<L00>(w.c2, w.c1, w.c0));
    const uint64_t a1 = sel(w.c3, lop3c<L11>(w.c2, w.c1, w.c0), lop3c<L10>(w.c2, w.c1, w.c0));
    return sel(w.f, a1, a0);
  } else {
    return sel(w.f, lop3c<L10>(w.c2, w.c1, w.c0), lop3c<L00>(w.c2, w.c1, w.c0));
  }
}

template <int M>
__device__ __forceinline__ void planes(Word& w, const uint4& x) {
  const uint64_t r0 = (uint64_t)x.x | ((uint64_t)x.y << 32);
  const uint64_t r1 = (uint64_t)x.z | ((uint64_t)x.w << 32);
  const uint64_t t0 = tab<kLut00[2 * M], kLut01[2 * M], kLut10[2 * M], kLut11[2 * M]>(w);
  const uint64_t d0 = w.und & t0 & ~r0;
  w.und &= ~(r0 ^ t0);
  const uint64_t t1 = tab<kLut00[2 * M + 1], kLut01[2 * M + 1], kLut10[2 * M + 1], kLut11[2 * M + 1]>(w);
  const uint64_t d1 = w.und & t1 & ~r1;
  w.und &= ~(r1 ^ t1);
  w.lt |= d0 | d1;
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

// pairs 8..15 with the tables from shared memory: lut[f * 64 + h * 32 + p]
__device__ __noinline__ Decided tail(uint64_t c0, uint64_t c1, uint64_t c2w, uint64_t c3, uint64_t f, uint64_t und,
                                     uint64_t lt, const BitsParams& p, const Tick tk, uint32_t site, uint32_t c2,
                                     const uint8_t* lut) {
  constexpr int NC = kDilute ? 16 : 8;
  uint64_t m[NC];
#pragma unroll
  for (int u = 0; u < NC; ++u) {
    m[u] = ((u & 4) ? c2w : ~c2w) & ((u & 2) ? c1 : ~c1) & ((u & 1) ? c0 : ~c0);
    if (kDilute) m[u] &= (u & 8) ? c3 : ~c3;
  }
  for (uint32_t mm = 8; mm < 16u && und != 0ull; ++mm) {
    const uint4 x = philox10(site, tk.lo, c2 | (mm << 24), tk.hi, p.keys);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint64_t r = q == 0 ? ((uint64_t)x.x | ((uint64_t)x.y << 32)) : ((uint64_t)x.z | ((uint64_t)x.w << 32));
      const uint32_t pl = 2u * mm + (uint32_t)q;
      uint64_t tb = 0;
#pragma unroll
      for (int u = 0; u < NC; ++u) {
        const uint32_t h = (uint32_t)u >> 3, k = (uint32_t)u & 7u;
        const uint64_t b0 = 0ull - (uint64_t)((lut[h * 32u + pl] >> k) & 1u);
        const uint64_t b1 = 0ull - (uint64_t)((lut[64u + h * 32u + pl] >> k) & 1u);
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
                          const uint64_t* __restrict__ xbits, const uint8_t* __restrict__ lut_t) {
  using namespace ianus;
  using namespace ianus::jitf;
  __shared__ uint8_t s_lut[128];
  dependent_launch_entry();
  if (threadIdx.x < 128) s_lut[threadIdx.x] = lut_t[threadIdx.x];
  __syncthreads();
#ifdef IANUS_JIT_L
  constexpr Geom geom = kJitGeom;
  const int g = blockIdx.y, tslot = 0;  // one temperature
  constexpr uint64_t slots = R;
#else
  const int gt = blockIdx.y;  // g * K + tslot (K = 1)
  const int g = gt / p.K, tslot = gt - g * p.K;
  const Geom geom = p.geom;
  const uint64_t slots = (uint64_t)p.slots;
#endif
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  const uint32_t N = geom.N;
  const uint64_t* Jg = p.J + (uint64_t)g * D * N;
  const uint64_t* Hg = hbits + (uint64_t)g * N;
  const uint64_t* Xg = xbits + (uint64_t)g * N;
  uint64_t* s0 = p.spins + ((uint64_t)g * slots + (uint64_t)(tslot * R)) * N;
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
    uint64_t xs = ~0ull, xw[2 * D], l0 = 0, l1 = 0, l2 = 0;
    if (kDilute) {
      xs = __ldg(Xg + n.self);
      xw[0] = __ldg(Xg + n.xp);
      xw[1] = __ldg(Xg + n.xm);
      xw[2] = __ldg(Xg + n.yp);
      xw[3] = __ldg(Xg + n.ym);
      if (D == 3) {
        xw[4] = __ldg(Xg + n.zp);
        xw[5] = __ldg(Xg + n.zm);
      }
      uint64_t lo[2 * D];
#pragma unroll
      for (int j = 0; j < 2 * D; ++j) lo[j] = ~xw[j];
      count_unsat<D>(lo, l0, l1, l2);
    }
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
      if (kDilute) {
        uint64_t hi[2 * D];
#pragma unroll
        for (int j = 0; j < 2 * D; ++j) hi[j] = xw[j] & ~e[j];
        uint64_t h0, h1, h2;
        count_unsat<D>(hi, h0, h1, h2);
        // t = 2 (h2 h1 h0) + (l2 l1 l0) <= 4D < 16
        const uint64_t k1 = h0 & l1;
        const uint64_t k2 = (h1 & l2) | (h1 & k1) | (l2 & k1);
        w[a].c0 = l0;
        w[a].c1 = h0 ^ l1;
        w[a].c2 = h1 ^ l2 ^ k1;
        w[a].c3 = h2 ^ k2;
      } else {
        count_unsat<D>(e, w[a].c0, w[a].c1, w[a].c2);
        w[a].c3 = 0;
      }
      w[a].f = ~(b ^ hb);
    }
#pragma unroll
    for (int a = 0; a < R; ++a) {
      Word& x = w[a];
      x.lt = tab<IANUS_JIT_ALWAYS00, IANUS_JIT_ALWAYS01, IANUS_JIT_ALWAYS10, IANUS_JIT_ALWAYS11>(x) & xs;
      x.und = tab<IANUS_JIT_NEED00, IANUS_JIT_NEED01, IANUS_JIT_NEED10, IANUS_JIT_NEED11>(x) & xs;
      const uint32_t c2 = (TAG_SPIN << 28) | ((uint32_t)(tslot * R + a) << 12) | (uint32_t)g;
      pairs<0>(x, p, tk, n.site, c2);
      if (x.und != 0ull) {
        const Decided d = tail(x.c0, x.c1, x.c2, x.c3, x.f, x.und, x.lt, p, tk, n.site, c2, s_lut);
        x.lt = d.lt;
      }
      const uint64_t flip = ((ALGO == 0) ? x.lt : ~x.lt) & xs;
      if (flip) s0[(uint64_t)a * N + n.self] ^= flip;
    }
  }
}
