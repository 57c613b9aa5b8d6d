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
// instead of seven AND-ORs with per-class masks.  Plane pairs 0..3 use their
// tables as immediates; the rarer later pairs use per-class masks and the
// tables from shared memory.
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
// IANUS_JIT_BLOCK: threads per block (default 256).
#ifndef IANUS_JIT_BLOCK
#define IANUS_JIT_BLOCK 256
#endif
constexpr int kBlock = IANUS_JIT_BLOCK;
// IANUS_JIT_L, IANUS_JIT_LH, IANUS_JIT_LL: the lattice side and the base-2
// logarithms of L/2 and L (0 when L is not a power of two).  The kernel runs
// at one temperature (n_temps = 1, so slots = R); with the geometry fixed at
// compile time the index arithmetic folds, and the replicas' words of a
// site, N words apart, are reached by constant offsets from one address.
// IANUS_JIT_MODE 0: all plane pairs in lockstep across the warp (pairs
// 0..7 with immediate tables, then run-time tables); 1: pairs 0..PHASEA-1 in
// lockstep, then a per-warp queue (below); 2 (two replicas): as 0, with the
// two replicas' plane loops interleaved in one thread, so that two
// independent Philox chains are in flight (a decided replica's extra block is
// masked out by its undecided-lane word).  IANUS_JIT_MINB: blocks per SM the
// register allocation must allow.
constexpr int kMode = IANUS_JIT_MODE;
constexpr int kPhaseA = IANUS_JIT_PHASEA;
constexpr int kUnrolled = kMode == 1 ? kPhaseA : 8;
// IANUS_JIT_GROUP 2: the Philox blocks of two consecutive plane pairs are
// computed back to back before either is compared, so that two independent
// round chains are in flight.  A warp runs a pair whenever any of its words
// needs it, so the second block is almost never extra issue work.
#ifndef IANUS_JIT_GROUP
#define IANUS_JIT_GROUP 1
#endif
constexpr int kGroup = IANUS_JIT_GROUP;
// IANUS_JIT_JRELOAD 1: each replica reads its coupling words again (L1 hits)
// instead of keeping the six words of the site live across the plane loop.
#ifndef IANUS_JIT_JRELOAD
#define IANUS_JIT_JRELOAD 0
#endif
constexpr bool kJReload = IANUS_JIT_JRELOAD != 0;
// IANUS_JIT_UFIRST 1: the class planes (u2 u1 u0) of every replica of the
// site are computed before the first plane loop, so that all of the site's
// loads are in flight together (one L2 round trip per site, not per replica).
#ifndef IANUS_JIT_UFIRST
#define IANUS_JIT_UFIRST 0
#endif
constexpr bool kUFirst = IANUS_JIT_UFIRST != 0 && kMode != 2;

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

// Planes 2M and 2M+1 from their Philox block x, compile-time tables.
template <int M>
__device__ __forceinline__ void planes(Word& w, const uint4& x) {
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

// One plane pair: planes 2M and 2M+1.
template <int M>
__device__ __forceinline__ void pair(Word& w, const BitsParams& p, const Tick& tk, uint32_t site, uint32_t c2) {
  const uint4 x = philox10(site, tk.lo, c2 | ((uint32_t)M << 24), tk.hi, p.keys);
  planes<M>(w, x);
}

template <int M>
__device__ __forceinline__ void pairs2(Word& w0, Word& w1, const BitsParams& p, const Tick& tk, uint32_t site,
                                       uint32_t c2a, uint32_t c2b) {
  if constexpr (M < kUnrolled) {
    if ((w0.und | w1.und) == 0ull) return;
    pair<M>(w0, p, tk, site, c2a);
    pair<M>(w1, p, tk, site, c2b);
    pairs2<M + 1>(w0, w1, p, tk, site, c2a, c2b);
  }
}

// Pairs M..END-1 in lockstep with immediate tables (two at a time with
// IANUS_JIT_GROUP 2).
template <int M, int END>
__device__ __forceinline__ void pairs_range(Word& w, const BitsParams& p, const Tick& tk, uint32_t site, uint32_t c2) {
  if constexpr (M < END) {
    if (w.und == 0ull) return;
    if constexpr (kGroup == 2 && M + 1 < END) {
      const uint4 xa = philox10(site, tk.lo, c2 | ((uint32_t)M << 24), tk.hi, p.keys);
      const uint4 xb = philox10(site, tk.lo, c2 | ((uint32_t)(M + 1) << 24), tk.hi, p.keys);
      planes<M>(w, xa);
      planes<M + 1>(w, xb);
      pairs_range<M + 2, END>(w, p, tk, site, c2);
    } else {
      pair<M>(w, p, tk, site, c2);
      pairs_range<M + 1, END>(w, p, tk, site, c2);
    }
  }
}

template <int M>
__device__ __forceinline__ void pairs(Word& w, const BitsParams& p, const Tick& tk, uint32_t site, uint32_t c2) {
  pairs_range<M, kUnrolled>(w, p, tk, site, c2);
}

// Modes 0 and 2 (and the queued words of mode 1): pairs 8..15 of one word,
// run-time tables.  Rarely entered; the word is passed and returned by value
// so that the caller's state never has to live in local memory.
struct Decided {
  uint64_t und, lt;
};

__device__ __noinline__ Decided tail_lockstep(uint64_t u0, uint64_t u1, uint64_t u2, uint64_t und, uint64_t lt,
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
      const uint32_t tab = lut[2u * mm + (uint32_t)q];
      uint64_t tb = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) tb |= m[u] & (0ull - (uint64_t)((tab >> u) & 1u));
      lt |= und & tb & ~r;
      und &= ~(r ^ tb);
    }
  }
  return Decided{und, lt};
}

__device__ __forceinline__ void finish_tail(Word& w, const BitsParams& p, const Tick& tk, uint32_t site, uint32_t c2,
                                            const uint8_t* lut) {
  if (w.und != 0ull) {
    const Decided d = tail_lockstep(w.u0, w.u1, w.u2, w.und, w.lt, p, tk, site, c2, lut);
    w.und = d.und;
    w.lt = d.lt;
  }
}

// ---- compaction of the lazy plane loop (mode 1) ----
//
// A warp's 32 words need different numbers of plane pairs (a 64-lane word is
// decided after ~3.9 pairs on average, the slowest of 32 words after ~6.4).
// Pairs 0..PHASEA-1 run in lockstep; the few words still undecided (about a
// fifth after 4 pairs) are appended to a per-warp queue in shared memory, and
// whenever 32 are queued the warp finishes them together: pairs PHASEA..7
// in lockstep with immediate tables, then the run-time tail.  Every word is
// written exactly once, by whichever lane finishes it; during a colour-c pass
// only colour-c words are written, so the order does not matter.

constexpr int kWarps = kBlock / 32;
constexpr uint32_t kQ = 64;  // queue capacity: < 32 left + <= 32 pushed

struct Queue {
  uint64_t u0[kQ], u1[kQ], u2[kQ], und[kQ], lt[kQ];
  uint32_t self[kQ], site[kQ], tag[kQ];  // tag = replica
};

struct Ctx {
  const BitsParams* p;
  int g, tslot;
  const uint8_t* lut;  // shared-memory copy of the 32 tables
  Tick tk;
  uint64_t* sp0;       // spins of the block's first replica; replica a is a * N further
};

__device__ __forceinline__ uint32_t sigma_c2(const Ctx& c, uint32_t a) {
  const uint32_t sigma = (uint32_t)(c.tslot * R) + a;
  return (TAG_SPIN << 28) | (sigma << 12) | (uint32_t)c.g;
}

__device__ __forceinline__ uint32_t sites_of(const BitsParams& p) {
#ifdef IANUS_JIT_L
  return kJitSites;
#else
  return p.geom.N;
#endif
}

__device__ __forceinline__ void finish(const Ctx& c, uint32_t self, uint32_t a, const Word& w) {
  uint64_t* sp = c.sp0 + (uint64_t)a * sites_of(*c.p);
  const uint64_t flip = (ALGO == 0) ? w.lt : ~w.lt;
  if (flip) sp[self] ^= flip;
}


// Warp-wide append of the lanes with pred set; n is warp-uniform.
__device__ __forceinline__ void push(Queue& q, uint32_t& n, bool pred, const Word& w, uint32_t self, uint32_t site,
                                     uint32_t tag) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t m = __ballot_sync(0xffffffffu, pred);
  if (pred) {
    const uint32_t i = n + __popc(m & ((1u << lane) - 1u));
    q.u0[i] = w.u0;
    q.u1[i] = w.u1;
    q.u2[i] = w.u2;
    q.und[i] = w.und;
    q.lt[i] = w.lt;
    q.self[i] = self;
    q.site[i] = site;
    q.tag[i] = tag;
  }
  n += __popc(m);
  __syncwarp();
}

// Finish the top `take` (<= 32) queued words.
__device__ __forceinline__ void round(Queue& q, uint32_t& n, uint32_t take, const Ctx& c) {
  const uint32_t lane = threadIdx.x & 31u;
  const bool has = lane < take;
  Word w;
  uint32_t self = 0, site = 0, a = 0;
  w.u0 = w.u1 = w.u2 = w.und = w.lt = 0;
  if (has) {
    const uint32_t i = n - take + lane;
    w.u0 = q.u0[i];
    w.u1 = q.u1[i];
    w.u2 = q.u2[i];
    w.und = q.und[i];
    w.lt = q.lt[i];
    self = q.self[i];
    site = q.site[i];
    a = q.tag[i];
  }
  __syncwarp();
  n -= take;
  const uint32_t c2 = sigma_c2(c, a);
  pairs_range<kPhaseA, 8>(w, *c.p, c.tk, site, c2);
  finish_tail(w, *c.p, c.tk, site, c2, c.lut);
  if (has) finish(c, self, a, w);
}

}  // namespace jit
}  // namespace ianus

extern "C" __global__ void __launch_bounds__(ianus::jit::kBlock, IANUS_JIT_MINB)
    ianus_jit_sweep(const ianus::BitsParams p, const uint8_t* __restrict__ lut_t) {
  using namespace ianus;
  using namespace ianus::jit;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ uint8_t s_lut[32];
  dependent_launch_entry();
  if (threadIdx.x < 32) s_lut[threadIdx.x] = lut_t[threadIdx.x];
  __syncthreads();
  Queue* q = reinterpret_cast<Queue*>(dyn_smem) + (threadIdx.x >> 5);  // one queue per warp (mode 1)
  uint32_t nq = 0;
  Ctx c;
  c.p = &p;
#ifdef IANUS_JIT_L
  constexpr Geom geom = kJitGeom;
  c.g = blockIdx.y;  // one temperature: blockIdx.y = g
  c.tslot = 0;
  constexpr uint64_t slots = R;
#else
  const int gt = blockIdx.y;  // g * K + tslot
  c.g = gt / p.K;
  c.tslot = gt - c.g * p.K;
  const Geom geom = p.geom;
  const uint64_t slots = (uint64_t)p.slots;
#endif
  c.lut = s_lut;
  c.tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  const uint32_t N = geom.N;
  c.sp0 = p.spins + ((uint64_t)c.g * slots + (uint64_t)(c.tslot * R)) * N;
  const uint64_t* Jg = p.J + (uint64_t)c.g * D * N;
  const uint32_t w_begin = blockIdx.x * p.words_per_block;
  const uint32_t w_end = min(w_begin + p.words_per_block, geom.half);
  for (uint32_t base = w_begin; base < w_end; base += kBlock) {  // uniform across the block
    const uint32_t wi = base + threadIdx.x;
    const bool valid = wi < w_end;
    Nbr n;
    uint64_t jw[2 * D];
    if (valid) {
      n = split_neighbours_t<P2>(geom, p.colour, wi);
    }
    if (valid && !(kJReload && !kUFirst && !(kMode == 2 && R == 2))) {
      jw[0] = __ldg(Jg + n.self);
      jw[1] = __ldg(Jg + n.xm);
      jw[2] = __ldg(Jg + N + n.self);
      jw[3] = __ldg(Jg + N + n.ym);
      if (D == 3) {
        jw[4] = __ldg(Jg + 2u * N + n.self);
        jw[5] = __ldg(Jg + 2u * N + n.zm);
      }
    }
    if (kMode == 2 && R == 2) {
      if (!valid) continue;
      Word wa[2];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const uint64_t* sp = c.sp0 + (uint64_t)a * N;
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
        count_unsat<D>(e, wa[a].u0, wa[a].u1, wa[a].u2);
        wa[a].lt = kAlways ? lop3c<kAlways>(wa[a].u2, wa[a].u1, wa[a].u0) : 0ull;
        wa[a].und = lop3c<kNeed>(wa[a].u2, wa[a].u1, wa[a].u0);
      }
      const uint32_t c2a = sigma_c2(c, 0u), c2b = sigma_c2(c, 1u);
      pairs2<0>(wa[0], wa[1], p, c.tk, n.site, c2a, c2b);
      finish_tail(wa[0], p, c.tk, n.site, c2a, s_lut);
      finish_tail(wa[1], p, c.tk, n.site, c2b, s_lut);
      finish(c, n.self, 0u, wa[0]);
      finish(c, n.self, 1u, wa[1]);
      continue;
    }
    uint64_t uu[R][3];
    if (kUFirst && valid) {
#pragma unroll
      for (int a = 0; a < R; ++a) {
        const uint64_t* sp = c.sp0 + (uint64_t)a * N;
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
        count_unsat<D>(e, uu[a][0], uu[a][1], uu[a][2]);
      }
    }
#pragma unroll
    for (int a = 0; a < R; ++a) {
      Word w;
      w.und = 0;
      w.lt = 0;
      w.u0 = w.u1 = w.u2 = 0;
      uint32_t c2 = 0;
      if (valid && kUFirst) {
        w.u0 = uu[a][0];
        w.u1 = uu[a][1];
        w.u2 = uu[a][2];
      } else if (valid) {
        const uint64_t* sp = c.sp0 + (uint64_t)a * N;
        const uint64_t b = sp[n.self];
        uint64_t e[2 * D];
        if (kJReload) {  // coupling words from L1 again for each replica: none held across the plane loop
          e[0] = b ^ sp[n.xp] ^ __ldg(Jg + n.self);
          e[1] = b ^ sp[n.xm] ^ __ldg(Jg + n.xm);
          e[2] = b ^ sp[n.yp] ^ __ldg(Jg + N + n.self);
          e[3] = b ^ sp[n.ym] ^ __ldg(Jg + N + n.ym);
          if (D == 3) {
            e[4] = b ^ sp[n.zp] ^ __ldg(Jg + 2u * N + n.self);
            e[5] = b ^ sp[n.zm] ^ __ldg(Jg + 2u * N + n.zm);
          }
        } else {
          e[0] = b ^ sp[n.xp] ^ jw[0];
          e[1] = b ^ sp[n.xm] ^ jw[1];
          e[2] = b ^ sp[n.yp] ^ jw[2];
          e[3] = b ^ sp[n.ym] ^ jw[3];
          if (D == 3) {
            e[4] = b ^ sp[n.zp] ^ jw[4];
            e[5] = b ^ sp[n.zm] ^ jw[5];
          }
        }
        count_unsat<D>(e, w.u0, w.u1, w.u2);
      }
      if (valid) {
        w.lt = kAlways ? lop3c<kAlways>(w.u2, w.u1, w.u0) : 0ull;
        w.und = lop3c<kNeed>(w.u2, w.u1, w.u0);
        c2 = sigma_c2(c, (uint32_t)a);
        pairs<0>(w, p, c.tk, n.site, c2);
        if (kMode != 1) {
          finish_tail(w, p, c.tk, n.site, c2, s_lut);
          finish(c, n.self, (uint32_t)a, w);
        }
      }
      if (kMode != 1) continue;
      const bool pend = valid && w.und != 0ull;
      push(*q, nq, pend, w, valid ? n.self : 0u, valid ? n.site : 0u, (uint32_t)a);
      if (valid && !pend) finish(c, n.self, (uint32_t)a, w);
      if (nq >= 32u) round(*q, nq, 32u, c);
    }
  }
  if (kMode == 1 && nq > 0u) round(*q, nq, nq, c);
}
