// jit_sweep_lt.cuh -- bit-sliced sweep for lane-uniform thresholds (one
// temperature), specialised at run time (jit.cu) with the truth tables as
// lop3 immediates and the lattice geometry as constants.  Preamble macros as
// for jit_sweep.cuh: IANUS_JIT_D, _ALGO, _R (1 or 2), _P2, _LUTS, _ALWAYS,
// _NEED, _L, _LH, _LL, _BLOCK, _MINB.
//
// The update is the look-up-table compare of Sec. 3.2 in bit-sliced form:
// the 64 lanes of a word are 64 samples, the class u = (u2 u1 u0) of a lane
// is its number of unsatisfied bonds, and the random number of a lane is
// compared with its class threshold one bit-plane at a time, most
// significant first, two planes per Philox4x32-10 block.  Three things set
// this kernel apart:
//
// * Rounds 0 and 1 of the Philox block split into a part that depends on
//   the site only and a part that depends on (slot, plane pair, group,
//   sweep) only.  Counter word c0 is the site, c2 the tag / pair / slot /
//   group word, c1 and c3 the sweep.  After round 0, words 0 and 1 depend
//   on c2 alone and words 2 and 3 on the site alone; after round 1 each
//   word is a site part XOR a block-uniform part.  The block computes the
//   uniform parts of its 16 x R blocks once; a thread computes the site
//   part once per site; each block then costs two XORs and rounds 2..9.
// * The plane compare keeps two words per 64 lanes: und (not yet decided)
//   and res (the decision r < T where decided).  At a plane with threshold
//   bits t and random bits r, res takes t on the undecided lanes (at the
//   deciding plane r != t and r < T iff t = 1; on lanes that stay undecided
//   the value is overwritten later) and und drops the lanes with r != t:
//   three lop3 per 32 lanes with the threshold lop3 included.
// * Plane pairs 0..3 run for every word (a word needs pair m with
//   probability 1 - (1 - 4^-m)^64: 1, 1, 0.98, 0.64).  The decided lanes of
//   a word are then written by the thread that owns it.  A word with lanes
//   still undecided (a fifth of them) goes to a per-warp queue in shared
//   memory; a round takes 32 queued words, so all lanes of the warp work,
//   and runs pair 4 for them with its tables as immediates.  The lanes still
//   undecided after that (about 0.07 per word) go one by one, as 8-byte
//   items (site, lane, class, next pair, slot), to a second queue, whose
//   rounds compare an item's two random bits of one pair with the two
//   threshold bits of its class and either finish it or put it back with
//   the next pair.  Lanes finished from a queue are flipped by an atomic XOR
//   of their bits, since the word's owner has already written it and
//   several of its lanes may finish in one round.
#include "common.cuh"

namespace ianus {
namespace jlt {

constexpr int D = IANUS_JIT_D;
constexpr int ALGO = IANUS_JIT_ALGO;
constexpr int R = IANUS_JIT_R;
constexpr bool P2 = IANUS_JIT_P2 != 0;
constexpr uint32_t kLut[32] = {IANUS_JIT_LUTS};
constexpr uint32_t kAlways = IANUS_JIT_ALWAYS;
constexpr uint32_t kNeed = IANUS_JIT_NEED;
constexpr uint32_t kReach = (1u << (2 * D + 1)) - 1u;  // classes u = 0..2D occur
#ifndef IANUS_JIT_BLOCK
#define IANUS_JIT_BLOCK 128
#endif
constexpr int kBlock = IANUS_JIT_BLOCK;
constexpr int kWarps = kBlock / 32;
constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
constexpr uint32_t kFull = 0xffffffffu;
constexpr int kHeadPairs = 4;  // plane pairs every word runs
constexpr uint32_t kQ = 64;            // lane queue: < 32 left + <= 32 pushed
constexpr uint32_t kQW = 32 * (R + 1);  // word queue: < 32 left + <= 32 per slot pushed

// Class threshold as a 32-bit number: bit (31 - p) of T_u is bit u of the
// truth table of plane p.  Evaluated at compile time; used by the queued
// lanes.
__host__ __device__ constexpr uint32_t thr_of(int u) {
  uint32_t t = 0;
  for (int p = 0; p < 32; ++p) t |= ((kLut[p] >> u) & 1u) << (31 - p);
  return t;
}

__device__ __forceinline__ uint32_t class_threshold(uint32_t u) {
  constexpr uint32_t t0 = thr_of(0), t1 = thr_of(1), t2 = thr_of(2), t3 = thr_of(3), t4 = thr_of(4),
                     t5 = thr_of(5), t6 = thr_of(6), t7 = thr_of(7);
  const uint32_t v[8] = {t0, t1, t2, t3, t4, t5, t6, t7};
  uint32_t r = t0;
#pragma unroll
  for (int k = 1; k < 8; ++k) r = u == (uint32_t)k ? v[k] : r;
  return r;
}

template <uint32_t LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT & 0xFFu));
  return d;
}

// 32 lanes of a word: class planes, undecided lanes, decisions.
struct Half {
  uint32_t u0, u1, u2, und, res;
};

// Plane p of one half: threshold bits t = table p of (u2, u1, u0); res takes
// t where undecided (0xCA: a ? b : c); und keeps the lanes with r == t (0x90:
// a & ~(b ^ c)).
template <int P>
__device__ __forceinline__ void plane(Half& h, uint32_t r) {
  const uint32_t t = lop3<kLut[P]>(h.u2, h.u1, h.u0);
  h.res = lop3<0xCA>(h.und, t, h.res);
  h.und = lop3<0x90>(h.und, r, t);
}

// Site part of Philox rounds 0 and 1: with P0 = M0 * site, round 0 gives
// c3' = lo(P0) and c2' = hi(P0) ^ t_hi ^ k1[0]; round 1 multiplies c2' by M1.
struct SiteKey {
  uint32_t a;   // hi(M1 * c2'): c0'' = a ^ U.x
  uint32_t c1;  // lo(M1 * c2') = c1''
  uint32_t c3;  // c3' : c2'' = c3 ^ U.y
};

__device__ __forceinline__ SiteKey site_key(uint32_t site, uint32_t thi_k) {
  const uint64_t p0 = (uint64_t)kM0 * site;
  const uint32_t c2 = (uint32_t)(p0 >> 32) ^ thi_k;
  const uint64_t p1 = (uint64_t)kM1 * c2;
  return SiteKey{(uint32_t)(p1 >> 32), (uint32_t)p1, (uint32_t)p0};
}

// Rounds 2..9 from the state after round 1.
__device__ __forceinline__ uint4 rounds_rest(const SiteKey& s, const uint4& U, const PhiloxKeys& K) {
  uint32_t c0 = s.a ^ U.x, c1 = s.c1, c2 = s.c3 ^ U.y, c3 = U.z;
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)kM0 * c0;
    const uint64_t p1 = (uint64_t)kM1 * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ K.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ K.k1[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Planes 2M and 2M+1 of a 64-lane word from its block x: W_2M = x.x | x.y << 32,
// W_2M+1 = x.z | x.w << 32.
template <int M>
__device__ __forceinline__ void pair_planes(Half& lo, Half& hi, const uint4& x) {
  plane<2 * M>(lo, x.x);
  plane<2 * M>(hi, x.y);
  plane<2 * M + 1>(lo, x.z);
  plane<2 * M + 1>(hi, x.w);
}

// A queued lane: site, lane, class, next plane pair, slot.
struct Item {
  uint32_t site, meta;  // meta: lane | class << 6 | pair << 9 | slot << 13
};

// A queued word (undecided after pairs 0..3): site and slot, the undecided
// lanes and the class planes, in three parts so that each store and load is
// one 16- or 8-byte access.
struct WordQ {
  uint4 a[kQW];  // site, slot, und lo, und hi
  uint4 b[kQW];  // u0 lo, u0 hi, u1 lo, u1 hi
  uint2 c[kQW];  // u2 lo, u2 hi
};

struct Shared {
  uint4 u[R * 16];         // uniform parts of rounds 0..1 per (slot, pair)
  uint32_t thr[8];         // class thresholds
  WordQ wq[kWarps];        // per-warp queues of words that need pair kHeadPairs
  Item lq[kWarps][kQ];     // per-warp queues of single lanes (pairs kHeadPairs + 1 ..)
};

struct Ctx {
  const PhiloxKeys* keys;
  uint32_t thi_k;          // t_hi ^ k1[0]
  uint64_t* sp0;           // spins of the group's slot 0; slot a is a * N further
  int colour;
};

__device__ __forceinline__ uint32_t self_of(uint32_t site, int colour) {
  constexpr uint32_t L = (uint32_t)IANUS_JIT_L;
  const uint32_t row = site / L, x = site - row * L;
  return (2u * row + (uint32_t)colour) * (L / 2u) + (x >> 1);
}

__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << (threadIdx.x & 31u)) - 1u; }

// One round over the top `take` (<= 32) queued lanes: one plane pair each.
// A lane whose random bits equal its threshold bits goes back with the next
// pair; after pair 15 (all 32 bits equal) r == T, which is not below.
__device__ __forceinline__ void lane_round(const Shared& sh, Item* q, uint32_t& nq, uint32_t take, const Ctx& c) {
  const uint32_t lane = threadIdx.x & 31u;
  const bool has = lane < take;
  Item it{0u, 0u};
  if (has) it = q[nq - take + lane];
  __syncwarp();
  nq -= take;
  bool again = false;
  if (has) {
    const uint32_t l = it.meta & 63u, cls = (it.meta >> 6) & 7u, m = (it.meta >> 9) & 15u, a = it.meta >> 13;
    const uint4 x = rounds_rest(site_key(it.site, c.thi_k), sh.u[a * 16u + m], *c.keys);
    const uint32_t w0 = l < 32u ? x.x : x.y, w1 = l < 32u ? x.z : x.w;
    const uint32_t rb = (((w0 >> (l & 31u)) & 1u) << 1) | ((w1 >> (l & 31u)) & 1u);
    const uint32_t tb = (sh.thr[cls] >> (30u - 2u * m)) & 3u;
    if (rb == tb && m < 15u) {
      again = true;
      it.meta += 1u << 9;
    } else {
      const bool lt = rb < tb;
      const bool flip = ALGO == 0 ? lt : !lt;
      if (flip) {
        uint64_t* w = c.sp0 + (uint64_t)a * kJitSites + self_of(it.site, c.colour);
        atomicXor((unsigned long long*)w, 1ull << l);
      }
    }
  }
  const uint32_t bal = __ballot_sync(kFull, again);
  if (again) q[nq + __popc(bal & lanemask_lt())] = it;
  nq += __popc(bal);
  __syncwarp();
}

// One round over the top `take` (<= 32) queued words: plane pair kHeadPairs
// with its tables as immediates; lanes decided there are flipped in place,
// lanes still undecided go to the lane queue one at a time.
__device__ __forceinline__ void word_round(Shared& sh, uint32_t& nw, uint32_t take, uint32_t& nl, const Ctx& c) {
  const uint32_t wp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  WordQ& wq = sh.wq[wp];
  Item* lq = sh.lq[wp];
  const bool has = lane < take;
  uint4 qa = make_uint4(0u, 0u, 0u, 0u), qb = qa;
  uint2 qc = make_uint2(0u, 0u);
  if (has) {
    const uint32_t i = nw - take + lane;
    qa = wq.a[i];
    qb = wq.b[i];
    qc = wq.c[i];
  }
  __syncwarp();
  nw -= take;
  Half lo{qb.x, qb.z, qc.x, qa.z, 0u}, hi{qb.y, qb.w, qc.y, qa.w, 0u};
  if (has) {
    const uint4 x = rounds_rest(site_key(qa.x, c.thi_k), sh.u[qa.y * 16u + kHeadPairs], *c.keys);
    pair_planes<kHeadPairs>(lo, hi, x);
    const uint32_t dlo = qa.z & ~lo.und, dhi = qa.w & ~hi.und;  // decided at this pair
    const uint64_t flip = ((uint64_t)((ALGO == 0 ? lo.res : ~lo.res) & dlo)) |
                          ((uint64_t)((ALGO == 0 ? hi.res : ~hi.res) & dhi) << 32);
    if (flip) {
      uint64_t* w = c.sp0 + (uint64_t)qa.y * kJitSites + self_of(qa.x, c.colour);
      atomicXor((unsigned long long*)w, flip);
    }
  }
  uint32_t plo = has ? lo.und : 0u, phi = has ? hi.und : 0u;
  for (;;) {
    const bool more = (plo | phi) != 0u;
    const uint32_t bal = __ballot_sync(kFull, more);
    if (bal == 0u) break;
    if (more) {
      const bool up = plo == 0u;
      const uint32_t w = up ? phi : plo;
      const uint32_t bit = w & (0u - w);
      const uint32_t s = 31u - __clz(bit);
      if (up) phi ^= bit;
      else plo ^= bit;
      const uint32_t v0 = up ? hi.u0 : lo.u0, v1 = up ? hi.u1 : lo.u1, v2 = up ? hi.u2 : lo.u2;
      const uint32_t cls = (((v2 >> s) & 1u) << 2) | (((v1 >> s) & 1u) << 1) | ((v0 >> s) & 1u);
      const uint32_t l = s + (up ? 32u : 0u);
      lq[nl + __popc(bal & lanemask_lt())] =
          Item{qa.x, l | (cls << 6) | ((uint32_t)(kHeadPairs + 1) << 9) | (qa.y << 13)};
    }
    nl += __popc(bal);
    __syncwarp();
    if (nl >= 32u) lane_round(sh, lq, nl, 32u, c);
  }
}

// Pairs 0..kHeadPairs-1 for the words of one site (R words, two Philox
// chains in flight: the slots for R = 2, consecutive pairs for R = 1).
template <int M>
__device__ __forceinline__ void head_pairs(Half (&lo)[R], Half (&hi)[R], const SiteKey& sk, const Shared& sh,
                                           const PhiloxKeys& K) {
  if constexpr (M < kHeadPairs) {
    if constexpr (R == 2) {
      const uint4 xa = rounds_rest(sk, sh.u[M], K);
      const uint4 xb = rounds_rest(sk, sh.u[16 + M], K);
      pair_planes<M>(lo[0], hi[0], xa);
      pair_planes<M>(lo[1], hi[1], xb);
      head_pairs<M + 1>(lo, hi, sk, sh, K);
    } else {
      const uint4 xa = rounds_rest(sk, sh.u[M], K);
      const uint4 xb = rounds_rest(sk, sh.u[M + 1], K);
      pair_planes<M>(lo[0], hi[0], xa);
      pair_planes<M + 1>(lo[0], hi[0], xb);
      head_pairs<M + 2>(lo, hi, sk, sh, K);
    }
  }
}

}  // namespace jlt
}  // namespace ianus

extern "C" __global__ void __launch_bounds__(ianus::jlt::kBlock, IANUS_JIT_MINB)
    ianus_jit_sweep_lt(const ianus::BitsParams p) {
  using namespace ianus;
  using namespace ianus::jlt;
  __shared__ Shared sh;
  dependent_launch_entry();
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  const int g = blockIdx.y;  // one temperature: blockIdx.y = group
  // uniform parts of Philox rounds 0 and 1 for every (slot, pair)
  if (threadIdx.x < (unsigned)(R * 16)) {
    const uint32_t a = threadIdx.x >> 4, m = threadIdx.x & 15u;
    const uint32_t c2 = (TAG_SPIN << 28) | (m << 24) | (a << 12) | (uint32_t)g;
    const uint64_t p1 = (uint64_t)kM1 * c2;
    const uint32_t c0r = (uint32_t)(p1 >> 32) ^ tk.lo ^ p.keys.k0[0];
    const uint64_t p0 = (uint64_t)kM0 * c0r;
    sh.u[threadIdx.x] = make_uint4((uint32_t)p1 ^ p.keys.k0[1], (uint32_t)(p0 >> 32) ^ p.keys.k1[1], (uint32_t)p0, 0u);
  }
  if (threadIdx.x < 8) sh.thr[threadIdx.x] = class_threshold(threadIdx.x);
  __syncthreads();
  constexpr Geom geom = kJitGeom;
  constexpr uint32_t N = kJitSites;
  Ctx c;
  c.keys = &p.keys;
  c.thi_k = tk.hi ^ p.keys.k1[0];
  c.sp0 = p.spins + (uint64_t)g * R * N;
  c.colour = p.colour;
  const uint64_t* Jg = p.J + (uint64_t)g * D * N;
  WordQ& wq = sh.wq[threadIdx.x >> 5];
  uint32_t nw = 0, nl = 0;
  const uint32_t w_begin = blockIdx.x * p.words_per_block;
  const uint32_t w_end = min(w_begin + p.words_per_block, geom.half);
  for (uint32_t base = w_begin; base < w_end; base += kBlock) {
    const uint32_t wi = base + threadIdx.x;
    if (__ballot_sync(kFull, wi < w_end) == 0u) break;  // warp past the end of the block's words
    const bool valid = wi < w_end;
    Half lo[R], hi[R];
    uint32_t site = 0;
    uint64_t b[R];
    Nbr n{};
    if (valid) {
      n = split_neighbours_t<P2>(geom, p.colour, wi);
      site = n.site;
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
        const uint64_t* sp = c.sp0 + (uint64_t)a * N;
        b[a] = sp[n.self];
        uint64_t e[2 * D];
        e[0] = b[a] ^ sp[n.xp] ^ jw[0];
        e[1] = b[a] ^ sp[n.xm] ^ jw[1];
        e[2] = b[a] ^ sp[n.yp] ^ jw[2];
        e[3] = b[a] ^ sp[n.ym] ^ jw[3];
        if (D == 3) {
          e[4] = b[a] ^ sp[n.zp] ^ jw[4];
          e[5] = b[a] ^ sp[n.zm] ^ jw[5];
        }
        uint64_t u0, u1, u2;
        count_unsat<D>(e, u0, u1, u2);
        lo[a] = Half{(uint32_t)u0, (uint32_t)u1, (uint32_t)u2, 0u, 0u};
        hi[a] = Half{(uint32_t)(u0 >> 32), (uint32_t)(u1 >> 32), (uint32_t)(u2 >> 32), 0u, 0u};
      }
    } else {
#pragma unroll
      for (int a = 0; a < R; ++a) {
        lo[a] = Half{0u, 0u, 0u, 0u, 0u};
        hi[a] = lo[a];
        b[a] = 0;
      }
    }
#pragma unroll
    for (int a = 0; a < R; ++a) {
      if (valid) {
        if constexpr ((kNeed & kReach) == kReach) {
          lo[a].und = hi[a].und = kFull;
        } else {
          lo[a].und = lop3<kNeed>(lo[a].u2, lo[a].u1, lo[a].u0);
          hi[a].und = lop3<kNeed>(hi[a].u2, hi[a].u1, hi[a].u0);
        }
        if constexpr ((kAlways & kReach) != 0u) {
          lo[a].res = lop3<kAlways>(lo[a].u2, lo[a].u1, lo[a].u0);
          hi[a].res = lop3<kAlways>(hi[a].u2, hi[a].u1, hi[a].u0);
        }
      }
    }
    const SiteKey sk = site_key(site, c.thi_k);
    head_pairs<0>(lo, hi, sk, sh, p.keys);
    // decided lanes: flip where (r < T) != heat bath
#pragma unroll
    for (int a = 0; a < R; ++a) {
      const uint64_t und = (uint64_t)lo[a].und | ((uint64_t)hi[a].und << 32);
      const uint64_t res = (uint64_t)lo[a].res | ((uint64_t)hi[a].res << 32);
      const uint64_t flip = (ALGO == 0 ? res : ~res) & ~und;
      if (valid && flip) c.sp0[(uint64_t)a * N + n.self] = b[a] ^ flip;
    }
    // queue the words with undecided lanes (slot 0's, then slot 1's)
#pragma unroll
    for (int a = 0; a < R; ++a) {
      const bool has = valid && (lo[a].und | hi[a].und) != 0u;
      const uint32_t bal = __ballot_sync(kFull, has);
      if (has) {
        const uint32_t i = nw + __popc(bal & lanemask_lt());
        wq.a[i] = make_uint4(site, (uint32_t)a, lo[a].und, hi[a].und);
        wq.b[i] = make_uint4(lo[a].u0, hi[a].u0, lo[a].u1, hi[a].u1);
        wq.c[i] = make_uint2(lo[a].u2, hi[a].u2);
      }
      nw += __popc(bal);
    }
    __syncwarp();
    while (nw >= 32u) word_round(sh, nw, 32u, nl, c);
  }
  while (nw > 0u) word_round(sh, nw, nw < 32u ? nw : 32u, nl, c);
  while (nl > 0u) lane_round(sh, sh.lq[threadIdx.x >> 5], nl, nl < 32u ? nl : 32u, c);
}
