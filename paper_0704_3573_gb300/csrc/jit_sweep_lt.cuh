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
//   memory; a round takes 32 queued words, so every lane of the warp has
//   one, and runs pairs 4, 5, ... in lockstep while any of them is
//   undecided (tables as immediates up to pair 7, read at run time after
//   that).  Its lanes are then flipped by an atomic XOR of their bits, since
//   the word's owner has already written the word.
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
#ifndef IANUS_JIT_PERSIST
#define IANUS_JIT_PERSIST 0
#endif
constexpr uint32_t kQW = 32 * (R + 1);  // word queue: < 32 left + <= 32 per slot pushed

// Truth table of plane p (0..31) at run time.
__device__ __forceinline__ uint32_t lut_of(uint32_t p) {
  constexpr uint32_t v[32] = {IANUS_JIT_LUTS};
  uint32_t r = v[0];
#pragma unroll
  for (int k = 1; k < 32; ++k) r = p == (uint32_t)k ? v[k] : r;
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
// With every lane undecided at plane 0 (every class compares, none always
// flips: the heat bath), plane 0 reduces to res = t, und = ~(r ^ t) (0xC3).
constexpr bool kAllUndecided = (kNeed & kReach) == kReach && (kAlways & kReach) == 0u;

template <int P>
__device__ __forceinline__ void plane(Half& h, uint32_t r) {
  const uint32_t t = lop3<kLut[P]>(h.u2, h.u1, h.u0);
  if constexpr (P == 0 && kAllUndecided) {
    h.res = t;
    h.und = lop3<0xC3>(r, t, r);
  } else {
    h.res = lop3<0xCA>(h.und, t, h.res);
    h.und = lop3<0x90>(h.und, r, t);
  }
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

// A queued word (undecided after pairs 0..3): site and slot, the undecided
// lanes and the class planes, in three parts so that each store and load is
// one 16- or 8-byte access.
struct WordQ {
  uint4 a[kQW];  // site, slot, und lo, und hi
  uint4 b[kQW];  // u0 lo, u0 hi, u1 lo, u1 hi
  uint2 c[kQW];  // u2 lo, u2 hi
};

// A warp's shared memory: its word queue, which before the first push holds
// the Philox blocks of pairs 0..kHeadPairs-1 of the warp's first sites,
// drawn before the kernel waits for the previous colour pass.
union WarpArea {
  WordQ wq;
  uint4 pre[kHeadPairs][R][32];
};

struct Shared {
  uint4 u[R * 16];         // uniform parts of rounds 0..1 per (slot, pair)
  uint8_t lut[32];         // truth tables of the planes (pairs 8..15 read them at run time)
  WarpArea wa[kWarps];     // per-warp queues of words that need pair kHeadPairs
  uint32_t left[kWarps];   // words each warp leaves queued at the end of its words
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

// Spin words.  In the persistent form other blocks write them during the
// launch, so they are read from L2 (ld.global.cg), never from a stale L1 line.
__device__ __forceinline__ uint64_t ld_spin(const uint64_t* p) {
#if IANUS_JIT_PERSIST
  return __ldcg((const unsigned long long*)p);
#else
  return *p;
#endif
}

// Plane p with its truth table given at run time (pairs 8..15, rarely
// reached): bit u of tab for a lane of class u, by a multiplexer tree.
__device__ __forceinline__ void plane_rt(Half& h, uint32_t r, uint32_t tab) {
  uint32_t m[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) m[k] = 0u - ((tab >> k) & 1u);
  const uint32_t a0 = lop3<0xCA>(h.u0, m[1], m[0]), a1 = lop3<0xCA>(h.u0, m[3], m[2]);
  const uint32_t a2 = lop3<0xCA>(h.u0, m[5], m[4]), a3 = lop3<0xCA>(h.u0, m[7], m[6]);
  const uint32_t b0 = lop3<0xCA>(h.u1, a1, a0), b1 = lop3<0xCA>(h.u1, a3, a2);
  const uint32_t t = lop3<0xCA>(h.u2, b1, b0);
  h.res = lop3<0xCA>(h.und, t, h.res);
  h.und = lop3<0x90>(h.und, r, t);
}

// Pairs M..7 of a queued word in lockstep across the warp, while any word
// of the warp is undecided, with the tables as immediates.
template <int M>
__device__ __forceinline__ void tail_pairs(Half& lo, Half& hi, const SiteKey& sk, const uint4* U,
                                           const PhiloxKeys& K) {
  if constexpr (M < 8) {
    if (!__any_sync(kFull, (lo.und | hi.und) != 0u)) return;
    pair_planes<M>(lo, hi, rounds_rest(sk, U[M], K));
    tail_pairs<M + 1>(lo, hi, sk, U, K);
  }
}

// One round over queued words, one per lane: item `idx` of warp `src`'s
// queue where `has`.  Pair kHeadPairs and the following ones run until every
// word of the warp is decided; the queued lanes are then flipped in place.
__device__ __forceinline__ void word_round_at(const Shared& sh, uint32_t src, uint32_t idx, bool has,
                                              const Ctx& c) {
  uint4 qa = make_uint4(0u, 0u, 0u, 0u), qb = qa;
  uint2 qc = make_uint2(0u, 0u);
  if (has) {
    const WordQ& wq = sh.wa[src].wq;
    qa = wq.a[idx];
    qb = wq.b[idx];
    qc = wq.c[idx];
  }
  Half lo{qb.x, qb.z, qc.x, qa.z, 0u}, hi{qb.y, qb.w, qc.y, qa.w, 0u};
  const SiteKey sk = site_key(qa.x, c.thi_k);
  const uint4* U = sh.u + qa.y * 16u;
  tail_pairs<kHeadPairs>(lo, hi, sk, U, *c.keys);
  for (uint32_t m = 8; m < 16u && __any_sync(kFull, (lo.und | hi.und) != 0u); ++m) {
    const uint4 x = rounds_rest(sk, U[m], *c.keys);
    const uint32_t t0 = sh.lut[2u * m], t1 = sh.lut[2u * m + 1u];
    plane_rt(lo, x.x, t0);
    plane_rt(hi, x.y, t0);
    plane_rt(lo, x.z, t1);
    plane_rt(hi, x.w, t1);
  }
  if (has) {
    // lanes still undecided after 32 planes have r == T: not below
    const uint32_t rlo = lo.res & ~lo.und, rhi = hi.res & ~hi.und;
    const uint64_t flip = ((uint64_t)((ALGO == 0 ? rlo : ~rlo) & qa.z)) | ((uint64_t)((ALGO == 0 ? rhi : ~rhi) & qa.w) << 32);
    if (flip) {
      uint64_t* w = c.sp0 + (uint64_t)qa.y * kJitSites + self_of(qa.x, c.colour);
      atomicXor((unsigned long long*)w, flip);
    }
  }
}

// The top `take` (<= 32) words of this warp's queue.
__device__ __forceinline__ void word_round(const Shared& sh, uint32_t& nw, uint32_t take, const Ctx& c) {
  const uint32_t wp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  word_round_at(sh, wp, nw - take + lane, lane < take, c);
  __syncwarp();  // every lane has read its item before the queue is pushed to again
  nw -= take;
}

// The words the warps left queued (fewer than 32 each), as full rounds
// spread over the warps: warp w takes rounds w, w + kWarps, ... of the
// concatenated queues.  Called by every thread of the block.
__device__ __forceinline__ void drain_block(Shared& sh, uint32_t nw, const Ctx& c) {
  const uint32_t wp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  if (lane == 0) sh.left[wp] = nw;
  __syncthreads();
  uint32_t off[kWarps], total = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    off[w] = total;
    total += sh.left[w];
  }
  for (uint32_t r = wp; 32u * r < total; r += kWarps) {
    const uint32_t k = 32u * r + lane;
    uint32_t src = 0, base = 0;
#pragma unroll
    for (int w = 1; w < kWarps; ++w)
      if (off[w] <= k) {
        src = (uint32_t)w;
        base = off[w];
      }
    word_round_at(sh, src, k - base, k < total, c);
  }
  __syncthreads();  // the queues are free again
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

// Pairs 0..kHeadPairs-1 from Philox blocks drawn earlier (WarpArea::pre).
template <int M>
__device__ __forceinline__ void head_pairs_pre(Half (&lo)[R], Half (&hi)[R], const WarpArea& wa, uint32_t lane) {
  if constexpr (M < kHeadPairs) {
#pragma unroll
    for (int a = 0; a < R; ++a) pair_planes<M>(lo[a], hi[a], wa.pre[M][a][lane]);
    head_pairs_pre<M + 1>(lo, hi, wa, lane);
  }
}

// Colour-c word w = row * L/2 + k of the split layout: the site x + L row
// with x = 2k + xpar, xpar the parity that gives the site colour c.  Since
// L = 2h the natural index is 2w + xpar, the word is w + (row + c) h, and
// the other colour's word of the same row and k is 2(w - k) + (1 - c) h + k;
// the y and z neighbours are that word plus or minus 2h and 2hL rows' worth
// of words, wrapped at the faces.
__device__ __forceinline__ Nbr neighbours_lt(uint32_t w, int colour) {
  constexpr uint32_t L = (uint32_t)IANUS_JIT_L, h = L / 2u;
  const uint32_t c = (uint32_t)colour;
  const uint32_t row = w / h, k = w - row * h;
  const uint32_t y = row % L, z = D == 3 ? row / L : 0u;
  const uint32_t xpar = (c ^ y ^ z) & 1u;
  Nbr n;
  n.self = w + (row + c) * h;
  n.site = 2u * w + xpar;
  const uint32_t base_o = 2u * (w - k) + (1u - c) * h;
  uint32_t kp = k + xpar, km = k + xpar - 1u;  // (x + 1) / 2 and (x - 1) / 2, mod h
  if (kp == h) kp = 0u;
  if (km == 0xffffffffu) km = h - 1u;
  n.xp = base_o + kp;
  n.xm = base_o + km;
  const uint32_t ko = base_o + k;
  n.yp = ko + (y == L - 1u ? 0u - 2u * h * (L - 1u) : 2u * h);
  n.ym = ko + (y == 0u ? 2u * h * (L - 1u) : 0u - 2u * h);
  if (D == 3) {
    n.zp = ko + (z == L - 1u ? 0u - 2u * h * L * (L - 1u) : 2u * h * L);
    n.zm = ko + (z == 0u ? 2u * h * L * (L - 1u) : 0u - 2u * h * L);
  } else {
    n.zp = n.zm = 0u;
  }
  return n;
}

// Natural site index of colour word w.
__device__ __forceinline__ uint32_t site_of_word(uint32_t w, int colour) {
  constexpr uint32_t L = (uint32_t)IANUS_JIT_L, h = L / 2u;
  const uint32_t row = w / h;
  const uint32_t y = row % L, z = D == 3 ? row / L : 0u;
  return 2u * w + (((uint32_t)colour ^ y ^ z) & 1u);
}

// Draws the Philox blocks of pairs 0..kHeadPairs-1 of every slot for the
// thread's first site (colour word w) into its warp's area.
__device__ __forceinline__ void draw_first(Shared& sh, uint32_t w, const Ctx& c) {
  const uint32_t lane = threadIdx.x & 31u;
  WarpArea& wa = sh.wa[threadIdx.x >> 5];
  const SiteKey sk = site_key(site_of_word(w, c.colour), c.thi_k);
#pragma unroll
  for (int m = 0; m < kHeadPairs; ++m)
#pragma unroll
    for (int a = 0; a < R; ++a) wa.pre[m][a][lane] = rounds_rest(sk, sh.u[a * 16 + m], *c.keys);
}

// The colour-c words [w_begin, w_end) of one group (word w = row * L/2 + k
// of the colour's half rows): pairs 0..3 for every word, then the queues,
// drained before returning.
__device__ __forceinline__ void sweep_words(Shared& sh, const Ctx& c, const uint64_t* __restrict__ Jg,
                                            uint32_t w_begin, uint32_t w_end, bool first_drawn) {
  constexpr uint32_t N = kJitSites;
  WordQ& wq = sh.wa[threadIdx.x >> 5].wq;
  uint32_t nw = 0;
  for (uint32_t base = w_begin; base < w_end; base += kBlock) {
    const uint32_t wi = base + threadIdx.x;
    if (__ballot_sync(kFull, wi < w_end) == 0u) break;  // warp past the end of the block's words
    const bool valid = wi < w_end;
    Half lo[R], hi[R];
    uint32_t site = 0;
    uint64_t b[R];
    Nbr n{};
    if (valid) {
      n = neighbours_lt(wi, c.colour);
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
        b[a] = ld_spin(sp + n.self);
        uint64_t e[2 * D];
        e[0] = b[a] ^ ld_spin(sp + n.xp) ^ jw[0];
        e[1] = b[a] ^ ld_spin(sp + n.xm) ^ jw[1];
        e[2] = b[a] ^ ld_spin(sp + n.yp) ^ jw[2];
        e[3] = b[a] ^ ld_spin(sp + n.ym) ^ jw[3];
        if (D == 3) {
          e[4] = b[a] ^ ld_spin(sp + n.zp) ^ jw[4];
          e[5] = b[a] ^ ld_spin(sp + n.zm) ^ jw[5];
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
    if (first_drawn && base == w_begin) {  // the blocks of the first sites were drawn before the wait
      head_pairs_pre<0>(lo, hi, sh.wa[threadIdx.x >> 5], threadIdx.x & 31u);
      __syncwarp();  // every lane has read them before the warp's queue reuses the area
    } else {
      const SiteKey sk = site_key(site, c.thi_k);
      head_pairs<0>(lo, hi, sk, sh, *c.keys);
    }
    // decided lanes: flip where (r < T) != heat bath, one lop3 per half:
    // b ^ (res & ~und) (0xB4, Metropolis) or b ^ (~res & ~und) (0xE1)
#pragma unroll
    for (int a = 0; a < R; ++a) {
      constexpr uint32_t kFlip = ALGO == 0 ? 0xB4u : 0xE1u;
      const uint32_t nlo = lop3<kFlip>((uint32_t)b[a], lo[a].res, lo[a].und);
      const uint32_t nhi = lop3<kFlip>((uint32_t)(b[a] >> 32), hi[a].res, hi[a].und);
      if (valid) c.sp0[(uint64_t)a * N + n.self] = (uint64_t)nlo | ((uint64_t)nhi << 32);
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
    while (nw >= 32u) word_round(sh, nw, 32u, c);
  }
  drain_block(sh, nw, c);
}

// Uniform parts of Philox rounds 0 and 1 for every (slot, pair) of group g
// at sweep tk (threads 0 .. 16R - 1).
__device__ __forceinline__ void fill_uniform(Shared& sh, uint32_t g, const Tick& tk, const PhiloxKeys& K) {
  if (threadIdx.x < (unsigned)(R * 16)) {
    const uint32_t a = threadIdx.x >> 4, m = threadIdx.x & 15u;
    const uint32_t c2 = (TAG_SPIN << 28) | (m << 24) | (a << 12) | g;
    const uint64_t p1 = (uint64_t)kM1 * c2;
    const uint32_t c0r = (uint32_t)(p1 >> 32) ^ tk.lo ^ K.k0[0];
    const uint64_t p0 = (uint64_t)kM0 * c0r;
    sh.u[threadIdx.x] = make_uint4((uint32_t)p1 ^ K.k0[1], (uint32_t)(p0 >> 32) ^ K.k1[1], (uint32_t)p0, 0u);
  }
}

}  // namespace jlt
}  // namespace ianus

#if !IANUS_JIT_PERSIST

// One colour pass: block (x, g) updates colour words [x wpb, (x + 1) wpb) of
// group g.
extern "C" __global__ void __launch_bounds__(ianus::jlt::kBlock, IANUS_JIT_MINB)
    ianus_jit_sweep_lt(const ianus::BitsParams p) {
  using namespace ianus;
  using namespace ianus::jlt;
  __shared__ Shared sh;
  // Before the wait for the previous colour pass nothing it writes is read:
  // the sweep index (a launch parameter, or the captured graph's counter,
  // written before the graph starts) and the Philox blocks of this thread's
  // first site, which depend on the site and the sweep only.  Drawing them
  // here uses the SMs the previous launch's last blocks leave idle.
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  const uint32_t g = blockIdx.y;  // one temperature: blockIdx.y = group
  fill_uniform(sh, g, tk, p.keys);
  if (threadIdx.x < 32) sh.lut[threadIdx.x] = (uint8_t)lut_of(threadIdx.x);
  __syncthreads();
  Ctx c;
  c.keys = &p.keys;
  c.thi_k = tk.hi ^ p.keys.k1[0];
  c.sp0 = p.spins + (uint64_t)g * R * kJitSites;
  c.colour = p.colour;
  const uint32_t w_begin = blockIdx.x * p.words_per_block;
  const uint32_t w_end = min(w_begin + p.words_per_block, kJitGeom.half);
  draw_first(sh, min(w_begin + threadIdx.x, kJitGeom.half - 1u), c);
  dependent_launch_entry();
  sweep_words(sh, c, p.J + (uint64_t)g * D * kJitSites, w_begin, w_end, true);
}

#else

namespace ianus {
namespace jlt {

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits until *f >= target (acquire at GPU scope), at most timeout_ns.
__device__ __forceinline__ bool wait_flag(const uint32_t* f, uint32_t target, uint64_t timeout_ns) {
  const uint64_t t0 = global_ns();
  uint32_t nap = 32;
  for (;;) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    if (v >= target) return true;
    if (global_ns() - t0 > timeout_ns) return false;
    __nanosleep(nap);
    if (nap < 256u) nap <<= 1;
  }
}

// Block of group-row r when rows [j Rg / cpg, (j + 1) Rg / cpg) belong to block j.
__device__ __forceinline__ uint32_t owner(uint32_t r, uint32_t cpg, uint32_t Rg) {
  return (uint32_t)((((uint64_t)r + 1u) * cpg - 1u) / Rg);
}

}  // namespace jlt
}  // namespace ianus

// npass colour passes in one launch, the blocks of a pass separated by
// bounded waits on their neighbours' progress flags (see PersistParams).
// Launched cooperatively, so that every block is resident.
extern "C" __global__ void __launch_bounds__(ianus::jlt::kBlock, IANUS_JIT_MINB)
    ianus_jit_sweep_ltp(const ianus::BitsParams p, const ianus::PersistParams pp) {
  using namespace ianus;
  using namespace ianus::jlt;
  __shared__ Shared sh;
  __shared__ int s_abort;
  const uint32_t b = blockIdx.x;
  if ((int32_t)b == pp.skip_block) return;
  constexpr uint32_t L = (uint32_t)IANUS_JIT_L, h = L / 2u, Rg = kJitSites / L;
  constexpr uint32_t W = D == 3 ? L : 1u;  // rows between a site and its farthest neighbour
  const uint32_t cpg = pp.cpg, g = b / cpg, j = b - g * cpg;
  const uint32_t ra = (uint32_t)(((uint64_t)j * Rg) / cpg), rb = (uint32_t)(((uint64_t)(j + 1u) * Rg) / cpg);
  // blocks owning the rows of the cyclic interval [ra - W, rb + W)
  uint32_t dlo = 0, ndep = cpg;
  if (rb - ra + 2u * W < Rg) {
    dlo = owner((ra + Rg - W) % Rg, cpg, Rg);
    const uint32_t dhi = owner((rb - 1u + W) % Rg, cpg, Rg);
    ndep = (dhi + cpg - dlo) % cpg + 1u;
  }
  if (threadIdx.x < 32) sh.lut[threadIdx.x] = (uint8_t)lut_of(threadIdx.x);
  if (threadIdx.x == 0) s_abort = 0;
  Ctx c;
  c.keys = &p.keys;
  c.sp0 = p.spins + (uint64_t)g * R * kJitSites;
  const uint64_t* Jg = p.J + (uint64_t)g * D * kJitSites;
  const uint64_t t0 = (uint64_t)pp.t0_lo | ((uint64_t)pp.t0_hi << 32);
  for (uint32_t pass = 0; pass < pp.npass; ++pass) {
    const uint64_t t = t0 + (pass >> 1);
    const Tick tk{(uint32_t)t, (uint32_t)(t >> 32)};
    if ((pass & 1u) == 0u) {  // a new sweep: its uniform Philox parts
      fill_uniform(sh, g, tk, p.keys);
      __syncthreads();
    }
    c.thi_k = tk.hi ^ p.keys.k1[0];
    c.colour = (int)(pass & 1u);
    // the Philox blocks of the first sites depend on the sweep only: drawn
    // while the neighbours may still be finishing the previous pass
    draw_first(sh, min(ra * h + threadIdx.x, kJitGeom.half - 1u), c);
    if (pass > 0u) {
      if (threadIdx.x < 32u) {
        bool ok = true;
        for (uint32_t d = threadIdx.x; d < ndep; d += 32u) {
          const uint32_t blk = g * cpg + (dlo + d) % cpg;
          if (blk != b && ok) ok = wait_flag(pp.flags + blk, pass, pp.timeout_ns);
        }
        if (!__all_sync(kFull, ok) && threadIdx.x == 0) {
          atomicOr(pp.err, ERR_TIMEOUT);
          s_abort = 1;
        }
        __threadfence();
      }
      __syncthreads();
      if (s_abort) return;
    }
    sweep_words(sh, c, Jg, ra * h, rb * h, true);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(pp.flags + b), "r"(pass + 1u) : "memory");
    }
  }
}

#endif
