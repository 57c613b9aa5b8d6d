// sweep_planes.cuh -- the bit-sliced sweep against per-lane threshold planes
// (every lane may be at its own temperature: parallel tempering, several
// temperatures, lattices below the size where the lane-uniform kernel is
// specialised).  Shared by the precompiled kernels of k_msc.cu (geometry
// from the launch parameters) and by a kernel compiled at run time by jit.cu
// (IANUS_JIT_PLANES, geometry as constants).
//
// Update cell (Sec. 3.2) in bit-sliced form, per word: the unsatisfied-bond
// words e_j = b_i ^ b_j ^ c_ij, their count u as bit-planes (u2 u1 u0), and
// the lazy compare of the lane's random number against its class threshold
// from the most significant plane down.
#pragma once
#include "common.cuh"

namespace ianus {
namespace planes {

constexpr int kPlanesBlock = 256;

// ALGO 0 = Metropolis (only classes u < D need a random number),
// ALGO 1 = heat bath (all 2D+1 classes).
//
// The generic kernel below draws against per-lane threshold planes staged in
// shared memory (every lane may be at its own temperature).  A warp's 32
// words need different numbers of plane pairs; for the heat bath (~4 pairs a
// word on average, ~6.5 for the slowest of 32) the lazy compare runs in two
// phases: the first kPhaseA pairs in lockstep, then the words still
// undecided go to a per-warp queue in shared memory, and whenever 32 are
// queued the warp finishes them together.  Every word is written once, by
// the lane that finishes it; a colour-c pass writes colour-c words only, so
// the order of the writes does not matter.  Metropolis words need fewer
// pairs (only the classes with dE > 0 draw), and there the queue's registers
// cost more occupancy than it saves: each word runs to the end in place.

constexpr int kWarpsPerBlock = kPlanesBlock / 32;
constexpr uint32_t kQueue = 64;  // < 32 left + <= 32 pushed

// Undecided words of one warp: class planes, lazy-compare state, where the
// word goes and which replica (a) of the block it belongs to.
struct WordQueue {
  uint64_t u0[kQueue], u1[kQueue], u2[kQueue], und[kQueue], lt[kQueue];
  uint32_t self[kQueue], site[kQueue], a[kQueue];
};

// Shared memory of the generic kernel: R replicas' threshold planes, their
// Philox parts shared by the block ([R][16] uint4), then the warps' queues
// (Q).
// Blocks of more replicas than this compute the shared Philox parts inline
// instead of staging them (their planes alone nearly fill shared memory).
constexpr int kUniformMaxR = 64;

__host__ __device__ inline uint64_t bits_sweep_smem(int R, bool Q = true) {
  return (uint64_t)R * kPlanes * kMaxClasses * sizeof(uint64_t) + (R <= kUniformMaxR ? (uint64_t)R * 16 * 16 : 0) +
         (Q ? kWarpsPerBlock * sizeof(WordQueue) : 0);
}

// Plane pairs before a heat-bath word can be queued.
constexpr uint32_t kPhaseA = 4u;

struct LazyWord {
  uint64_t u0, u1, u2, und, lt;
};

// Threshold bit-plane of the lanes' classes: row[u] selected by the class
// bits (u2 u1 u0) with a tree of bitwise multiplexers (x ? a : b is one
// lop3).  Only undecided lanes use the result, and their classes take a
// random: u < D for Metropolis (so u2 = 0, and u1 = 0 in 2D), u <= 2D for the
// heat bath (u = 7 never occurs, so class 6 needs no partner).
template <int D, int ALGO>
__device__ __forceinline__ uint64_t class_select(const uint64_t* row, uint64_t u0, uint64_t u1, uint64_t u2) {
  auto mux = [](uint64_t x, uint64_t a, uint64_t b) { return (x & a) | (~x & b); };
  if (ALGO == 0) {
    const uint64_t t01 = mux(u0, row[1], row[0]);
    return D == 3 ? mux(u1, row[2], t01) : t01;
  }
  const uint64_t a = mux(u0, row[1], row[0]), b = mux(u0, row[3], row[2]);
  const uint64_t lo = mux(u1, b, a);
  if (D == 2) return mux(u2, row[4], lo);
  const uint64_t c = mux(u0, row[5], row[4]);
  return mux(u2, mux(u1, row[6], c), lo);
}

// Philox rounds 0 and 1 of the plane stream, counter (site, t_lo, c2, t_hi),
// split: the products of round 0 are M0 site and M1 c2, so after round 1
// the state is (s1 ^ u1, s2, u2 ^ s3, u3) with s from the site and the
// sweep's high word only (the site key, once per site and sweep) and u from
// c2 and the sweep's low word only (once per plane pair, slot and sweep,
// shared by every site of a block).  Rounds 2..9 then run as usual.
struct PlaneSiteKey {
  uint32_t s1, s2, s3;
};

__device__ __forceinline__ PlaneSiteKey plane_site_key(uint32_t site, const Tick& tk, const PhiloxKeys& K) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * site;
  const uint32_t b = (uint32_t)(p0 >> 32) ^ tk.hi ^ K.k1[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * b;
  return PlaneSiteKey{(uint32_t)(p1 >> 32), (uint32_t)p1, (uint32_t)p0};
}

// The shared part of counter word c2 (w unused).
__device__ __forceinline__ uint4 plane_uniform(uint32_t c2, const Tick& tk, const PhiloxKeys& K) {
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
  const uint32_t a = (uint32_t)(p1 >> 32) ^ tk.lo ^ K.k0[0];
  const uint64_t p0 = (uint64_t)0xD2511F53u * a;
  return make_uint4((uint32_t)p1 ^ K.k0[1], (uint32_t)(p0 >> 32) ^ K.k1[1], (uint32_t)p0, 0u);
}

__device__ __forceinline__ uint4 philox10_split(const PlaneSiteKey& s, const uint4& u, const PhiloxKeys& K) {
  uint32_t c0 = s.s1 ^ u.x, c1 = s.s2, c2 = u.y ^ s.s3, c3 = u.z;
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ K.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ K.k1[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Shared parts of the 16 plane pairs of `slots` consecutive slots
// sigma0.. of group g (counter word c2 = TAG_SPIN | pair | slot | group):
// u[a * 16 + m], filled by the block's threads.
__device__ __forceinline__ void plane_uniform_table(uint4* u, int slots, int sigma0, uint32_t g, const Tick& tk,
                                                    const PhiloxKeys& K) {
  for (int i = (int)threadIdx.x; i < slots * 16; i += (int)blockDim.x) {
    const uint32_t a = (uint32_t)i >> 4, m = (uint32_t)i & 15u;
    const uint32_t c2 = (TAG_SPIN << 28) | (m << 24) | ((uint32_t)(sigma0 + (int)a) << 12) | g;
    u[i] = plane_uniform(c2, tk, K);
  }
}

// Plane pairs mm0, mm0 + 1, ... (below mm_end) of one word against the
// per-lane planes tpa, two Philox blocks at a time (two independent round
// chains in flight), from the site key and the slot's shared parts ua[16]
// (null: computed here from the slot's counter word c2base and tk); stops
// when every lane is decided.
template <int D, int ALGO>
__device__ __forceinline__ void bits_plane_pairs(LazyWord& w, const uint64_t* tpa, const uint4* ua,
                                                 const PlaneSiteKey& sk, const PhiloxKeys& keys, uint32_t c2base,
                                                 const Tick& tk, uint32_t mm0, uint32_t mm_end) {
  uint64_t und = w.und, lt = w.lt;
#pragma unroll 1
  for (uint32_t mm = mm0; mm < mm_end && und != 0ull; mm += 2u) {
    const uint4 ma = ua ? ua[mm] : plane_uniform(c2base | (mm << 24), tk, keys);
    const uint4 mb = ua ? ua[mm + 1u] : plane_uniform(c2base | ((mm + 1u) << 24), tk, keys);
    const uint4 xa = philox10_split(sk, ma, keys);
    const uint4 xb = philox10_split(sk, mb, keys);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4& x = q < 2 ? xa : xb;
      const uint64_t r = (q & 1) == 0 ? ((uint64_t)x.x | ((uint64_t)x.y << 32))
                                      : ((uint64_t)x.z | ((uint64_t)x.w << 32));
      const uint64_t tb = class_select<D, ALGO>(tpa + (2u * mm + (uint32_t)q) * kMaxClasses, w.u0, w.u1, w.u2);
      lt |= und & ~r & tb;
      und &= ~(r ^ tb);
    }
  }
  w.und = und;
  w.lt = lt;
}

// Start of a word's lazy compare: lanes that always flip (threshold 2^32)
// are decided, and for Metropolis so are the lanes with dE <= 0 (u >= D,
// which are among them).
template <int D, int ALGO>
__device__ __forceinline__ LazyWord bits_word_start(const uint64_t* tpa, uint64_t u0, uint64_t u1, uint64_t u2) {
  LazyWord w;
  w.u0 = u0;
  w.u1 = u1;
  w.u2 = u2;
  const uint64_t always = class_select<D, 1>(tpa + 32 * kMaxClasses, u0, u1, u2);
  w.lt = always;
  // Metropolis: u < D draws (3D: u2 = 0 and not u = 3; 2D: u2 = u1 = 0)
  const uint64_t need = D == 3 ? ~u2 & ~(u1 & u0) : ~u2 & ~u1;
  w.und = (ALGO == 0) ? (~always & need) : ~always;
  return w;
}

// Class planes of one replica's word: the spin word b and the count of
// unsatisfied bonds as bit-planes.
template <int D>
__device__ __forceinline__ void bits_class_planes(const uint64_t* sp, const Nbr& n, const uint64_t* jw, uint64_t& b,
                                                  uint64_t& u0, uint64_t& u1, uint64_t& u2) {
  b = sp[n.self];
  uint64_t e[2 * D];
  e[0] = b ^ sp[n.xp] ^ jw[0];
  e[1] = b ^ sp[n.xm] ^ jw[1];
  e[2] = b ^ sp[n.yp] ^ jw[2];
  e[3] = b ^ sp[n.ym] ^ jw[3];
  if (D == 3) {
    e[4] = b ^ sp[n.zp] ^ jw[4];
    e[5] = b ^ sp[n.zm] ^ jw[5];
  }
  count_unsat<D>(e, u0, u1, u2);
}

// Everything a word's update needs besides its own state.
struct SweepCtx {
  const BitsParams* p;
  const uint64_t* tp;  // shared-memory planes of the block's replicas
  const uint4* U;      // shared-memory Philox parts of the block's replicas, [R][16] (null above kUniformMaxR)
  uint64_t* sp0;       // spins of the block's first replica
  Tick tk;
  int g, tslot, R;
};

// Counter word c2 of replica a's plane stream without the pair (bits 24..27).
__device__ __forceinline__ uint32_t bits_c2(const SweepCtx& c, uint32_t a) {
  const uint32_t sigma = (uint32_t)(c.tslot * c.R) + a;
  return (TAG_SPIN << 28) | (sigma << 12) | (uint32_t)c.g;
}

__device__ __forceinline__ const uint4* bits_u(const SweepCtx& c, uint32_t a) { return c.U ? c.U + 16u * a : nullptr; }

// Warp-wide append of the lanes with pred set; n is warp-uniform.
__device__ __forceinline__ void queue_push(WordQueue& q, uint32_t& n, bool pred, const LazyWord& w, uint32_t self,
                                           uint32_t site, uint32_t a) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t mk = __ballot_sync(0xffffffffu, pred);
  if (pred) {
    const uint32_t i = n + __popc(mk & ((1u << lane) - 1u));
    q.u0[i] = w.u0;
    q.u1[i] = w.u1;
    q.u2[i] = w.u2;
    q.und[i] = w.und;
    q.lt[i] = w.lt;
    q.self[i] = self;
    q.site[i] = site;
    q.a[i] = a;
  }
  n += __popc(mk);
  __syncwarp();
}

// Finish the top `take` (<= 32) queued words: pairs kPhaseA.. to the end.
template <int D, int ALGO>
__device__ __forceinline__ void queue_round(WordQueue& q, uint32_t& n, uint32_t take, const SweepCtx& c) {
  const uint32_t lane = threadIdx.x & 31u;
  const bool has = lane < take;
  LazyWord w;
  w.u0 = w.u1 = w.u2 = w.und = w.lt = 0;
  uint32_t self = 0, site = 0, a = 0;
  if (has) {
    const uint32_t i = n - take + lane;
    w.u0 = q.u0[i];
    w.u1 = q.u1[i];
    w.u2 = q.u2[i];
    w.und = q.und[i];
    w.lt = q.lt[i];
    self = q.self[i];
    site = q.site[i];
    a = q.a[i];
  }
  __syncwarp();
  n -= take;
  if (has) {
    bits_plane_pairs<D, ALGO>(w, c.tp + (uint64_t)a * kPlanes * kMaxClasses, bits_u(c, a),
                              plane_site_key(site, c.tk, c.p->keys), c.p->keys, bits_c2(c, a), c.tk, kPhaseA, 16u);
    uint64_t* sp = c.sp0 + (uint64_t)a * c.p->geom.N;
    const uint64_t flip = (ALGO == 0) ? w.lt : ~w.lt;
    if (flip) sp[self] ^= flip;
  }
}

// Phase A of one replica's word, then either its write or its place in the
// queue (Q); without the queue, all its plane pairs and its write.
template <int D, int ALGO, bool Q>
__device__ __forceinline__ void bits_update(WordQueue& q, uint32_t& nq, const SweepCtx& c, bool valid, const Nbr& n,
                                            const PlaneSiteKey& sk, uint32_t a, uint64_t b, uint64_t u0, uint64_t u1,
                                            uint64_t u2) {
  const uint64_t* tpa = c.tp + (uint64_t)a * kPlanes * kMaxClasses;
  LazyWord w;
  w.und = 0;
  if (valid) {
    w = bits_word_start<D, ALGO>(tpa, u0, u1, u2);
    bits_plane_pairs<D, ALGO>(w, tpa, bits_u(c, a), sk, c.p->keys, bits_c2(c, a), c.tk, 0u, Q ? kPhaseA : 16u);
  }
  if (!Q) {
    const uint64_t flip = (ALGO == 0) ? w.lt : ~w.lt;
    if (valid && flip) c.sp0[(uint64_t)a * c.p->geom.N + n.self] = b ^ flip;
    return;
  }
  const bool pend = valid && w.und != 0ull;
  queue_push(q, nq, pend, w, valid ? n.self : 0u, valid ? n.site : 0u, a);
  if (valid && !pend) {
    const uint64_t flip = (ALGO == 0) ? w.lt : ~w.lt;
    if (flip) c.sp0[(uint64_t)a * c.p->geom.N + n.self] = b ^ flip;
  }
  if (nq >= 32u) queue_round<D, ALGO>(q, nq, 32u, c);
}

// With a compile-time replica count RT, the class planes of every replica of
// a word are computed before the first replica's update, so that all the
// word's loads are in flight together; with RT = 0 the replicas go in turn.
template <int D, int ALGO, int RT, bool P2, bool Q>
__device__ __forceinline__ void sweep_planes_body(const BitsParams& p, const Geom& geom) {
  extern __shared__ uint64_t sm_tp[];  // [R][kPlanes][kMaxClasses], [R][16] Philox parts, then the queues
  const int R = RT > 0 ? RT : p.R;
  const int gt = blockIdx.y;  // g * K + tslot
  const int g = gt / p.K, tslot = gt - g * p.K;
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  uint4* sm_u = reinterpret_cast<uint4*>(sm_tp + (uint64_t)R * kPlanes * kMaxClasses);
  const bool staged_u = R <= kUniformMaxR;
  // stage this block's threshold planes and Philox parts
  {
    const uint64_t* src = p.tp + ((uint64_t)g * p.slots + (uint64_t)tslot * R) * kPlanes * kMaxClasses;
    for (int k = threadIdx.x; k < R * kPlanes * kMaxClasses; k += kPlanesBlock) sm_tp[k] = src[k];
    if (staged_u) plane_uniform_table(sm_u, R, tslot * R, (uint32_t)g, tk, p.keys);
  }
  __syncthreads();
  WordQueue& q = reinterpret_cast<WordQueue*>(sm_u + (staged_u ? (uint64_t)R * 16 : 0))[threadIdx.x >> 5];
  uint32_t nq = 0;
  const uint32_t N = geom.N;
  const uint64_t* Jg = p.J + (uint64_t)g * D * N;
  SweepCtx c;
  c.p = &p;
  c.tp = sm_tp;
  c.U = staged_u ? sm_u : nullptr;
  c.sp0 = p.spins + ((uint64_t)g * p.slots + (uint64_t)tslot * R) * N;
  c.tk = tk;
  c.g = g;
  c.tslot = tslot;
  c.R = R;
  const uint32_t w_begin = blockIdx.x * p.words_per_block;
  const uint32_t w_end = min(w_begin + p.words_per_block, geom.half);
  for (uint32_t base = w_begin; base < w_end; base += kPlanesBlock) {  // uniform across the block
    const uint32_t wi = base + threadIdx.x;
    const bool valid = wi < w_end;
    if (!Q && !valid) break;  // without the queue, threads need not stay together
    Nbr n;
    n.self = n.site = 0;
    uint64_t jw[2 * D];
    if (valid) {
      n = split_neighbours_t<P2>(geom, p.colour, wi);
      jw[0] = __ldg(Jg + n.self);
      jw[1] = __ldg(Jg + n.xm);
      jw[2] = __ldg(Jg + N + n.self);
      jw[3] = __ldg(Jg + N + n.ym);
      if (D == 3) {
        jw[4] = __ldg(Jg + 2u * N + n.self);
        jw[5] = __ldg(Jg + 2u * N + n.zm);
      }
    }
    const PlaneSiteKey sk = plane_site_key(n.site, c.tk, p.keys);  // shared by the word's replicas
    if (RT > 0) {
      uint64_t b[RT > 0 ? RT : 1], u0[RT > 0 ? RT : 1], u1[RT > 0 ? RT : 1], u2[RT > 0 ? RT : 1];
#pragma unroll
      for (int a = 0; a < RT; ++a) {
        b[a] = u0[a] = u1[a] = u2[a] = 0;
        if (valid) bits_class_planes<D>(c.sp0 + (uint64_t)a * N, n, jw, b[a], u0[a], u1[a], u2[a]);
      }
#pragma unroll
      for (int a = 0; a < RT; ++a)
        bits_update<D, ALGO, Q>(q, nq, c, valid, n, sk, (uint32_t)a, b[a], u0[a], u1[a], u2[a]);
    } else {
#pragma unroll 1
      for (int a = 0; a < R; ++a) {
        uint64_t b = 0, u0 = 0, u1 = 0, u2 = 0;
        if (valid) bits_class_planes<D>(c.sp0 + (uint64_t)a * N, n, jw, b, u0, u1, u2);
        bits_update<D, ALGO, Q>(q, nq, c, valid, n, sk, (uint32_t)a, b, u0, u1, u2);
      }
    }
  }
  if (Q && nq > 0u) queue_round<D, ALGO>(q, nq, nq, c);
}


}  // namespace planes
}  // namespace ianus

#ifdef IANUS_JIT_PLANES
// Run-time compiled instance: IANUS_JIT_D, IANUS_JIT_ALGO, IANUS_JIT_RT (1, 2,
// or 0 for a run-time replica count), IANUS_JIT_P2, IANUS_JIT_Q (per-warp
// queues), IANUS_JIT_MINB (blocks per SM) and the geometry macros of
// common.cuh.
extern "C" __global__ void __launch_bounds__(ianus::planes::kPlanesBlock, IANUS_JIT_MINB)
    ianus_jit_planes_sweep(const ianus::BitsParams p) {
  constexpr ianus::Geom geom = ianus::kJitGeom;
  ianus::dependent_launch_entry();
  ianus::planes::sweep_planes_body<IANUS_JIT_D, IANUS_JIT_ALGO, IANUS_JIT_RT, IANUS_JIT_P2 != 0, IANUS_JIT_Q != 0>(
      p, geom);
}
#endif
