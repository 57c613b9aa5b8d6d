// k_msc.cu -- the bit-sliced multispin layout (IANUS_LAYOUT_BITS64).
//
// A 64-bit word holds one site of 64 independent disorder samples (lane l =
// sample mod 64), the multi-sample idea of Sec. 4.1.1 carried to a GPU word,
// with an independent random stream per sample.  Words of one colour are
// stored next to each other (checkerboard-split order, Sec. 3.1), so the own
// word, the 2D neighbour words and the coupling words of a warp are
// contiguous loads.
//
// Update cell (Sec. 3.2) in bit-sliced form, per word:
//   e_j = b_i ^ b_j ^ c_ij                    unsatisfied-bond bits (2D words)
//   (u2,u1,u0) = carry-save adder tree of the e_j  (u = 0..2D per lane)
//   m_u = lanes whose count is u              (class masks)
//   threshold bit-plane p: t_p = OR_u (m_u & TP[u][p])
//   lazy compare from the most significant plane: lanes stay undecided while
//   their random bit equals the threshold bit; lt collects r < T.
//   flip = lt ^ inv (Metropolis: inv = 0; heat bath: inv = ~0)
// TP[u][p] are 64-bit lane masks, so every lane can carry its own threshold
// (parallel tempering moves temperatures per sample).
#include <algorithm>
#include <cmath>

#include "lattice.h"
#include "sweep_planes.cuh"

namespace ianus {

namespace {

constexpr int kBlock = 256;

using planes::bits_sweep_smem;
using planes::class_select;

// The per-lane-plane sweep, precompiled (sweep_planes.cuh).
template <int D, int ALGO, int RT, bool P2, bool Q = (ALGO == 1)>
__global__ void __launch_bounds__(kBlock, Q ? 3 : 4) k_sweep_bits(const BitsParams p) {
  planes::sweep_planes_body<D, ALGO, RT, P2, Q>(p, p.geom);
}

// Random-field model (Eq. 2 with h_i = +-|h|, x_i = 1): the class of a lane
// is (u, f) with f = [s_i h_i > 0] = ~(b_i ^ hb_i), hb_i = lane bit set
// where h_i < 0.  TP[p][8 f + u] are per-lane threshold planes as above; a
// lane with T = 2^32 is decided without a random number, every other lane
// compares (T = 0 lanes end at the first set bit of r).
template <int D, int ALGO, bool P2>
__global__ void __launch_bounds__(kBlock) k_sweep_bits_field(const BitsParams p, const uint64_t* __restrict__ hbits) {
  constexpr int NF = kFieldPlaneClasses;
  extern __shared__ uint64_t sm_tp[];  // [R][kPlanes][NF]
  const int R = p.R;
  const int gt = blockIdx.y;
  const int g = gt / p.K, tslot = gt - g * p.K;
  {
    const uint64_t* src = p.tp + ((size_t)g * p.slots + (size_t)tslot * R) * kPlanes * NF;
    for (int k = threadIdx.x; k < R * kPlanes * NF; k += kBlock) sm_tp[k] = src[k];
  }
  __syncthreads();
  const Geom geom = p.geom;
  const uint32_t N = geom.N;
  const uint64_t* Jg = p.J + (size_t)g * D * N;
  const uint64_t* Hg = hbits + (size_t)g * N;
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  const uint32_t w_begin = blockIdx.x * p.words_per_block;
  const uint32_t w_end = min(w_begin + p.words_per_block, geom.half);
  for (uint32_t w = w_begin + threadIdx.x; w < w_end; w += kBlock) {
    const Nbr n = split_neighbours_t<P2>(geom, p.colour, w);
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
#pragma unroll 1
    for (int a = 0; a < R; ++a) {
      const int sigma = tslot * R + a;
      uint64_t* sp = p.spins + ((size_t)g * p.slots + sigma) * N;
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
      uint64_t u0, u1, u2;
      count_unsat<D>(e, u0, u1, u2);
      const uint64_t f = ~(b ^ hb);
      uint64_t mc[2][2 * D + 1];
#pragma unroll
      for (int u = 0; u <= 2 * D; ++u) {
        const uint64_t m = ((u & 4) ? u2 : ~u2) & ((u & 2) ? u1 : ~u1) & ((u & 1) ? u0 : ~u0);
        mc[0][u] = m & ~f;
        mc[1][u] = m & f;
      }
      const uint64_t* tpa = sm_tp + (size_t)a * kPlanes * NF;
      uint64_t always = 0;
#pragma unroll
      for (int u = 0; u <= 2 * D; ++u)
        always |= (mc[0][u] & tpa[32 * NF + u]) | (mc[1][u] & tpa[32 * NF + 8 + u]);
      uint64_t lt = always;
      uint64_t und = ~always;
      const uint32_t c2 = (TAG_SPIN << 28) | ((uint32_t)sigma << 12) | (uint32_t)g;
#pragma unroll 1
      for (uint32_t mm = 0; mm < 16u && und != 0ull; ++mm) {
        const uint4 x = philox10(n.site, tk.lo, c2 | (mm << 24), tk.hi, p.keys);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const uint64_t r = q == 0 ? ((uint64_t)x.x | ((uint64_t)x.y << 32))
                                    : ((uint64_t)x.z | ((uint64_t)x.w << 32));
          const uint64_t* row = tpa + (2u * mm + (uint32_t)q) * NF;
          uint64_t tb = 0;
#pragma unroll
          for (int u = 0; u <= 2 * D; ++u) tb |= (mc[0][u] & row[u]) | (mc[1][u] & row[8 + u]);
          lt |= und & ~r & tb;
          und &= ~(r ^ tb);
        }
      }
      const uint64_t flip = (ALGO == 0) ? lt : ~lt;
      if (flip) sp[n.self] = b ^ flip;
    }
  }
}

// Diluted model (DAFF; Eq. 2 with x_i in {0,1}), generic per-lane planes.
// Per neighbour j the bond contributes c_j = x_j (1 - 2 e_j) to v (e_j the
// unsatisfied bit); c_j + 1 in {0, 1, 2} is 2 hi_j + lo_j with hi_j = x_j &
// ~e_j and lo_j = ~x_j, so t = v + 2D = 2 sum(hi) + sum(lo), 4 bit-planes.
// The plane class is 16 f + t.  Empty sites are never updated.
template <int D, int ALGO, bool P2>
__global__ void __launch_bounds__(kBlock) k_sweep_bits_dilute(const BitsParams p, const uint64_t* __restrict__ hbits,
                                                              const uint64_t* __restrict__ xbits) {
  constexpr int NF = kDiluteClasses;
  constexpr int NT = 4 * D + 1;  // t = 0..4D
  extern __shared__ uint64_t sm_tp[];  // [R][kPlanes][NF]
  const int R = p.R;
  const int gt = blockIdx.y;
  const int g = gt / p.K, tslot = gt - g * p.K;
  {
    const uint64_t* src = p.tp + ((size_t)g * p.slots + (size_t)tslot * R) * kPlanes * NF;
    for (int k = threadIdx.x; k < R * kPlanes * NF; k += kBlock) sm_tp[k] = src[k];
  }
  __syncthreads();
  const Geom geom = p.geom;
  const uint32_t N = geom.N;
  const uint64_t* Jg = p.J + (size_t)g * D * N;
  const uint64_t* Hg = hbits + (size_t)g * N;
  const uint64_t* Xg = xbits + (size_t)g * N;
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  const uint32_t w_begin = blockIdx.x * p.words_per_block;
  const uint32_t w_end = min(w_begin + p.words_per_block, geom.half);
  for (uint32_t w = w_begin + threadIdx.x; w < w_end; w += kBlock) {
    const Nbr n = split_neighbours_t<P2>(geom, p.colour, w);
    uint64_t jw[2 * D], xw[2 * D];
    jw[0] = __ldg(Jg + n.self);
    jw[1] = __ldg(Jg + n.xm);
    jw[2] = __ldg(Jg + N + n.self);
    jw[3] = __ldg(Jg + N + n.ym);
    xw[0] = __ldg(Xg + n.xp);
    xw[1] = __ldg(Xg + n.xm);
    xw[2] = __ldg(Xg + n.yp);
    xw[3] = __ldg(Xg + n.ym);
    if (D == 3) {
      jw[4] = __ldg(Jg + 2u * N + n.self);
      jw[5] = __ldg(Jg + 2u * N + n.zm);
      xw[4] = __ldg(Xg + n.zp);
      xw[5] = __ldg(Xg + n.zm);
    }
    const uint64_t hb = __ldg(Hg + n.self), xs = __ldg(Xg + n.self);
    uint64_t lo[2 * D];
#pragma unroll
    for (int j = 0; j < 2 * D; ++j) lo[j] = ~xw[j];
    uint64_t l0, l1, l2;
    count_unsat<D>(lo, l0, l1, l2);  // sum of lo_j
#pragma unroll 1
    for (int a = 0; a < R; ++a) {
      const int sigma = tslot * R + a;
      uint64_t* sp = p.spins + ((size_t)g * p.slots + sigma) * N;
      const uint64_t b = sp[n.self];
      uint64_t hi[2 * D];
      hi[0] = xw[0] & ~(b ^ sp[n.xp] ^ jw[0]);
      hi[1] = xw[1] & ~(b ^ sp[n.xm] ^ jw[1]);
      hi[2] = xw[2] & ~(b ^ sp[n.yp] ^ jw[2]);
      hi[3] = xw[3] & ~(b ^ sp[n.ym] ^ jw[3]);
      if (D == 3) {
        hi[4] = xw[4] & ~(b ^ sp[n.zp] ^ jw[4]);
        hi[5] = xw[5] & ~(b ^ sp[n.zm] ^ jw[5]);
      }
      uint64_t h0, h1, h2;
      count_unsat<D>(hi, h0, h1, h2);
      // t = 2 (h2 h1 h0) + (l2 l1 l0) <= 4D < 16
      const uint64_t t0 = l0, t1 = h0 ^ l1, k1 = h0 & l1;
      const uint64_t t2 = h1 ^ l2 ^ k1, k2 = (h1 & l2) | (h1 & k1) | (l2 & k1);
      const uint64_t t3 = h2 ^ k2;
      const uint64_t f = ~(b ^ hb);
      uint64_t mc[2][NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const uint64_t m = ((t & 8) ? t3 : ~t3) & ((t & 4) ? t2 : ~t2) & ((t & 2) ? t1 : ~t1) & ((t & 1) ? t0 : ~t0);
        mc[0][t] = m & ~f;
        mc[1][t] = m & f;
      }
      const uint64_t* tpa = sm_tp + (size_t)a * kPlanes * NF;
      uint64_t always = 0;
#pragma unroll
      for (int t = 0; t < NT; ++t) always |= (mc[0][t] & tpa[32 * NF + t]) | (mc[1][t] & tpa[32 * NF + 16 + t]);
      always &= xs;
      uint64_t lt = always;
      uint64_t und = ~always & xs;
      const uint32_t c2 = (TAG_SPIN << 28) | ((uint32_t)sigma << 12) | (uint32_t)g;
#pragma unroll 1
      for (uint32_t mm = 0; mm < 16u && und != 0ull; ++mm) {
        const uint4 x = philox10(n.site, tk.lo, c2 | (mm << 24), tk.hi, p.keys);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const uint64_t r = q == 0 ? ((uint64_t)x.x | ((uint64_t)x.y << 32))
                                    : ((uint64_t)x.z | ((uint64_t)x.w << 32));
          const uint64_t* row = tpa + (2u * mm + (uint32_t)q) * NF;
          uint64_t tb = 0;
#pragma unroll
          for (int t = 0; t < NT; ++t) tb |= (mc[0][t] & row[t]) | (mc[1][t] & row[16 + t]);
          lt |= und & ~r & tb;
          und &= ~(r ^ tb);
        }
      }
      const uint64_t flip = ((ALGO == 0) ? lt : ~lt) & xs;
      if (flip) sp[n.self] = b ^ flip;
    }
  }
}

// Site disorder of the bit-sliced field models, lane bit l of word (g, i)
// for sample 64 g + l: hbits = [h_i < 0] (RFIM: the H stream; DAFF: 0),
// xbits = [x_i = 1] (RFIM: all; DAFF: r_x < T_occ, r_x from the 32 planes of
// the X stream compared from the most significant plane down).
__global__ void k_init_sites_bits(uint64_t* hbits, uint64_t* xbits, Geom geom, int G, int rfim, int daff,
                                  uint64_t T_occ, PhiloxKeys keys) {
  const uint64_t total = (uint64_t)G * geom.N;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t g = (uint32_t)(idx / geom.N), i = (uint32_t)(idx - (uint64_t)g * geom.N);
    const uint32_t L = (uint32_t)geom.L;
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    const size_t j = (size_t)g * geom.N + split_index(geom, x, y, z);
    uint64_t hw = 0, xw = ~0ull;
    if (rfim) {
      const uint4 r = philox10(i, 0u, (TAG_H << 28) | g, 0u, keys);
      hw = (uint64_t)r.x | ((uint64_t)r.y << 32);
    }
    if (daff) {
      if (T_occ >= kTwo32) {
        xw = ~0ull;
      } else {
        uint64_t lt = 0, und = ~0ull;
        for (uint32_t m = 0; m < 16u && und != 0ull; ++m) {
          const uint4 r = philox10(i, 0u, (TAG_X << 28) | (m << 24) | g, 0u, keys);
          for (int q = 0; q < 2; ++q) {
            const uint64_t w = q == 0 ? ((uint64_t)r.x | ((uint64_t)r.y << 32)) : ((uint64_t)r.z | ((uint64_t)r.w << 32));
            const uint64_t tb = ((T_occ >> (31u - (2u * m + (uint32_t)q))) & 1ull) ? ~0ull : 0ull;
            lt |= und & ~w & tb;
            und &= ~(w ^ tb);
          }
        }
        xw = lt;
      }
    }
    hbits[j] = hw;
    xbits[j] = xw;
  }
}

__global__ void k_get_sites_bits(const uint64_t* hbits, const uint64_t* xbits, int8_t* out_hs, int8_t* out_occ,
                                 Geom geom, int S) {
  const uint64_t total = (uint64_t)S * geom.N;
  const uint32_t L = (uint32_t)geom.L;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(idx % geom.N);
    const int s = (int)(idx / geom.N);
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    const size_t j = (size_t)(s >> 6) * geom.N + split_index(geom, x, y, z);
    out_hs[idx] = ((hbits[j] >> (s & 63)) & 1ull) ? -1 : 1;
    out_occ[idx] = (int8_t)((xbits[j] >> (s & 63)) & 1ull);
  }
}

__global__ void k_set_sites_bits(uint64_t* hbits, uint64_t* xbits, const int8_t* in_hs, const int8_t* in_occ,
                                 Geom geom, int S, int G) {
  const uint64_t total = (uint64_t)G * geom.N;
  const uint32_t L = (uint32_t)geom.L;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(idx % geom.N);
    const int g = (int)(idx / geom.N);
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    const size_t j = (size_t)g * geom.N + split_index(geom, x, y, z);
    uint64_t hw = hbits[j], xw = xbits[j];
    for (int l = 0; l < 64; ++l) {
      const int s = 64 * g + l;
      if (s >= S) break;
      const uint64_t hbit = in_hs[(size_t)s * geom.N + i] < 0 ? 1ull : 0ull;
      const uint64_t xbit = in_occ[(size_t)s * geom.N + i] ? 1ull : 0ull;
      hw = (hw & ~(1ull << l)) | (hbit << l);
      xw = (xw & ~(1ull << l)) | (xbit << l);
    }
    hbits[j] = hw;
    xbits[j] = xw;
  }
}

// ---- fused serving: several jobs in the lanes of one group ----
//
// One block per (word range, group).  The block stages the group's per-lane
// threshold planes and its segment table.  Per plane pair, every segment
// that still has undecided lanes draws one Philox block from its own stream
// (key of the job's seed, counter of the job's sweep t, group 0, slot 0) and
// contributes its bits 0..n-1 shifted to its lanes.  Heat-bath lanes flip on
// "not less" (inv lanes), Metropolis lanes on "less"; lanes of no live
// segment never flip.
template <int D, bool P2>
__global__ void __launch_bounds__(kBlock) k_sweep_fused(const BitsParams p, const Segment* __restrict__ segs,
                                                        const uint32_t* __restrict__ nseg) {
  __shared__ uint64_t tpa[kPlanes * kMaxClasses];
  __shared__ uint64_t s_mask[kMaxSegs];
  __shared__ uint32_t s_klo[kMaxSegs], s_khi[kMaxSegs];
  __shared__ Tick s_t[kMaxSegs];
  __shared__ uint32_t s_lane0[kMaxSegs], s_c2[kMaxSegs];
  __shared__ int s_n;
  __shared__ uint64_t s_live, s_inv;
  const int g = blockIdx.y;
  for (int k = threadIdx.x; k < kPlanes * kMaxClasses; k += kBlock)
    tpa[k] = p.tp[(size_t)g * kPlanes * kMaxClasses + k];
  if (threadIdx.x == 0) {
    const uint32_t ns = min(nseg[g], (uint32_t)kMaxSegs);
    uint64_t live = 0, inv = 0;
    int n = 0;
    for (uint32_t j = 0; j < ns; ++j) {
      const Segment sg = segs[(size_t)g * kMaxSegs + j];
      if (sg.t >= sg.t_end || sg.mask == 0ull) continue;
      s_mask[n] = sg.mask;
      s_klo[n] = sg.key_lo;
      s_khi[n] = sg.key_hi;
      s_t[n] = Tick{(uint32_t)sg.t, (uint32_t)(sg.t >> 32)};
      s_lane0[n] = sg.lane0;
      s_c2[n] = (TAG_SPIN << 28) | sg.jgroup;  // slot 0, the job's own group
      live |= sg.mask;
      if (sg.inv) inv |= sg.mask;
      ++n;
    }
    s_n = n;
    s_live = live;
    s_inv = inv;
  }
  __syncthreads();
  const uint64_t live = s_live, inv = s_inv;
  const int nsg = s_n;
  if (live == 0ull) return;
  const Geom geom = p.geom;
  const uint32_t N = geom.N;
  const uint64_t* Jg = p.J + (size_t)g * D * N;
  uint64_t* sp = p.spins + (size_t)g * N;  // one slot per group
  const uint32_t w_begin = blockIdx.x * p.words_per_block;
  const uint32_t w_end = min(w_begin + p.words_per_block, geom.half);
  for (uint32_t w = w_begin + threadIdx.x; w < w_end; w += kBlock) {
    const Nbr n = split_neighbours_t<P2>(geom, p.colour, w);
    const uint64_t b = sp[n.self];
    uint64_t e[2 * D];
    e[0] = b ^ sp[n.xp] ^ __ldg(Jg + n.self);
    e[1] = b ^ sp[n.xm] ^ __ldg(Jg + n.xm);
    e[2] = b ^ sp[n.yp] ^ __ldg(Jg + N + n.self);
    e[3] = b ^ sp[n.ym] ^ __ldg(Jg + N + n.ym);
    if (D == 3) {
      e[4] = b ^ sp[n.zp] ^ __ldg(Jg + 2u * N + n.self);
      e[5] = b ^ sp[n.zm] ^ __ldg(Jg + 2u * N + n.zm);
    }
    uint64_t u0, u1, u2;
    count_unsat<D>(e, u0, u1, u2);
    // a segment's lanes may hold either algorithm's planes: select over all classes
    const uint64_t always = class_select<D, 1>(tpa + 32 * kMaxClasses, u0, u1, u2);
    uint64_t lt = always;
    uint64_t und = ~always & live;
#pragma unroll 1
    for (uint32_t mm = 0; mm < 16u && und != 0ull; ++mm) {
      uint64_t r0 = 0, r1 = 0;
#pragma unroll 1
      for (int j = 0; j < nsg; ++j) {
        const uint64_t mk = s_mask[j];
        if (!(und & mk)) continue;
        const uint4 x = philox10_key(n.site, s_t[j].lo, s_c2[j] | (mm << 24), s_t[j].hi, s_klo[j], s_khi[j]);
        const uint32_t sh = s_lane0[j];
        r0 |= (((uint64_t)x.x | ((uint64_t)x.y << 32)) << sh) & mk;
        r1 |= (((uint64_t)x.z | ((uint64_t)x.w << 32)) << sh) & mk;
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const uint64_t r = q == 0 ? r0 : r1;
        const uint64_t tb = class_select<D, 1>(tpa + (2u * mm + (uint32_t)q) * kMaxClasses, u0, u1, u2);
        lt |= und & ~r & tb;
        und &= ~(r ^ tb);
      }
    }
    const uint64_t flip = (lt ^ inv) & live;
    if (flip) sp[n.self] = b ^ flip;
  }
}

// A job's couplings and initial spins, as samples 64 jgroup + b of its own
// lattice (group jgroup, slot 0 of the J and INIT streams under the job's
// key), written into lanes lane0 + b of group g.
__global__ void k_load_segment(uint64_t* spins, uint64_t* J, Geom geom, int g, uint32_t lane0, uint64_t mask,
                               uint32_t jgroup, PhiloxKeys keys) {
  const uint32_t L = (uint32_t)geom.L;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < geom.N; i += gridDim.x * blockDim.x) {
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    const uint32_t j = split_index(geom, x, y, z);
    for (int d = 0; d < geom.D; ++d) {
      const uint4 r = philox10(i, (uint32_t)d, (TAG_J << 28) | jgroup, 0u, keys);
      uint64_t* wp = J + ((size_t)g * geom.D + d) * geom.N + j;
      *wp = (*wp & ~mask) | ((((uint64_t)r.x | ((uint64_t)r.y << 32)) << lane0) & mask);
    }
    const uint4 r = philox10(i, 0u, (TAG_INIT << 28) | jgroup, 0u, keys);
    uint64_t* wp = spins + (size_t)g * geom.N + j;
    *wp = (*wp & ~mask) | ((((uint64_t)r.x | ((uint64_t)r.y << 32)) << lane0) & mask);
  }
}

__global__ void k_advance_segments(Segment* segs, const uint32_t* nseg, int G) {
  const int total = G * kMaxSegs;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int g = idx / kMaxSegs, j = idx - g * kMaxSegs;
    if ((uint32_t)j >= nseg[g]) continue;
    Segment& sg = segs[idx];
    if (sg.mask != 0ull && sg.t < sg.t_end) sg.t += 1;
  }
}

// ---- initialisation: one Philox block gives the word of 64 samples ----

__global__ void k_init_bits(uint64_t* spins, uint64_t* J, Geom geom, int G, int slots, int jmode,
                            PhiloxKeys keys) {
  const uint64_t total = (uint64_t)G * geom.N;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t g = (uint32_t)(idx / geom.N), i = (uint32_t)(idx - (uint64_t)g * geom.N);
    const uint32_t L = (uint32_t)geom.L;
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    const uint32_t j = split_index(geom, x, y, z);
    for (int d = 0; d < geom.D; ++d) {
      const uint4 r = philox10(i, (uint32_t)d, (TAG_J << 28) | g, 0u, keys);
      J[((size_t)g * geom.D + d) * geom.N + j] =
          jmode == 1 ? 0ull : (jmode == 2 ? ~0ull : ((uint64_t)r.x | ((uint64_t)r.y << 32)));
    }
    for (int sg = 0; sg < slots; ++sg) {
      const uint4 r = philox10(i, 0u, (TAG_INIT << 28) | ((uint32_t)sg << 12) | g, 0u, keys);
      spins[((size_t)g * slots + sg) * geom.N + j] = (uint64_t)r.x | ((uint64_t)r.y << 32);
    }
  }
}

// ---- threshold planes: TP[g][sigma][p][u], bit l = bit (31-p) of T of the
// temperature sample 64g+l holds in slot sigma; plane 32 = (T == 2^32). ----

// Threshold planes of one 64-lane word, one warp each: thread t holds the
// thresholds of lanes t and 32 + t, and plane q is the ballot of bit 31 - q
// (plane 32: threshold 2^32, "always").  Thread q < 32 keeps plane q, and
// thread 0 also the always plane; the caller stores them.
__device__ __forceinline__ void warp_planes(uint64_t T_lo, uint64_t T_hi, uint64_t& mine, uint64_t& always) {
  const uint32_t lane = threadIdx.x & 31u;
  always = (uint64_t)__ballot_sync(0xffffffffu, T_lo >= kTwo32) |
           ((uint64_t)__ballot_sync(0xffffffffu, T_hi >= kTwo32) << 32);
  mine = 0;
#pragma unroll 4
  for (uint32_t q = 0; q < 32u; ++q) {
    const uint32_t lo = __ballot_sync(0xffffffffu, T_lo < kTwo32 && ((T_lo >> (31u - q)) & 1ull));
    const uint32_t hi = __ballot_sync(0xffffffffu, T_hi < kTwo32 && ((T_hi >> (31u - q)) & 1ull));
    if (lane == q) mine = (uint64_t)lo | ((uint64_t)hi << 32);
  }
}

// TP[g][sigma][p][u] from the per-temperature thresholds thr[k][u] of each
// lane's temperature, one warp per (group, slot, class).
__global__ void k_build_planes(uint64_t* tp, const uint64_t* thr, const int32_t* temp_of, int G, int S, int R,
                               int K, int slots) {
  const int total = G * slots * kMaxClasses;
  const uint32_t lane = threadIdx.x & 31u;
  for (int idx = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); idx < total;
       idx += (int)((gridDim.x * blockDim.x) >> 5)) {  // uniform across the warp
    const int u = idx % kMaxClasses, rest = idx / kMaxClasses;
    const int sigma = rest % slots, g = rest / slots;
    const int tslot = sigma / R, a = sigma - tslot * R;
    uint64_t T[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int s = 64 * g + 32 * h + (int)lane;
      const int k = s < S ? temp_of[((size_t)s * R + a) * K + tslot] : tslot;
      T[h] = thr[(size_t)k * kMaxClasses + u];
    }
    uint64_t mine, always;
    warp_planes(T[0], T[1], mine, always);
    uint64_t* out = tp + ((size_t)g * slots + sigma) * kPlanes * kMaxClasses + u;
    out[(size_t)lane * kMaxClasses] = mine;
    if (lane == 0) out[(size_t)32 * kMaxClasses] = always;
  }
}

// Field planes: FTP[g][sigma][p][8 f + u] from the per-temperature field
// thresholds fthr[k][(v + 2D) * 2 + f], v = 2D - 2u; classes u > 2D stay 0.
// With dilution (NF = kDiluteClasses) the class is 16 f + t, field class
// t * 2 + f; classes t > 4D stay 0.  One warp per (group, slot, class).
__global__ void k_build_field_planes(uint64_t* ftp, const uint64_t* fthr, const int32_t* temp_of, int D, int G,
                                     int S, int R, int K, int slots, int NF) {
  const int total = G * slots * NF;
  const uint32_t lane = threadIdx.x & 31u;
  for (int idx = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); idx < total;
       idx += (int)((gridDim.x * blockDim.x) >> 5)) {  // uniform across the warp
    const int c = idx % NF, rest = idx / NF;
    const int sigma = rest % slots, g = rest / slots;
    const int tslot = sigma / R, a = sigma - tslot * R;
    const bool dil = NF == kDiluteClasses;
    const int u = dil ? (c & 15) : (c & 7), f = dil ? (c >> 4) : (c >> 3);
    const bool live = dil ? u <= 4 * D : u <= 2 * D;
    const int cls = (dil ? u : 4 * D - 2 * u) * 2 + f;
    uint64_t T[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int s = 64 * g + 32 * h + (int)lane;
      const int k = s < S ? temp_of[((size_t)s * R + a) * K + tslot] : tslot;
      if (live) T[h] = fthr[(size_t)k * kFieldClasses + cls];
    }
    uint64_t mine, always;
    warp_planes(T[0], T[1], mine, always);
    uint64_t* out = ftp + ((size_t)g * slots + sigma) * kPlanes * NF + c;
    out[(size_t)lane * NF] = mine;
    if (lane == 0) out[(size_t)32 * NF] = always;
  }
}

// ---- measurements: per-lane counts by vertical counters and warp bit-transposes ----
//
// Each thread adds the 64-bit words of its sites (bits of the unsatisfied
// forward bonds as a 2-bit number, the spin-down bits, the disagreement bits
// of two replicas) into per-lane counters held as bit-planes (LaneCounter),
// up to kMeasChunk words at a time.  A flush transposes each plane's low and
// high 32x32 halves across the warp, which leaves in thread t the plane bits
// of sample lanes t and 32 + t of all 32 threads, so a popcount weighted by
// the plane gives each lane's count over the warp's sites.  At the end the
// block sums its warps in shared memory and adds one value per lane and
// quantity to the accumulators.  Per site and configuration this gives U
// (E = 2U - D N), B (M = N - 2B) and X (Q = N - 2X).

constexpr int kMeasWarps = kBlock / 32;
constexpr int kMeasMaxQ = 7;  // quantities per block: U and B of two replicas, X, field F

// 32x32 bit transpose across the warp: afterwards thread j holds, in bit t,
// bit j of the word thread t passed in (five butterfly exchanges).
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t M[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const uint32_t sft = 16u >> i;
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, sft);
    x = (lane & sft) ? ((x & ~M[i]) | ((y >> sft) & M[i])) : ((x & M[i]) | ((y << sft) & ~M[i]));
  }
  return x;
}

// Per-lane counts held vertically across a thread's words: plane b has bit
// l set when bit b of lane l's count is set.  add1 adds 0/1 per lane, add2 a
// 2-bit number (s + 2 cy) per lane, both as ripple-carry adders over the
// planes; flush adds the warp's per-lane totals (lanes t and 32 + t in
// thread t) by one transpose per plane and half, and clears the counter.
// A counter of K planes holds up to 2^K - 1, which bounds the words a
// thread may add between flushes (kMeasChunk).
template <int K>
struct LaneCounter {
  uint64_t c[K];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int b = 0; b < K; ++b) c[b] = 0;
  }
  __device__ __forceinline__ void add1(uint64_t x) {
#pragma unroll
    for (int b = 0; b < K; ++b) {
      const uint64_t t = c[b] & x;
      c[b] ^= x;
      x = t;
    }
  }
  __device__ __forceinline__ void add2(uint64_t s, uint64_t cy) {
    const uint64_t t0 = c[0] & s;
    c[0] ^= s;
    uint64_t x = (c[1] & t0) | (c[1] & cy) | (t0 & cy);
    c[1] ^= t0 ^ cy;
#pragma unroll
    for (int b = 2; b < K; ++b) {
      const uint64_t t = c[b] & x;
      c[b] ^= x;
      x = t;
    }
  }
  __device__ __forceinline__ void flush(int shift, long long sign, long long& lo, long long& hi) {
#pragma unroll
    for (int b = 0; b < K; ++b) {
      lo += sign * ((long long)__popc(warp_transpose32((uint32_t)c[b])) << (shift + b));
      hi += sign * ((long long)__popc(warp_transpose32((uint32_t)(c[b] >> 32))) << (shift + b));
      c[b] = 0;
    }
  }
};

// Words a thread adds between flushes: 21 words of up to 3 (a site's
// forward bonds) fit 6 planes, of up to 1 fit 5.
constexpr int kMeasChunk = 21;
constexpr int kPlanesBond = 6, kPlanesBit = 5;

// Split index j -> split indices of the forward neighbours x+1, y+1, z+1.
struct Fwd {
  uint32_t x, y, z;
};

template <bool P2>
__device__ __forceinline__ Fwd split_forward(const Geom& g, uint32_t j) {
  const uint32_t h = (uint32_t)g.h, L = (uint32_t)g.L;
  uint32_t rc, k, y, z;
  if (P2) {
    rc = j >> g.lh;
    k = j & (h - 1u);
    y = (rc >> 1) & (L - 1u);
    z = (rc >> 1) >> g.lL;
  } else {
    rc = j / h;
    k = j - rc * h;
    y = (rc >> 1) % L;
    z = (rc >> 1) / L;
  }
  const uint32_t row = rc >> 1, c = rc & 1u, oc = c ^ 1u;
  const uint32_t x = 2u * k + ((c ^ (y + z)) & 1u);
  Fwd f;
  f.x = (2u * row + oc) * h + (x + 1u == L ? 0u : (x + 1u) >> 1);
  f.y = (2u * ((y + 1u == L ? 0u : y + 1u) + L * z) + oc) * h + k;
  f.z = g.D == 3 ? (2u * (y + L * (z + 1u == L ? 0u : z + 1u)) + oc) * h + k : 0u;
  return f;
}

// Unsatisfied forward bonds of a site as a 2-bit number (sum, carry).
template <int D>
__device__ __forceinline__ void bond_count(uint64_t b, uint64_t nx, uint64_t ny, uint64_t nz, uint64_t Jx,
                                           uint64_t Jy, uint64_t Jz, uint64_t& s1, uint64_t& c1) {
  const uint64_t ex = b ^ nx ^ Jx, ey = b ^ ny ^ Jy;
  if (D == 3) {
    const uint64_t ez = b ^ nz ^ Jz;
    s1 = ex ^ ey ^ ez;
    c1 = (ex & ey) | (ex & ez) | (ey & ez);
  } else {
    s1 = ex ^ ey;
    c1 = ex & ey;
  }
}

// Block reduction of the per-thread lane totals tot[q][2] and one atomic add
// per (lane, quantity) into acc[sample][row_of(q)][field_of(q)].
__device__ __forceinline__ void block_flush(long long (*red)[64], const long long (*tot)[2], int nq, int g, int S,
                                            int64_t* acc, const int* row_off, const int* field, int row_stride) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = 0; q < nq; ++q) {
    red[warp * kMeasMaxQ + q][lane] = tot[q][0];
    red[warp * kMeasMaxQ + q][32 + lane] = tot[q][1];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nq * 64; idx += kBlock) {
    const int q = idx >> 6, l = idx & 63;
    long long v = 0;
    for (int w = 0; w < kMeasWarps; ++w) v += red[w * kMeasMaxQ + q][l];
    const int s = 64 * g + l;
    if (s < S && v != 0)
      atomicAdd((unsigned long long*)&acc[((size_t)s * row_stride + row_off[q]) * kAccStride + field[q]],
                (unsigned long long)v);
  }
}

// One temperature (slot = replica): U and B of every replica and, with two
// replicas, X, in one pass.  Grid (chunks, groups).
template <int D, int R, bool P2>
__global__ void __launch_bounds__(kBlock, 2) k_measure_bits_k1(const uint64_t* __restrict__ spins,
                                                            const uint64_t* __restrict__ J, int64_t* acc, Geom geom,
                                                            int S) {
  __shared__ long long red[kMeasWarps * kMeasMaxQ][64];
  const int g = blockIdx.y;
  const uint32_t N = geom.N;
  const uint64_t* Jg = J + (size_t)g * D * N;
  const uint64_t* sg = spins + (size_t)g * R * N;
  constexpr int NQ = 2 * R + (R == 2 ? 1 : 0);
  long long tot[NQ][2];
#pragma unroll
  for (int q = 0; q < NQ; ++q) tot[q][0] = tot[q][1] = 0;
  LaneCounter<kPlanesBond> cu[R];
  LaneCounter<kPlanesBit> cb[R], cx;
#pragma unroll
  for (int a = 0; a < R; ++a) {
    cu[a].zero();
    cb[a].zero();
  }
  cx.zero();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * kBlock;
  uint32_t base = blockIdx.x * kBlock + (threadIdx.x & ~31u);  // uniform across the warp
  while (base < N) {
    for (int n = 0; n < kMeasChunk && base < N; ++n, base += stride) {
      const uint32_t j = base + lane;
      if (j >= N) continue;
      const Fwd f = split_forward<P2>(geom, j);
      const uint64_t Jx = Jg[j], Jy = Jg[N + j], Jz = D == 3 ? Jg[2u * N + j] : 0ull;
      uint64_t bw[R];
#pragma unroll
      for (int a = 0; a < R; ++a) {
        const uint64_t* sp = sg + (size_t)a * N;
        uint64_t s1, c1;
        bw[a] = sp[j];
        bond_count<D>(bw[a], sp[f.x], sp[f.y], D == 3 ? sp[f.z] : 0ull, Jx, Jy, Jz, s1, c1);
        cu[a].add2(s1, c1);
        cb[a].add1(bw[a]);
      }
      if (R == 2) cx.add1(bw[0] ^ bw[R - 1]);
    }
#pragma unroll
    for (int a = 0; a < R; ++a) {
      cu[a].flush(0, 1, tot[2 * a][0], tot[2 * a][1]);
      cb[a].flush(0, 1, tot[2 * a + 1][0], tot[2 * a + 1][1]);
    }
    if (R == 2) cx.flush(0, 1, tot[NQ - 1][0], tot[NQ - 1][1]);
  }
  int row_off[NQ], field[NQ];
#pragma unroll
  for (int a = 0; a < R; ++a) {
    row_off[2 * a] = row_off[2 * a + 1] = a;
    field[2 * a] = 0;
    field[2 * a + 1] = 1;
  }
  if (R == 2) {
    row_off[NQ - 1] = 0;
    field[NQ - 1] = 6;
  }
  block_flush(red, tot, NQ, g, S, acc, row_off, field, R);
}

// Any number of temperatures: U and B of one slot.  Grid (chunks, groups x
// slots).
template <int D, bool P2, bool EONLY = false>
__global__ void __launch_bounds__(kBlock) k_measure_bits(const uint64_t* __restrict__ spins,
                                                         const uint64_t* __restrict__ J, int64_t* acc, Geom geom,
                                                         int S, int R, int K, int slots) {
  __shared__ long long red[kMeasWarps * kMeasMaxQ][64];
  const int gt = blockIdx.y;  // g * slots + sigma
  const int g = gt / slots, sigma = gt - g * slots;
  const uint32_t N = geom.N;
  const uint64_t* Jg = J + (size_t)g * D * N;
  const uint64_t* sp = spins + ((size_t)g * slots + sigma) * N;
  long long tot[2][2] = {{0, 0}, {0, 0}};
  LaneCounter<kPlanesBond> cu;
  LaneCounter<kPlanesBit> cb;
  cu.zero();
  cb.zero();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * kBlock;
  uint32_t base = blockIdx.x * kBlock + (threadIdx.x & ~31u);  // uniform across the warp
  while (base < N) {
    for (int n = 0; n < kMeasChunk && base < N; ++n, base += stride) {
      const uint32_t j = base + lane;
      if (j >= N) continue;
      const Fwd f = split_forward<P2>(geom, j);
      const uint64_t bw = sp[j];
      uint64_t s1, c1;
      bond_count<D>(bw, sp[f.x], sp[f.y], D == 3 ? sp[f.z] : 0ull, Jg[j], Jg[N + j], D == 3 ? Jg[2u * N + j] : 0ull,
                    s1, c1);
      cu.add2(s1, c1);
      if (!EONLY) cb.add1(bw);
    }
    cu.flush(0, 1, tot[0][0], tot[0][1]);
    if (!EONLY) cb.flush(0, 1, tot[1][0], tot[1][1]);
  }
  const int row_off[2] = {sigma, sigma}, field[2] = {0, 1};
  block_flush(red, tot, EONLY ? 1 : 2, g, S, acc, row_off, field, slots);
}

// Field models (RFIM, DAFF) of one slot, values rather than counts:
// E_J = sum over forward bonds with both ends occupied of (2 e - 1), as
// 2 U - O with U, O the per-site counts of occupied unsatisfied and occupied
// bonds (each a 2-bit sum); M = sum x s = X - 2 sum x b and F = sum sign(h)
// x s = X - 2 sum x (b ^ hb), X = sum x.  acc[0..2] = E_J, M, F.
template <int D, bool P2>
__global__ void __launch_bounds__(kBlock) k_measure_field_bits(const uint64_t* __restrict__ spins,
                                                               const uint64_t* __restrict__ J,
                                                               const uint64_t* __restrict__ hbits,
                                                               const uint64_t* __restrict__ xbits, int64_t* acc,
                                                               Geom geom, int S, int slots) {
  __shared__ long long red[kMeasWarps * kMeasMaxQ][64];
  const int gt = blockIdx.y;  // g * slots + sigma
  const int g = gt / slots, sigma = gt - g * slots;
  const uint32_t N = geom.N;
  const uint64_t* Jg = J + (size_t)g * D * N;
  const uint64_t* sp = spins + ((size_t)g * slots + sigma) * N;
  const uint64_t* Hg = hbits + (size_t)g * N;
  const uint64_t* Xg = xbits + (size_t)g * N;
  long long tot[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  // U: occupied unsatisfied forward bonds, O: occupied forward bonds,
  // X: occupied sites, XB: occupied down spins, XF: occupied against the field
  LaneCounter<kPlanesBond> cuu, coo;
  LaneCounter<kPlanesBit> cxs, cxb, cxf;
  cuu.zero();
  coo.zero();
  cxs.zero();
  cxb.zero();
  cxf.zero();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * kBlock;
  uint32_t base = blockIdx.x * kBlock + (threadIdx.x & ~31u);  // uniform across the warp
  while (base < N) {
    for (int n = 0; n < kMeasChunk && base < N; ++n, base += stride) {
      const uint32_t j = base + lane;
      if (j >= N) continue;
      const Fwd f = split_forward<P2>(geom, j);
      const uint64_t b = sp[j];
      const uint64_t xs = Xg[j];
      const uint64_t ox = xs & Xg[f.x], oy = xs & Xg[f.y], oz = D == 3 ? xs & Xg[f.z] : 0ull;
      const uint64_t ux = ox & (b ^ sp[f.x] ^ Jg[j]), uy = oy & (b ^ sp[f.y] ^ Jg[N + j]);
      const uint64_t uz = D == 3 ? oz & (b ^ sp[f.z] ^ Jg[2u * N + j]) : 0ull;
      cuu.add2(ux ^ uy ^ uz, (ux & uy) | (ux & uz) | (uy & uz));
      coo.add2(ox ^ oy ^ oz, (ox & oy) | (ox & oz) | (oy & oz));
      cxs.add1(xs);
      cxb.add1(xs & b);
      cxf.add1(xs & (b ^ Hg[j]));
    }
    // E_J = 2U - O, M = X - 2 XB, F = X - 2 XF
    cuu.flush(1, 1, tot[0][0], tot[0][1]);
    coo.flush(0, -1, tot[0][0], tot[0][1]);
    long long xl = 0, xh = 0;
    cxs.flush(0, 1, xl, xh);
    tot[1][0] += xl;
    tot[1][1] += xh;
    tot[2][0] += xl;
    tot[2][1] += xh;
    cxb.flush(1, -1, tot[1][0], tot[1][1]);
    cxf.flush(1, -1, tot[2][0], tot[2][1]);
  }
  const int row_off[3] = {sigma, sigma, sigma}, field[3] = {0, 1, 2};
  block_flush(red, tot, 3, g, S, acc, row_off, field, slots);
}

// Overlap at temperature k between replicas 0 and 1 (Sec. 4.1).  After
// parallel-tempering swaps the configuration holding temperature k differs
// per sample, so the word of replica a at temperature k is assembled lane by
// lane: W_a = OR_t (sel[a][t] & spins[t*R + a]), sel[a][t] = lanes whose
// temperature k sits in slot t.  X = count per lane of W_0 ^ W_1, Q = N - 2X,
// stored in acc[s][k*R][6].  Grid (chunks, groups x temperatures).
// With occupations (field models) the value Q = sum x (1 - 2 (w0 ^ w1)) is
// stored instead of the count.
__global__ void __launch_bounds__(kBlock) k_overlap_bits(const uint64_t* __restrict__ spins,
                                                         const int32_t* __restrict__ slot_at,
                                                         const uint64_t* __restrict__ xbits, int64_t* acc,
                                                         uint32_t N, int S, int R, int K, int slots) {
  extern __shared__ uint64_t sel[];  // [2][K]
  __shared__ long long red[kMeasWarps * kMeasMaxQ][64];
  const int gk = blockIdx.y;
  const int g = gk / K, k = gk - g * K;
  for (int t = threadIdx.x; t < 2 * K; t += kBlock) {
    const int a = t / K, ts = t - a * K;
    uint64_t m = 0;
    for (int l = 0; l < 64; ++l) {
      const int s = 64 * g + l;
      const int at = s < S ? slot_at[((size_t)s * R + a) * K + k] : k;
      if (at == ts) m |= 1ull << l;
    }
    sel[t] = m;
  }
  __syncthreads();
  const uint64_t* sg = spins + (size_t)g * slots * N;
  long long tot[1][2] = {{0, 0}};
  LaneCounter<kPlanesBit> cd, cw;  // disagreements (occupied), occupied sites
  cd.zero();
  cw.zero();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * kBlock;
  uint32_t base = blockIdx.x * kBlock + (threadIdx.x & ~31u);  // uniform across the warp
  while (base < N) {
    for (int n = 0; n < kMeasChunk && base < N; ++n, base += stride) {
      const uint32_t j = base + lane;
      if (j >= N) continue;
      uint64_t w0 = 0, w1 = 0;
      for (int t = 0; t < K; ++t) {
        const uint64_t m0 = sel[t], m1 = sel[K + t];
        if (m0) w0 |= m0 & sg[((size_t)t * R + 0) * N + j];
        if (m1) w1 |= m1 & sg[((size_t)t * R + 1) * N + j];
      }
      if (xbits) {
        const uint64_t xw = xbits[(size_t)g * N + j];
        cw.add1(xw);
        cd.add1(xw & (w0 ^ w1));
      } else {
        cd.add1(w0 ^ w1);
      }
    }
    if (xbits) {  // Q = sum x (1 - 2 (w0 ^ w1))
      cw.flush(0, 1, tot[0][0], tot[0][1]);
      cd.flush(1, -1, tot[0][0], tot[0][1]);
    } else {
      cd.flush(0, 1, tot[0][0], tot[0][1]);
    }
  }
  const int row_off[1] = {k * R}, field[1] = {6};
  block_flush(red, tot, 1, g, S, acc, row_off, field, slots);
}

// ---- layout conversions (natural int8 <-> bit-sliced split words) ----

__global__ void k_get_spins_bits(const uint64_t* spins, int8_t* out, Geom geom, int S, int slots) {
  const uint64_t total = (uint64_t)S * slots * geom.N;
  const uint32_t L = (uint32_t)geom.L;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(idx % geom.N);
    const uint64_t rest = idx / geom.N;
    const int sg = (int)(rest % slots), s = (int)(rest / slots);
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    const uint64_t w = spins[((size_t)(s >> 6) * slots + sg) * geom.N + split_index(geom, x, y, z)];
    out[idx] = ((w >> (s & 63)) & 1ull) ? -1 : 1;
  }
}

__global__ void k_set_spins_bits(uint64_t* spins, const int8_t* in, Geom geom, int S, int G, int slots) {
  const uint64_t total = (uint64_t)G * slots * geom.N;
  const uint32_t L = (uint32_t)geom.L;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(idx % geom.N);
    const uint64_t rest = idx / geom.N;
    const int sg = (int)(rest % slots), g = (int)(rest / slots);
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    uint64_t* wp = &spins[((size_t)g * slots + sg) * geom.N + split_index(geom, x, y, z)];
    uint64_t w = *wp;
    for (int l = 0; l < 64; ++l) {
      const int s = 64 * g + l;
      if (s >= S) break;
      const uint64_t bit = in[((size_t)s * slots + sg) * geom.N + i] < 0 ? 1ull : 0ull;
      w = (w & ~(1ull << l)) | (bit << l);
    }
    *wp = w;
  }
}

__global__ void k_get_couplings_bits(const uint64_t* J, int8_t* out, Geom geom, int S) {
  const uint64_t total = (uint64_t)S * geom.D * geom.N;
  const uint32_t L = (uint32_t)geom.L;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(idx % geom.N);
    const uint64_t rest = idx / geom.N;
    const int d = (int)(rest % geom.D), s = (int)(rest / geom.D);
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    const uint64_t w = J[((size_t)(s >> 6) * geom.D + d) * geom.N + split_index(geom, x, y, z)];
    out[idx] = ((w >> (s & 63)) & 1ull) ? -1 : 1;
  }
}

__global__ void k_set_couplings_bits(uint64_t* J, const int8_t* in, Geom geom, int S, int G) {
  const uint64_t total = (uint64_t)G * geom.D * geom.N;
  const uint32_t L = (uint32_t)geom.L;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(idx % geom.N);
    const uint64_t rest = idx / geom.N;
    const int d = (int)(rest % geom.D), g = (int)(rest / geom.D);
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    uint64_t* wp = &J[((size_t)g * geom.D + d) * geom.N + split_index(geom, x, y, z)];
    uint64_t w = *wp;
    for (int l = 0; l < 64; ++l) {
      const int s = 64 * g + l;
      if (s >= S) break;
      const uint64_t bit = in[((size_t)s * geom.D + d) * geom.N + i] < 0 ? 1ull : 0ull;
      w = (w & ~(1ull << l)) | (bit << l);
    }
    *wp = w;
  }
}

inline unsigned grid_for(uint64_t total, unsigned block = 256, unsigned cap = 152u * 16u) {
  uint64_t g = (total + block - 1) / block;
  if (g > cap) g = cap;
  if (g == 0) g = 1;
  return (unsigned)g;
}

template <int D, int ALGO, int RT, bool P2, bool Q>
cudaError_t sweep_launch(Lattice& lat, const BitsParams& p, dim3 grid) {
  const size_t smem = bits_sweep_smem(lat.R, Q);
  if (smem > 48 * 1024) {  // many replicas: opt in to more than 48 KiB of planes and queues
    cudaError_t e = cudaFuncSetAttribute(k_sweep_bits<D, ALGO, RT, P2, Q>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_sweep_bits<D, ALGO, RT, P2, Q><<<grid, kBlock, smem, lat.stream>>>(p);
  return cudaGetLastError();
}

template <int D, int ALGO, bool P2>
cudaError_t sweep_dispatch(Lattice& lat, const BitsParams& p, dim3 grid, size_t) {
  if (lat.R == 1) return sweep_launch<D, ALGO, 1, P2, ALGO == 1>(lat, p, grid);
  if (lat.R == 2) return sweep_launch<D, ALGO, 2, P2, ALGO == 1>(lat, p, grid);
  // the heat bath's queues when they fit beside the planes (up to 97 replicas)
  if (ALGO == 1 && bits_sweep_smem(lat.R, true) <= 227u * 1024u)
    return sweep_launch<D, ALGO, 0, P2, true>(lat, p, grid);
  return sweep_launch<D, ALGO, 0, P2, false>(lat, p, grid);
}

template <int D, int ALGO>
cudaError_t sweep_dispatch2(Lattice& lat, const BitsParams& p, dim3 grid, size_t smem) {
  return lat.geom.lL > 0 ? sweep_dispatch<D, ALGO, true>(lat, p, grid, smem)
                         : sweep_dispatch<D, ALGO, false>(lat, p, grid, smem);
}

template <int D, int ALGO, bool P2>
cudaError_t field_launch(Lattice& lat, const BitsParams& p, dim3 grid, size_t smem) {
  if (lat.dilute) {
    auto kern = k_sweep_bits_dilute<D, ALGO, P2>;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<grid, kBlock, smem, lat.stream>>>(p, lat.hbits, lat.xbits);
    return cudaGetLastError();
  }
  auto kern = k_sweep_bits_field<D, ALGO, P2>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, kBlock, smem, lat.stream>>>(p, lat.hbits);
  return cudaGetLastError();
}

cudaError_t field_dispatch(Lattice& lat, const BitsParams& p, dim3 grid, size_t smem, int algo) {
  const bool p2 = lat.geom.lL > 0;
  if (lat.D == 3) {
    if (algo) return p2 ? field_launch<3, 1, true>(lat, p, grid, smem) : field_launch<3, 1, false>(lat, p, grid, smem);
    return p2 ? field_launch<3, 0, true>(lat, p, grid, smem) : field_launch<3, 0, false>(lat, p, grid, smem);
  }
  if (algo) return p2 ? field_launch<2, 1, true>(lat, p, grid, smem) : field_launch<2, 1, false>(lat, p, grid, smem);
  return p2 ? field_launch<2, 0, true>(lat, p, grid, smem) : field_launch<2, 0, false>(lat, p, grid, smem);
}

// Shapes of the run-time specialised sweep (variants 2..): lockstep plane
// loop or per-warp queues entered after phase_a pairs; registers capped so
// that min_blocks blocks of 256 threads fit on an SM.
struct JitShape {
  int mode, phase_a, min_blocks, group, jreload, ufirst, block;
};
constexpr JitShape kJitShapes[] = {
    {0, 8, 3, 1, 0, 0, 256}, {0, 8, 4, 1, 0, 0, 256}, {1, 4, 3, 1, 0, 0, 256}, {1, 4, 4, 1, 0, 0, 256},
    {1, 3, 3, 1, 0, 0, 256}, {1, 5, 3, 1, 0, 0, 256}, {2, 8, 2, 1, 0, 0, 256}, {2, 8, 3, 1, 0, 0, 256},
    {0, 8, 3, 2, 0, 0, 256}, {1, 4, 3, 2, 0, 0, 256}, {1, 6, 3, 2, 0, 0, 256}, {1, 4, 4, 2, 1, 0, 256},
    {0, 8, 4, 2, 1, 0, 256}, {0, 8, 4, 1, 1, 0, 256}, {1, 4, 4, 1, 1, 0, 256}, {1, 4, 3, 2, 0, 1, 256},
    {0, 8, 4, 2, 0, 1, 256}, {0, 8, 3, 2, 0, 1, 256}, {1, 4, 7, 2, 0, 1, 128}, {1, 4, 6, 2, 0, 1, 128},
    // mode 3: the lane-queue kernel (jit_sweep_lt.cuh), blocks/SM and block size
    {3, 4, 8, 1, 0, 0, 128}, {3, 4, 6, 1, 0, 0, 128}, {3, 4, 4, 1, 0, 0, 256},
    // mode 4: its persistent form; phase_a = least colour words per block / 128
    {4, 4, 8, 1, 0, 0, 128}, {4, 1, 8, 1, 0, 0, 128}, {4, 4, 4, 1, 0, 0, 256}};
constexpr int kNumJitShapes = sizeof(kJitShapes) / sizeof(kJitShapes[0]);
static_assert(kNumJitShapes + 1 == kMaxVariant, "variants 2..kMaxVariant are the shapes");
constexpr int kAutoJitVariant = 24;  // the lane-queue kernel, 4 blocks of 256 per SM

// The specialised kernel shape (>= 2) that variant `variant` selects on this
// lattice with lane-uniform tables (ulut_ok), or 1 for the per-lane kernel.
int jit_variant_of(const Lattice& lat, int variant, bool ulut_ok) {
  int v = variant == 0 ? kAutoJitVariant : variant;
  bool ok = lat.K == 1 && ulut_ok && v >= 2 && v < 2 + kNumJitShapes && (lat.R == 1 || lat.R == 2);
  if (ok && kJitShapes[v - 2].mode == 2 && lat.R != 2) v = 2;  // the interleaved shape needs two replicas
  return ok ? v : 1;
}

// The specialised kernel shape the next sweep uses (>= 2), or 1 for the
// precompiled per-lane kernel.
int jit_variant_for(const Lattice& lat) { return jit_variant_of(lat, lat.variant, lat.ulut_ok); }

}  // namespace

int specialised_variant(const Lattice& lat, int variant) { return jit_variant_of(lat, variant, true); }

bool persistent_variant(const Lattice& lat) {
  const int v = jit_variant_for(lat);
  return v >= 2 && kJitShapes[v - 2].mode == 4 && !lat.field && lat.flags;
}

cudaError_t launch_sweep_persistent(Lattice& lat, int inv, uint64_t t0, uint32_t nsweeps, bool* ran) {
  *ran = false;
  const int v = jit_variant_for(lat);
  if (v < 2 || kJitShapes[v - 2].mode != 4 || nsweeps == 0) return cudaSuccess;
  const JitShape& js = kJitShapes[v - 2];
  prepare_sweep_bits(lat, inv);
  if (!lat.jit) return cudaSuccess;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)lat.jit, js.block, 0) != cudaSuccess) {
    cudaGetLastError();
    return cudaSuccess;
  }
  // blocks per group: as many as are resident at once, each with at least
  // phase_a * 128 colour words and at least one row
  const uint32_t Rg = lat.N / (uint32_t)lat.L, h = (uint32_t)lat.L / 2u;
  const uint32_t resident = (uint32_t)sms * (uint32_t)per_sm;
  uint32_t cpg = resident / (uint32_t)lat.G;
  const uint32_t min_words = 128u * (uint32_t)js.phase_a;
  cpg = std::min(cpg, std::max<uint32_t>(1u, Rg * h / min_words));
  cpg = std::min(cpg, Rg);
  const uint64_t blocks = (uint64_t)cpg * (uint64_t)lat.G;
  if (cpg == 0 || blocks > (uint64_t)resident || blocks > (uint64_t)kMaxPersistBlocks) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(lat.flags, 0, (size_t)blocks * 4, lat.stream);
  if (e != cudaSuccess) return e;
  BitsParams p;
  p.spins = (uint64_t*)lat.spins;
  p.J = (const uint64_t*)lat.J;
  p.tp = lat.tp;
  p.geom = lat.geom;
  p.G = lat.G;
  p.R = lat.R;
  p.K = lat.K;
  p.slots = lat.slots;
  p.colour = 0;
  p.t_lo = (uint32_t)t0;
  p.t_hi = (uint32_t)(t0 >> 32);
  p.words_per_block = 0;
  p.keys = lat.keys;
  p.t_dev = nullptr;
  PersistParams pp;
  pp.flags = lat.flags;
  pp.err = lat.err;
  pp.npass = 2u * nsweeps;
  pp.cpg = cpg;
  pp.t0_lo = (uint32_t)t0;
  pp.t0_hi = (uint32_t)(t0 >> 32);
  pp.timeout_ns = lat.persist_timeout_ns;
  pp.skip_block = lat.persist_absent;
  void* args[] = {(void*)&p, (void*)&pp};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3((unsigned)js.block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = lat.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelExC(&cfg, (const void*)lat.jit, args);
  if (e == cudaErrorCooperativeLaunchTooLarge) {  // not resident at once here: per-pass kernels instead
    cudaGetLastError();
    return cudaSuccess;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  *ran = true;
  return cudaSuccess;
}

cudaKernel_t specialised_sweep_kernel(const Lattice& lat, const UniformLut& u, int algo, int v) {
  if (v < 2 || v >= 2 + kNumJitShapes) return nullptr;
  const JitShape& js = kJitShapes[v - 2];
  return jit_kernel(lat, u, algo, js.mode, js.phase_a, js.min_blocks, js.group, js.jreload, js.ufirst, js.block);
}

void prepare_sweep_bits(Lattice& lat, int inv) {
  const int algo = inv ? 1 : 0;
  if (lat.field) {
    if (lat.flut_ok && lat.variant != 1 && lat.jitf_algo != algo) {
      lat.jitf = jit_field_kernel(lat, algo, lat.dilute && lat.R == 2 ? 2 : 3);  // the diluted pair of replicas needs room
      lat.jitf_algo = algo;
    }
    return;
  }
  const int v = jit_variant_for(lat);
  if (v >= 2 && (lat.jit_algo != algo || lat.jit_variant != v)) {
    lat.jit = specialised_sweep_kernel(lat, lat.ulut, algo, v);
    lat.jit_algo = algo;
    lat.jit_variant = v;
  }
  // the per-lane planes (also the fallback of a failed specialisation),
  // compiled for the geometry unless variant 1 asks for the precompiled kernel
  if ((v < 2 || !lat.jit) && lat.variant != 1 && !lat.jitp_tried[algo]) {
    const int rt = lat.R == 1 || lat.R == 2 ? lat.R : 0;
    const bool q = algo == 1 && bits_sweep_smem(lat.R, true) <= 227u * 1024u;
    lat.jitp[algo] = jit_planes_kernel(lat, algo, rt, q, q ? 3 : 4, (size_t)bits_sweep_smem(lat.R, q));
    lat.jitp_tried[algo] = true;
  }
}

cudaError_t launch_init_bits(Lattice& lat, int jmode) {
  k_init_bits<<<grid_for((uint64_t)lat.G * lat.N), 256, 0, lat.stream>>>((uint64_t*)lat.spins, (uint64_t*)lat.J,
                                                                          lat.geom, lat.G, lat.slots, jmode, lat.keys);
  return cudaGetLastError();
}

cudaError_t launch_init_sites_bits(Lattice& lat, double occupation) {
  const uint64_t T_occ = (uint64_t)std::floor(std::ldexp(occupation, 32));
  k_init_sites_bits<<<grid_for((uint64_t)lat.G * lat.N), 256, 0, lat.stream>>>(
      lat.hbits, lat.xbits, lat.geom, lat.G, lat.disorder == IANUS_DISORDER_RFIM, lat.disorder == IANUS_DISORDER_DAFF,
      T_occ, lat.keys);
  return cudaGetLastError();
}

cudaError_t launch_get_sites_bits(Lattice& lat, int8_t* dev_hs, int8_t* dev_occ) {
  k_get_sites_bits<<<grid_for((uint64_t)lat.S * lat.N), 256, 0, lat.stream>>>(lat.hbits, lat.xbits, dev_hs, dev_occ,
                                                                             lat.geom, lat.S);
  return cudaGetLastError();
}

cudaError_t launch_set_sites_bits(Lattice& lat, const int8_t* dev_hs, const int8_t* dev_occ) {
  k_set_sites_bits<<<grid_for((uint64_t)lat.G * lat.N), 256, 0, lat.stream>>>(lat.hbits, lat.xbits, dev_hs, dev_occ,
                                                                               lat.geom, lat.S, lat.G);
  return cudaGetLastError();
}

cudaError_t launch_load_segment(Lattice& lat, int group, uint32_t lane0, uint32_t n, uint32_t jgroup,
                                PhiloxKeys job_keys) {
  const uint64_t mask = (n >= 64u ? ~0ull : ((1ull << n) - 1ull)) << lane0;
  k_load_segment<<<grid_for(lat.N), 256, 0, lat.stream>>>((uint64_t*)lat.spins, (uint64_t*)lat.J, lat.geom, group,
                                                          lane0, mask, jgroup, job_keys);
  return cudaGetLastError();
}

cudaError_t launch_advance_segments(Lattice& lat) {
  k_advance_segments<<<grid_for((uint64_t)lat.G * kMaxSegs, 128), 128, 0, lat.stream>>>(lat.segs, lat.nseg, lat.G);
  return cudaGetLastError();
}

cudaError_t launch_sweep_fused(Lattice& lat, int colour) {
  BitsParams p;
  p.spins = (uint64_t*)lat.spins;
  p.J = (const uint64_t*)lat.J;
  p.tp = lat.tp;
  p.geom = lat.geom;
  p.G = lat.G;
  p.R = 1;
  p.K = 1;
  p.slots = 1;
  p.colour = colour;
  p.t_lo = p.t_hi = 0;
  p.keys = lat.keys;
  p.t_dev = nullptr;
  const uint32_t half = lat.geom.half;
  uint32_t target_blocks = (152u * 8u + (uint32_t)lat.G - 1) / (uint32_t)lat.G;
  uint32_t wpb = (half + target_blocks - 1) / target_blocks;
  wpb = ((wpb + kBlock - 1) / kBlock) * kBlock;
  if (wpb < (uint32_t)kBlock) wpb = kBlock;
  p.words_per_block = wpb;
  dim3 grid((half + wpb - 1) / wpb, (unsigned)lat.G);
  const bool p2 = lat.geom.lL > 0;
  if (lat.D == 3) {
    if (p2)
      k_sweep_fused<3, true><<<grid, kBlock, 0, lat.stream>>>(p, lat.segs, lat.nseg);
    else
      k_sweep_fused<3, false><<<grid, kBlock, 0, lat.stream>>>(p, lat.segs, lat.nseg);
  } else {
    if (p2)
      k_sweep_fused<2, true><<<grid, kBlock, 0, lat.stream>>>(p, lat.segs, lat.nseg);
    else
      k_sweep_fused<2, false><<<grid, kBlock, 0, lat.stream>>>(p, lat.segs, lat.nseg);
  }
  return cudaGetLastError();
}

cudaError_t launch_build_field_planes(Lattice& lat) {
  k_build_field_planes<<<grid_for((uint64_t)lat.G * lat.slots * lat.fpc * 32, 256), 256, 0, lat.stream>>>(
      lat.ftp, lat.fthr, lat.temp_of, lat.D, lat.G, lat.S, lat.R, lat.K, lat.slots, lat.fpc);
  return cudaGetLastError();
}

cudaError_t launch_build_planes(Lattice& lat) {
  k_build_planes<<<grid_for((uint64_t)lat.G * lat.slots * kMaxClasses * 32, 256), 256, 0, lat.stream>>>(
      lat.tp, lat.thr, lat.temp_of, lat.G, lat.S, lat.R, lat.K, lat.slots);
  return cudaGetLastError();
}

size_t sweep_bits_smem(int R) { return bits_sweep_smem(R, false); }

// Launches a sweep kernel with programmatic stream serialisation: its blocks
// may become resident while the previous kernel on the stream drains, and its
// entry (dependent_launch_entry) holds them until that kernel has completed.
// Inside a stream capture this becomes a programmatic edge of the graph.  A
// refused launch returns its error and leaves no pending error behind.
cudaError_t launch_dependent(const void* k, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelExC(&cfg, k, args);
  if (e != cudaSuccess) cudaGetLastError();
  return e;
}

cudaError_t launch_sweep_bits(Lattice& lat, int colour, uint64_t t, int inv) {
  BitsParams p;
  p.spins = (uint64_t*)lat.spins;
  p.J = (const uint64_t*)lat.J;
  p.tp = lat.tp;
  p.geom = lat.geom;
  p.G = lat.G;
  p.R = lat.R;
  p.K = lat.K;
  p.slots = lat.slots;
  p.colour = colour;
  p.t_lo = (uint32_t)(t & 0xffffffffu);
  p.t_hi = (uint32_t)(t >> 32);
  p.keys = lat.keys;
  p.t_dev = lat.capturing ? lat.t_dev : nullptr;
  // blocks per (group, temperature slot): enough to fill the GPU ~4 deep
  const uint32_t half = lat.geom.half;
  const uint32_t gts = (uint32_t)(lat.G * lat.K);
  uint32_t target_blocks = (152u * 8u + gts - 1) / gts;
  uint32_t wpb;
  if (lat.block_words) {  // explicit shape: whole warps
    wpb = (lat.block_words + 31u) / 32u * 32u;
  } else {
    wpb = (half + target_blocks - 1) / target_blocks;
    wpb = ((wpb + kBlock - 1) / kBlock) * kBlock;
    if (wpb < (uint32_t)kBlock) wpb = kBlock;
  }
  p.words_per_block = wpb;
  dim3 grid((half + wpb - 1) / wpb, gts);
  const size_t smem = (size_t)lat.R * kPlanes * kMaxClasses * sizeof(uint64_t);
  const int algo = inv ? 1 : 0;
  if (lat.field) {
    // one temperature: the field kernel specialised at run time for the
    // lattice's tables (variants 0 (large lattices) and 2..); else per-lane planes
    const uint64_t words = (uint64_t)lat.G * lat.slots * lat.N;
    const bool want_jit = lat.flut_ok && lat.variant != 1 && (lat.variant != 0 || words >= (1ull << 20));
    if (want_jit) {
      prepare_sweep_bits(lat, inv);
      if (lat.jitf) {
        const uint64_t* hb = lat.hbits;
        const uint64_t* xb = lat.xbits;
        const uint8_t* lut = (const uint8_t*)(lat.fthr + (size_t)lat.K * kFieldClasses);
        void* args[] = {(void*)&p, (void*)&hb, (void*)&xb, (void*)&lut};
        return launch_dependent((const void*)lat.jitf, grid, dim3(kBlock), args, 0, lat.stream);
      }
    }
    p.tp = lat.ftp;
    const size_t fsmem = (size_t)lat.R * kPlanes * lat.fpc * sizeof(uint64_t);
    return field_dispatch(lat, p, grid, fsmem, algo);
  }
  // Lane-uniform thresholds (one temperature): the kernel specialised for
  // them at run time.  Variants (ianus_set_variant): 0 = automatic (the
  // lane-queue shape with one temperature and one or two replicas, else the
  // per-lane planes; small lattices take the resident sweep before they get
  // here), 1 = per-lane planes, 2.. = a specialised kernel shape from
  // kJitShapes.  A compile costs a fraction of a second and is cached.
  const int v = jit_variant_for(lat);
  if (v >= 2) {
    const JitShape& js = kJitShapes[v - 2];
    prepare_sweep_bits(lat, inv);
    // mode 4 (persistent) passes that run one at a time use its per-pass form
    const cudaKernel_t k3 = js.mode == 4 ? jit_lt_kernel(lat, lat.ulut, algo, js.min_blocks, js.block) : lat.jit;
    if (k3 && (js.mode == 3 || js.mode == 4)) {
      // one wave: about min_blocks blocks per SM in all, whole warps of words
      uint32_t w3;
      if (lat.block_words) {
        w3 = (lat.block_words + 31u) / 32u * 32u;
      } else {
        const uint32_t per_group = std::max<uint32_t>(1u, 152u * (uint32_t)js.min_blocks / (uint32_t)lat.G);
        w3 = (half + per_group - 1u) / per_group;
        w3 = std::max<uint32_t>(32u, (w3 + 31u) / 32u * 32u);
      }
      p.words_per_block = w3;
      void* args[] = {(void*)&p};
      return launch_dependent((const void*)k3, dim3((half + w3 - 1u) / w3, (unsigned)lat.G), dim3(js.block), args, 0,
                              lat.stream);
    }
    if (lat.jit) {
      const uint8_t* lut_t = (const uint8_t*)(lat.thr + (size_t)lat.K * kMaxClasses);
      void* args[] = {(void*)&p, (void*)&lut_t};
      return launch_dependent((const void*)lat.jit, grid, dim3(js.block), args,
                              js.mode == 1 ? kJitSmemBytes / 256 * js.block : 0, lat.stream);
    }
  }
  // Per-lane planes: the kernel compiled for the lattice's geometry, else
  // (variant 1, or no run-time compiler) the precompiled one.
  if (lat.variant != 1) {
    prepare_sweep_bits(lat, inv);
    if (lat.jitp[algo]) {
      const bool q = algo == 1 && bits_sweep_smem(lat.R, true) <= 227u * 1024u;
      void* args[] = {(void*)&p};
      return launch_dependent((const void*)lat.jitp[algo], grid, dim3(kBlock), args,
                              (size_t)bits_sweep_smem(lat.R, q), lat.stream);
    }
  }
  if (lat.D == 3)
    return algo ? sweep_dispatch2<3, 1>(lat, p, grid, smem) : sweep_dispatch2<3, 0>(lat, p, grid, smem);
  return algo ? sweep_dispatch2<2, 1>(lat, p, grid, smem) : sweep_dispatch2<2, 0>(lat, p, grid, smem);
}

// Blocks along the lattice for a measurement kernel with `ys` blocks across:
// about two blocks per SM in all, each warp taking 32 words at a time, and
// enough that a thread adds at most kMeasChunk words (one counter flush).
inline unsigned meas_blocks(uint32_t N, unsigned ys) {
  unsigned want = (152u * 2u + ys - 1u) / ys;
  const unsigned one_flush = (N + kBlock * kMeasChunk - 1) / (kBlock * kMeasChunk);
  if (want < one_flush) want = one_flush;
  const unsigned most = (N + kBlock - 1) / kBlock;
  return want < 1u ? 1u : (want > most ? most : want);
}

template <int D, bool P2>
cudaError_t measure_dispatch(Lattice& lat, int want_q, bool energy_only) {
  const uint64_t* sp = (const uint64_t*)lat.spins;
  const uint64_t* J = (const uint64_t*)lat.J;
  if (energy_only && !lat.field) {  // U of every configuration, for the PT swap
    dim3 grid(meas_blocks(lat.N, (unsigned)(lat.G * lat.slots)), (unsigned)(lat.G * lat.slots));
    k_measure_bits<D, P2, true><<<grid, kBlock, 0, lat.stream>>>(sp, J, lat.acc, lat.geom, lat.S, lat.R, lat.K,
                                                                 lat.slots);
    return cudaGetLastError();
  }
  if (lat.K == 1 && (lat.R == 1 || lat.R == 2) && !lat.field) {
    // one pass for E, M and (R == 2) Q
    dim3 grid(meas_blocks(lat.N, (unsigned)lat.G), (unsigned)lat.G);
    if (lat.R == 2)
      k_measure_bits_k1<D, 2, P2><<<grid, kBlock, 0, lat.stream>>>(sp, J, lat.acc, lat.geom, lat.S);
    else
      k_measure_bits_k1<D, 1, P2><<<grid, kBlock, 0, lat.stream>>>(sp, J, lat.acc, lat.geom, lat.S);
    return cudaGetLastError();
  }
  dim3 grid(meas_blocks(lat.N, (unsigned)(lat.G * lat.slots)), (unsigned)(lat.G * lat.slots));
  if (lat.field)
    k_measure_field_bits<D, P2><<<grid, kBlock, 0, lat.stream>>>(sp, J, lat.hbits, lat.xbits, lat.acc, lat.geom,
                                                                 lat.S, lat.slots);
  else
    k_measure_bits<D, P2><<<grid, kBlock, 0, lat.stream>>>(sp, J, lat.acc, lat.geom, lat.S, lat.R, lat.K, lat.slots);
  if (want_q && lat.R >= 2) {
    dim3 gq(meas_blocks(lat.N, (unsigned)(lat.G * lat.K)), (unsigned)(lat.G * lat.K));
    k_overlap_bits<<<gq, kBlock, 2 * lat.K * sizeof(uint64_t), lat.stream>>>(
        sp, lat.slot_at, lat.field ? lat.xbits : nullptr, lat.acc, lat.N, lat.S, lat.R, lat.K, lat.slots);
  }
  return cudaGetLastError();
}

cudaError_t launch_measure_bits(Lattice& lat, int want_q, bool energy_only) {
  cudaError_t e = cudaMemsetAsync(lat.acc, 0, (size_t)lat.S * lat.slots * kAccStride * sizeof(int64_t), lat.stream);
  if (e != cudaSuccess) return e;
  const bool p2 = lat.geom.lL > 0;
  if (lat.D == 3)
    return p2 ? measure_dispatch<3, true>(lat, want_q, energy_only)
              : measure_dispatch<3, false>(lat, want_q, energy_only);
  return p2 ? measure_dispatch<2, true>(lat, want_q, energy_only)
            : measure_dispatch<2, false>(lat, want_q, energy_only);
}

cudaError_t launch_get_spins_bits(Lattice& lat, int8_t* dev_out) {
  k_get_spins_bits<<<grid_for((uint64_t)lat.S * lat.slots * lat.N), 256, 0, lat.stream>>>(
      (const uint64_t*)lat.spins, dev_out, lat.geom, lat.S, lat.slots);
  return cudaGetLastError();
}

cudaError_t launch_set_spins_bits(Lattice& lat, const int8_t* dev_in) {
  k_set_spins_bits<<<grid_for((uint64_t)lat.G * lat.slots * lat.N), 256, 0, lat.stream>>>(
      (uint64_t*)lat.spins, dev_in, lat.geom, lat.S, lat.G, lat.slots);
  return cudaGetLastError();
}

cudaError_t launch_get_couplings_bits(Lattice& lat, int8_t* dev_out) {
  k_get_couplings_bits<<<grid_for((uint64_t)lat.S * lat.D * lat.N), 256, 0, lat.stream>>>(
      (const uint64_t*)lat.J, dev_out, lat.geom, lat.S);
  return cudaGetLastError();
}

cudaError_t launch_set_couplings_bits(Lattice& lat, const int8_t* dev_in) {
  k_set_couplings_bits<<<grid_for((uint64_t)lat.G * lat.D * lat.N), 256, 0, lat.stream>>>(
      (uint64_t*)lat.J, dev_in, lat.geom, lat.S, lat.G);
  return cudaGetLastError();
}

}  // namespace ianus
