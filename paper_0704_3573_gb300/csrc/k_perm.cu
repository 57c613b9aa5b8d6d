// k_perm.cu -- the glassy Potts model of Eq. (3),
// H = -sum_<ij> delta(s_i, pi_ij(s_j)), with quenched permutation couplings
// pi_ij of (0,1,2,3), heat bath, in 2, 3 or 4 dimensions (Sec. 4.2 runs it in
// 3D and 4D).
//
// Storage follows IANUS_LAYOUT_U8X4: a 32-bit word holds one site of 4
// samples (byte b = sample 4q+b, state 0..3); a coupling word holds the 8-bit
// permutation codes pi(0) | pi(1) << 2 | pi(2) << 4 | pi(3) << 6 of the 4
// samples (the paper's 8-bit Potts couplings, Sec. 3.2).  Sites are in the
// checkerboard-split order of Sec. 3.1 generalised to D dimensions: word
// (2 row + c) h + x / 2, where row = i / L collects the coordinates after x
// and c is the colour, so every neighbour of a colour-c word is a colour-(1-c)
// word with the same x / 2 (or x / 2 +- 1 along x).
//
// Update of one sample: each of the 2D bonds is satisfied by exactly one
// state k of s_i, k = pi(s_j) for a forward bond (i, j = i + e_d) and
// k = pi^-1(s_j) for a backward bond (j = i - e_d, i); the counts n_k are
// packed in nibbles and (n0, n1, n2) index a compact table of cumulative
// heat-bath thresholds (n3 = 2D - n0 - n1 - n2), read through the L1 cache.
#include <algorithm>

#include "lattice.h"

namespace ianus {

namespace {

constexpr int kBlock = 256;
constexpr uint32_t kIdentityCode = 0xE4u;  // (0, 1, 2, 3)

template <int D>
struct PermNbr {
  uint32_t self, site;
  uint32_t fw[D], bw[D];  // split indices of i + e_d and i - e_d
};

// Colour-c word w -> its split index, natural index and neighbours.
template <int D>
__device__ __forceinline__ PermNbr<D> perm_neighbours(const Geom& g, int c, uint32_t w) {
  const uint32_t h = (uint32_t)g.h, L = (uint32_t)g.L;
  const uint32_t row = w / h, k = w - row * h;
  uint32_t co[D > 1 ? D : 2];
  uint32_t r = row, psum = 0;
#pragma unroll
  for (int d = 1; d < D; ++d) {
    co[d] = r % L;
    r /= L;
    psum += co[d];
  }
  const uint32_t xpar = (uint32_t)(c ^ (int)psum) & 1u;
  const uint32_t oc = 1u - (uint32_t)c;
  PermNbr<D> n;
  n.self = (2u * row + (uint32_t)c) * h + k;
  n.site = 2u * k + xpar + L * row;
  const uint32_t base_o = (2u * row + oc) * h;
  n.fw[0] = base_o + (xpar ? (k + 1u == h ? 0u : k + 1u) : k);  // (x + 1) / 2 mod h
  n.bw[0] = base_o + (xpar ? k : (k == 0u ? h - 1u : k - 1u));  // (x - 1) / 2 mod h
  uint32_t stride = 1;
#pragma unroll
  for (int d = 1; d < D; ++d) {
    const uint32_t rp = co[d] + 1u == L ? row - (L - 1u) * stride : row + stride;
    const uint32_t rm = co[d] == 0u ? row + (L - 1u) * stride : row - stride;
    n.fw[d] = (2u * rp + oc) * h + k;
    n.bw[d] = (2u * rm + oc) * h + k;
    stride *= L;
  }
  return n;
}

// Natural index -> split index, any D.
__device__ __forceinline__ uint32_t perm_split(const Geom& g, uint32_t i) {
  const uint32_t L = (uint32_t)g.L;
  const uint32_t x = i % L, row = i / L;
  uint32_t r = row, psum = x;
  for (int d = 1; d < g.D; ++d) {
    psum += r % L;
    r /= L;
  }
  return (2u * row + (psum & 1u)) * (uint32_t)g.h + x / 2u;
}

// Code of permutation number p (lexicographic): digit p / 6 picks the first
// value among the four, then p / 2 mod 3 among the remaining three, etc.
__device__ __forceinline__ uint32_t perm_code_of(uint32_t p) {
  uint32_t pool = kIdentityCode;  // remaining values, increasing, 2 bits each
  uint32_t code = 0;
  const uint32_t wgt[3] = {6u, 2u, 1u};
#pragma unroll
  for (int pos = 0; pos < 3; ++pos) {
    const uint32_t pick = p / wgt[pos];
    p -= pick * wgt[pos];
    code |= ((pool >> (2u * pick)) & 3u) << (2 * pos);
    const uint32_t low = pool & ((1u << (2u * pick)) - 1u);
    pool = low | ((pool >> (2u * pick + 2u)) << (2u * pick));
  }
  return code | ((pool & 3u) << 6);
}

// pi^-1 as a code: field pi(v) of the result holds v.
__device__ __forceinline__ uint32_t inverse_code(uint32_t code) {
  uint32_t inv = 0;
#pragma unroll
  for (uint32_t v = 0; v < 4u; ++v) inv |= v << (2u * ((code >> (2u * v)) & 3u));
  return inv;
}

struct PermParams {
  uint32_t* spins;         // [slots][Q4][N]
  const uint32_t* J;       // [Q4][D][N] permutation codes
  const uint4* tab;        // [K][(2D+1)^3] {T0, T1, T2, always flags}
  const int32_t* temp_of;  // [S][R][K]
  Geom geom;
  int S, R, K, Q4, slots;
  int colour;
  uint32_t t_lo, t_hi;
  uint32_t words_per_block;
  PhiloxKeys keys;
  const uint64_t* t_dev;  // non-null in captured graphs
};

template <int D>
__global__ void __launch_bounds__(kBlock) k_sweep_perm(const PermParams p) {
  constexpr uint32_t B = 2 * D + 1;
  constexpr uint32_t NT = B * B * B;
  __shared__ uint8_t inv_s[256];
  for (uint32_t c = threadIdx.x; c < 256u; c += kBlock) inv_s[c] = (uint8_t)inverse_code(c);
  dependent_launch_entry();  // the table above reads no memory
  const int sq = blockIdx.y;  // sigma * Q4 + q
  const int sigma = sq / p.Q4, q = sq - sigma * p.Q4;
  const int tslot = sigma / p.R, a = sigma - tslot * p.R;
  const Geom geom = p.geom;
  const uint32_t N = geom.N;
  const uint32_t* Jq = p.J + (size_t)q * D * N;
  uint32_t* sp = p.spins + ((size_t)sigma * p.Q4 + q) * N;
  const uint4* tab[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int s = 4 * q + b;
    const int k = s < p.S ? p.temp_of[((size_t)s * p.R + a) * p.K + tslot] : tslot;
    tab[b] = p.tab + (size_t)k * NT;
  }
  const uint32_t c2 = (TAG_POTTS << 28) | ((uint32_t)sigma << 16) | (uint32_t)q;
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  __syncthreads();
  const uint32_t w_begin = blockIdx.x * p.words_per_block;
  const uint32_t w_end = min(w_begin + p.words_per_block, geom.half);
  for (uint32_t w = w_begin + threadIdx.x; w < w_end; w += kBlock) {
    const PermNbr<D> n = perm_neighbours<D>(geom, p.colour, w);
    uint32_t sf[D], sb[D], jf[D], jb[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      sf[d] = sp[n.fw[d]];
      sb[d] = sp[n.bw[d]];
      jf[d] = __ldg(Jq + (size_t)d * N + n.self);
      jb[d] = __ldg(Jq + (size_t)d * N + n.bw[d]);
    }
    const uint4 x = philox10(n.site, tk.lo, c2, tk.hi, p.keys);
    const uint32_t rr[4] = {x.x, x.y, x.z, x.w};
    uint32_t out = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      uint32_t npk = 0;  // nibble k = n_k
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const uint32_t s_f = (sf[d] >> (8 * b)) & 3u;
        const uint32_t tf = (jf[d] >> (8 * b + 2 * s_f)) & 3u;  // pi(s_j)
        const uint32_t s_b = (sb[d] >> (8 * b)) & 3u;
        const uint32_t tb = ((uint32_t)inv_s[(jb[d] >> (8 * b)) & 0xFFu] >> (2 * s_b)) & 3u;  // pi^-1(s_j)
        npk += (1u << (4 * tf)) + (1u << (4 * tb));
      }
      const uint32_t n0 = npk & 15u, n1 = (npk >> 4) & 15u, n2 = (npk >> 8) & 15u;
      const uint4 T = __ldg(tab[b] + n0 + B * (n1 + B * n2));
      const uint32_t r = rr[b];
      const uint32_t ge0 = !((T.w & 1u) || r < T.x);
      const uint32_t ge1 = !((T.w & 2u) || r < T.y);
      const uint32_t ge2 = !((T.w & 4u) || r < T.z);
      out |= (ge0 + ge1 + ge2) << (8 * b);
    }
    sp[n.self] = out;
  }
}

// Couplings from the PERM stream (jmode 0) or identity permutations (jmode
// 1); initial states from the PINIT stream, as for the J-weighted Potts glass.
__global__ void k_init_perm(uint32_t* spins, uint32_t* J, Geom geom, int Q4, int slots, int jmode, PhiloxKeys keys) {
  const uint64_t total = (uint64_t)Q4 * geom.N;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t q = (uint32_t)(idx / geom.N), i = (uint32_t)(idx - (uint64_t)q * geom.N);
    const uint32_t j = perm_split(geom, i);
    for (int d = 0; d < geom.D; ++d) {
      uint32_t w = 0;
      if (jmode == 1) {
        w = kIdentityCode * 0x01010101u;
      } else {
        const uint4 r = philox10(i, (uint32_t)d, (TAG_PERM << 28) | q, 0u, keys);
        const uint32_t xs[4] = {r.x, r.y, r.z, r.w};
        for (int b = 0; b < 4; ++b) w |= perm_code_of((uint32_t)(((uint64_t)xs[b] * 24u) >> 32)) << (8 * b);
      }
      J[((size_t)q * geom.D + d) * geom.N + j] = w;
    }
    for (int sg = 0; sg < slots; ++sg) {
      const uint4 r = philox10(i, 0u, (TAG_PINIT << 28) | ((uint32_t)sg << 16) | q, 0u, keys);
      spins[((size_t)sg * Q4 + q) * geom.N + j] =
          (r.x >> 30) | ((r.y >> 30) << 8) | ((r.z >> 30) << 16) | ((r.w >> 30) << 24);
    }
  }
}

// Per (slot, quad) block: E = -sum over forward bonds of delta(s_i, pi(s_j))
// and the state counts of the 4 samples (Sec. 4.1 observables).
constexpr int kPermMeasIters = 32;

template <int D>
__global__ void __launch_bounds__(kBlock) k_measure_perm(const uint32_t* __restrict__ spins,
                                                         const uint32_t* __restrict__ J, int64_t* acc, Geom geom,
                                                         int S, int Q4, int slots) {
  const int sq = blockIdx.y;
  const int sigma = sq / Q4, q = sq - sigma * Q4;
  const uint32_t N = geom.N, h = (uint32_t)geom.h;
  const uint32_t* Jq = J + (size_t)q * D * N;
  const uint32_t* sp = spins + ((size_t)sigma * Q4 + q) * N;
  const uint32_t base = blockIdx.x * (uint32_t)(kBlock * kPermMeasIters);
  long long v[4][5];  // per sample: E, n0..n3
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int f = 0; f < 5; ++f) v[b][f] = 0;
  for (int it = 0; it < kPermMeasIters; ++it) {
    const uint32_t j = base + (uint32_t)it * kBlock + threadIdx.x;
    if (j >= N) continue;
    const uint32_t rc = j / h, k = j - rc * h;
    const PermNbr<D> n = perm_neighbours<D>(geom, (int)(rc & 1u), (rc >> 1) * h + k);
    const uint32_t si = sp[j];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const uint32_t sj = sp[n.fw[d]];
      const uint32_t code = Jq[(size_t)d * N + j];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const uint32_t t = (code >> (8 * b + 2 * ((sj >> (8 * b)) & 3u))) & 3u;
        if (t == ((si >> (8 * b)) & 3u)) v[b][0] -= 1;
      }
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) v[b][1 + ((si >> (8 * b)) & 3u)] += 1;
  }
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int f = 0; f < 5; ++f)
      for (int off = 16; off > 0; off >>= 1) v[b][f] += __shfl_down_sync(0xffffffffu, v[b][f], off);
  if ((threadIdx.x & 31) == 0) {
    for (int b = 0; b < 4; ++b) {
      const int s = 4 * q + b;
      if (s >= S) continue;
      int64_t* ac = acc + ((size_t)s * slots + sigma) * kAccStride;
      atomicAdd((unsigned long long*)&ac[0], (unsigned long long)v[b][0]);
      for (int f = 0; f < 4; ++f) atomicAdd((unsigned long long*)&ac[2 + f], (unsigned long long)v[b][1 + f]);
    }
  }
}

// natural order [S][per][N] <-> packed split words, any D.  Spins: words
// [per = slots][Q4][N]; couplings (by_quad): words [Q4][per = D][N].
__device__ __forceinline__ size_t perm_word_row(bool by_quad, int m, int q, int Q4, int per, uint32_t N) {
  return by_quad ? ((size_t)q * per + m) * N : ((size_t)m * Q4 + q) * N;
}

__global__ void k_get_bytes_perm(const uint32_t* words, int8_t* out, Geom geom, int S, int Q4, int per,
                                 bool by_quad) {
  const uint64_t total = (uint64_t)S * per * geom.N;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(idx % geom.N);
    const uint64_t rest = idx / geom.N;
    const int m = (int)(rest % per), s = (int)(rest / per);
    const uint32_t w = words[perm_word_row(by_quad, m, s >> 2, Q4, per, geom.N) + perm_split(geom, i)];
    out[idx] = (int8_t)(uint8_t)(w >> (8 * (s & 3)));
  }
}

__global__ void k_set_bytes_perm(uint32_t* words, const int8_t* in, Geom geom, int S, int Q4, int per, bool by_quad,
                                 uint32_t mask) {
  const uint64_t total = (uint64_t)Q4 * per * geom.N;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(idx % geom.N);
    const uint64_t rest = idx / geom.N;
    const int m = (int)(rest % per), q = (int)(rest / per);
    uint32_t* wp = &words[perm_word_row(by_quad, m, q, Q4, per, geom.N) + perm_split(geom, i)];
    uint32_t w = *wp;
    for (int b = 0; b < 4; ++b) {
      const int s = 4 * q + b;
      if (s >= S) break;
      const uint32_t v = (uint32_t)(uint8_t)in[((size_t)s * per + m) * geom.N + i] & mask;
      w = (w & ~(0xFFu << (8 * b))) | (v << (8 * b));
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

}  // namespace

cudaError_t launch_init_perm(Lattice& lat, int jmode) {
  k_init_perm<<<grid_for((uint64_t)lat.Q4 * lat.N), 256, 0, lat.stream>>>(
      (uint32_t*)lat.spins, (uint32_t*)lat.J, lat.geom, lat.Q4, lat.slots, jmode, lat.keys);
  return cudaGetLastError();
}

cudaError_t launch_sweep_perm(Lattice& lat, int colour, uint64_t t) {
  PermParams p;
  p.spins = (uint32_t*)lat.spins;
  p.J = (const uint32_t*)lat.J;
  p.tab = lat.ptab;
  p.temp_of = lat.temp_of;
  p.geom = lat.geom;
  p.S = lat.S;
  p.R = lat.R;
  p.K = lat.K;
  p.Q4 = lat.Q4;
  p.slots = lat.slots;
  p.colour = colour;
  p.t_lo = (uint32_t)(t & 0xffffffffu);
  p.t_hi = (uint32_t)(t >> 32);
  p.keys = lat.keys;
  p.t_dev = lat.capturing ? lat.t_dev : nullptr;
  const uint32_t half = lat.geom.half;
  const uint32_t ys = (uint32_t)(lat.slots * lat.Q4);
  uint32_t target_blocks = (152u * 8u + ys - 1) / ys;
  uint32_t wpb = (half + target_blocks - 1) / target_blocks;
  wpb = ((wpb + kBlock - 1) / kBlock) * kBlock;
  if (wpb < (uint32_t)kBlock) wpb = kBlock;
  p.words_per_block = wpb;
  dim3 grid((half + wpb - 1) / wpb, ys);
  void* args[] = {(void*)&p};
  const void* k = lat.D == 4   ? (const void*)k_sweep_perm<4>
                  : lat.D == 3 ? (const void*)k_sweep_perm<3>
                               : (const void*)k_sweep_perm<2>;
  return launch_dependent(k, grid, dim3(kBlock), args, 0, lat.stream);
}

cudaError_t launch_measure_perm(Lattice& lat, int want_q) {
  cudaError_t e = cudaMemsetAsync(lat.acc, 0, (size_t)lat.S * lat.slots * kAccStride * sizeof(int64_t), lat.stream);
  if (e != cudaSuccess) return e;
  const uint32_t per_block = kBlock * kPermMeasIters;
  dim3 grid((lat.N + per_block - 1) / per_block, (unsigned)(lat.slots * lat.Q4));
  const uint32_t* sp = (const uint32_t*)lat.spins;
  const uint32_t* J = (const uint32_t*)lat.J;
  if (lat.D == 4)
    k_measure_perm<4><<<grid, kBlock, 0, lat.stream>>>(sp, J, lat.acc, lat.geom, lat.S, lat.Q4, lat.slots);
  else if (lat.D == 3)
    k_measure_perm<3><<<grid, kBlock, 0, lat.stream>>>(sp, J, lat.acc, lat.geom, lat.S, lat.Q4, lat.slots);
  else
    k_measure_perm<2><<<grid, kBlock, 0, lat.stream>>>(sp, J, lat.acc, lat.geom, lat.S, lat.Q4, lat.slots);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return want_q && lat.R >= 2 ? launch_overlap_potts(lat) : cudaSuccess;
}

cudaError_t launch_get_spins_perm(Lattice& lat, int8_t* dev_out) {
  k_get_bytes_perm<<<grid_for((uint64_t)lat.S * lat.slots * lat.N), 256, 0, lat.stream>>>(
      (const uint32_t*)lat.spins, dev_out, lat.geom, lat.S, lat.Q4, lat.slots, false);
  return cudaGetLastError();
}

cudaError_t launch_set_spins_perm(Lattice& lat, const int8_t* dev_in) {
  k_set_bytes_perm<<<grid_for((uint64_t)lat.slots * lat.Q4 * lat.N), 256, 0, lat.stream>>>(
      (uint32_t*)lat.spins, dev_in, lat.geom, lat.S, lat.Q4, lat.slots, false, 3u);
  return cudaGetLastError();
}

cudaError_t launch_get_couplings_perm(Lattice& lat, int8_t* dev_out) {
  k_get_bytes_perm<<<grid_for((uint64_t)lat.S * lat.D * lat.N), 256, 0, lat.stream>>>(
      (const uint32_t*)lat.J, dev_out, lat.geom, lat.S, lat.Q4, lat.D, true);
  return cudaGetLastError();
}

cudaError_t launch_set_couplings_perm(Lattice& lat, const int8_t* dev_in) {
  k_set_bytes_perm<<<grid_for((uint64_t)lat.Q4 * lat.D * lat.N), 256, 0, lat.stream>>>(
      (uint32_t*)lat.J, dev_in, lat.geom, lat.S, lat.Q4, lat.D, true, 0xFFu);
  return cudaGetLastError();
}

}  // namespace ianus
