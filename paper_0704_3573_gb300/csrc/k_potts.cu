// k_potts.cu -- q = 4 Potts glass, H = -sum_<ij> J_ij delta(s_i, s_j),
// heat-bath update (IANUS_LAYOUT_U8X4).
//
// A 32-bit word holds one site of 4 samples (byte b = sample 4q+b, state
// 0..3), the counterpart of the paper's 2-bit Potts spins (Sec. 3.2); one
// Philox block supplies the 4 random words of the word.  The local counts
// n_k = sum_j J_ij [s_j == k] are kept as four biased nibbles (n_k + 6) of a
// 16-bit value, which indexes a table of cumulative heat-bath thresholds
// (the look-up table of Sec. 3.2); the new state is the smallest k with
// r < T_k, else 3.  Words of one colour are contiguous (checkerboard-split
// order, Sec. 3.1).
#include <algorithm>

#include "lattice.h"

namespace ianus {

namespace {

constexpr int kBlock = 256;

struct PottsParams {
  uint32_t* spins;         // [slots][Q4][N]
  const uint32_t* J;       // [Q4][D][N]
  const uint4* ptab;       // [K][65536]
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
__global__ void __launch_bounds__(kBlock) k_sweep_potts(const PottsParams p) {
  dependent_launch_entry();
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
    tab[b] = p.ptab + (size_t)k * 65536u;
  }
  const uint32_t c2 = (TAG_POTTS << 28) | ((uint32_t)sigma << 16) | (uint32_t)q;
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  const uint32_t w_begin = blockIdx.x * p.words_per_block;
  const uint32_t w_end = min(w_begin + p.words_per_block, geom.half);
  for (uint32_t w = w_begin + threadIdx.x; w < w_end; w += kBlock) {
    const Nbr n = split_neighbours(geom, p.colour, w);
    uint32_t jw[2 * D], nb[2 * D];
    jw[0] = __ldg(Jq + n.self);
    jw[1] = __ldg(Jq + n.xm);
    jw[2] = __ldg(Jq + N + n.self);
    jw[3] = __ldg(Jq + N + n.ym);
    nb[0] = sp[n.xp];
    nb[1] = sp[n.xm];
    nb[2] = sp[n.yp];
    nb[3] = sp[n.ym];
    if (D == 3) {
      jw[4] = __ldg(Jq + 2u * N + n.self);
      jw[5] = __ldg(Jq + 2u * N + n.zm);
      nb[4] = sp[n.zp];
      nb[5] = sp[n.zm];
    }
    const uint4 x = philox10(n.site, tk.lo, c2, tk.hi, p.keys);
    const uint32_t rr[4] = {x.x, x.y, x.z, x.w};
    uint32_t out = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      uint32_t npk = 0x6666u;  // nibble k holds n_k + 6
#pragma unroll
      for (int j = 0; j < 2 * D; ++j) {
        const uint32_t st = (nb[j] >> (8 * b)) & 3u;
        const int Jv = (int)(int8_t)(uint8_t)(jw[j] >> (8 * b));
        npk += (uint32_t)(Jv << (4 * st));
      }
      const uint4 T = __ldg(tab[b] + npk);
      const uint32_t r = rr[b];
      const uint32_t ge0 = !((T.w & 1u) || r < T.x);
      const uint32_t ge1 = !((T.w & 2u) || r < T.y);
      const uint32_t ge2 = !((T.w & 4u) || r < T.z);
      out |= (ge0 + ge1 + ge2) << (8 * b);
    }
    sp[n.self] = out;
  }
}

__global__ void k_init_potts(uint32_t* spins, uint32_t* J, Geom geom, int Q4, int slots, int ferro,
                             PhiloxKeys keys) {
  const uint64_t total = (uint64_t)Q4 * geom.N;
  const uint32_t L = (uint32_t)geom.L;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t q = (uint32_t)(idx / geom.N), i = (uint32_t)(idx - (uint64_t)q * geom.N);
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    const uint32_t j = split_index(geom, x, y, z);
    const uint32_t g = q >> 4, l0 = 4u * (q & 15u);
    for (int d = 0; d < geom.D; ++d) {
      const uint4 r = philox10(i, (uint32_t)d, (TAG_J << 28) | g, 0u, keys);
      const uint64_t wbits = (uint64_t)r.x | ((uint64_t)r.y << 32);
      uint32_t w = 0;
      for (int b = 0; b < 4; ++b) {
        const uint32_t neg = ferro ? 0u : (uint32_t)((wbits >> (l0 + b)) & 1ull);
        w |= (neg ? 0xFFu : 0x01u) << (8 * b);
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

// Per (slot, quad) block: E = -sum_bonds J delta and the state counts of the
// 4 samples of the quad (Sec. 4.1 observables for the Potts glass).
constexpr int kPottsMeasIters = 32;

template <int D>
__global__ void __launch_bounds__(kBlock) k_measure_potts(const uint32_t* __restrict__ spins,
                                                          const uint32_t* __restrict__ J, int64_t* acc, Geom geom,
                                                          int S, int Q4, int slots) {
  const int sq = blockIdx.y;  // sigma * Q4 + q
  const int sigma = sq / Q4, q = sq - sigma * Q4;
  const uint32_t N = geom.N, L = (uint32_t)geom.L, h = (uint32_t)geom.h;
  const uint32_t* Jq = J + (size_t)q * D * N;
  const uint32_t* sp = spins + ((size_t)sigma * Q4 + q) * N;
  const uint32_t base = blockIdx.x * (uint32_t)(kBlock * kPottsMeasIters);
  long long v[4][5];  // per sample: E, n0..n3
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int f = 0; f < 5; ++f) v[b][f] = 0;
  for (int it = 0; it < kPottsMeasIters; ++it) {
    const uint32_t j = base + (uint32_t)it * kBlock + threadIdx.x;
    if (j >= N) continue;
    const uint32_t rc = j / h, k = j - rc * h;
    const uint32_t row = rc >> 1, c = rc & 1u;
    const uint32_t y = row % L, z = row / L;
    const uint32_t x = 2u * k + ((c ^ (y + z)) & 1u);
    const uint32_t si = sp[j];
    uint32_t nbw[D], jw[D];
    nbw[0] = sp[split_index(geom, (int)((x + 1u) % L), (int)y, (int)z)];
    nbw[1] = sp[split_index(geom, (int)x, (int)((y + 1u) % L), (int)z)];
    jw[0] = Jq[j];
    jw[1] = Jq[N + j];
    if (D == 3) {
      nbw[2] = sp[split_index(geom, (int)x, (int)y, (int)((z + 1u) % L))];
      jw[2] = Jq[2u * N + j];
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const uint32_t st = (si >> (8 * b)) & 3u;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const uint32_t sn = (nbw[d] >> (8 * b)) & 3u;
        if (sn == st) v[b][0] -= (int)(int8_t)(uint8_t)(jw[d] >> (8 * b));
      }
      v[b][1 + st] += 1;
    }
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

// Q = sum_i delta(s_i^0, s_i^1) between the replica-0 and replica-1
// configurations holding temperature k; stored in acc[s][k*R][6].
__global__ void __launch_bounds__(kBlock) k_overlap_potts(const uint32_t* __restrict__ spins,
                                                          const int32_t* __restrict__ slot_at, int64_t* acc,
                                                          uint32_t N, int S, int R, int K, int Q4, int slots) {
  const int qk = blockIdx.y;  // q * K + k
  const int q = qk / K, k = qk - q * K;
  const uint32_t* w0[4];
  const uint32_t* w1[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int s = 4 * q + b;
    const int t0 = s < S ? slot_at[((size_t)s * R + 0) * K + k] : k;
    const int t1 = s < S ? slot_at[((size_t)s * R + 1) * K + k] : k;
    w0[b] = spins + ((size_t)(t0 * R + 0) * Q4 + q) * N;
    w1[b] = spins + ((size_t)(t1 * R + 1) * Q4 + q) * N;
  }
  const uint32_t base = blockIdx.x * (uint32_t)(kBlock * kPottsMeasIters);
  long long v[4] = {0, 0, 0, 0};
  for (int it = 0; it < kPottsMeasIters; ++it) {
    const uint32_t j = base + (uint32_t)it * kBlock + threadIdx.x;
    if (j >= N) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) v[b] += (((w0[b][j] ^ w1[b][j]) >> (8 * b)) & 3u) == 0u ? 1 : 0;
  }
#pragma unroll
  for (int b = 0; b < 4; ++b)
    for (int off = 16; off > 0; off >>= 1) v[b] += __shfl_down_sync(0xffffffffu, v[b], off);
  if ((threadIdx.x & 31) == 0) {
    for (int b = 0; b < 4; ++b) {
      const int s = 4 * q + b;
      if (s < S)
        atomicAdd((unsigned long long*)&acc[((size_t)s * slots + (size_t)k * R) * kAccStride + 6],
                  (unsigned long long)v[b]);
    }
  }
}

__global__ void k_get_spins_potts(const uint32_t* spins, int8_t* out, Geom geom, int S, int Q4, int slots) {
  const uint64_t total = (uint64_t)S * slots * geom.N;
  const uint32_t L = (uint32_t)geom.L;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(idx % geom.N);
    const uint64_t rest = idx / geom.N;
    const int sg = (int)(rest % slots), s = (int)(rest / slots);
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    const uint32_t w = spins[((size_t)sg * Q4 + (s >> 2)) * geom.N + split_index(geom, x, y, z)];
    out[idx] = (int8_t)((w >> (8 * (s & 3))) & 3u);
  }
}

__global__ void k_set_spins_potts(uint32_t* spins, const int8_t* in, Geom geom, int S, int Q4, int slots) {
  const uint64_t total = (uint64_t)S * slots * geom.N;
  const uint32_t L = (uint32_t)geom.L;
  // one thread per (slot, quad, site) so that bytes of one word are written together
  const uint64_t words = (uint64_t)slots * Q4 * geom.N;
  (void)total;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < words;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(idx % geom.N);
    const uint64_t rest = idx / geom.N;
    const int q = (int)(rest % Q4), sg = (int)(rest / Q4);
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    uint32_t* wp = &spins[((size_t)sg * Q4 + q) * geom.N + split_index(geom, x, y, z)];
    uint32_t w = *wp;
    for (int b = 0; b < 4; ++b) {
      const int s = 4 * q + b;
      if (s >= S) break;
      const uint32_t v = (uint32_t)in[((size_t)s * slots + sg) * geom.N + i] & 3u;
      w = (w & ~(0xFFu << (8 * b))) | (v << (8 * b));
    }
    *wp = w;
  }
}

__global__ void k_get_couplings_potts(const uint32_t* J, int8_t* out, Geom geom, int S) {
  const uint64_t total = (uint64_t)S * geom.D * geom.N;
  const uint32_t L = (uint32_t)geom.L;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(idx % geom.N);
    const uint64_t rest = idx / geom.N;
    const int d = (int)(rest % geom.D), s = (int)(rest / geom.D);
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    const uint32_t w = J[((size_t)(s >> 2) * geom.D + d) * geom.N + split_index(geom, x, y, z)];
    out[idx] = (int8_t)(uint8_t)(w >> (8 * (s & 3)));
  }
}

__global__ void k_set_couplings_potts(uint32_t* J, const int8_t* in, Geom geom, int S, int Q4) {
  const uint64_t words = (uint64_t)Q4 * geom.D * geom.N;
  const uint32_t L = (uint32_t)geom.L;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < words;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(idx % geom.N);
    const uint64_t rest = idx / geom.N;
    const int d = (int)(rest % geom.D), q = (int)(rest / geom.D);
    const int x = (int)(i % L), y = (int)((i / L) % L), z = geom.D == 3 ? (int)(i / (L * L)) : 0;
    uint32_t* wp = &J[((size_t)q * geom.D + d) * geom.N + split_index(geom, x, y, z)];
    uint32_t w = *wp;
    for (int b = 0; b < 4; ++b) {
      const int s = 4 * q + b;
      if (s >= S) break;
      const uint32_t v = (uint32_t)(uint8_t)in[((size_t)s * geom.D + d) * geom.N + i];
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

cudaError_t launch_init_potts(Lattice& lat, int jmode) {
  if (lat.model == IANUS_POTTS4_PERM) return launch_init_perm(lat, jmode);
  const int ferro = jmode == 1;  // Potts lattices take the J stream or J = +1
  k_init_potts<<<grid_for((uint64_t)lat.Q4 * lat.N), 256, 0, lat.stream>>>(
      (uint32_t*)lat.spins, (uint32_t*)lat.J, lat.geom, lat.Q4, lat.slots, ferro, lat.keys);
  return cudaGetLastError();
}

cudaError_t launch_sweep_potts(Lattice& lat, int colour, uint64_t t) {
  if (lat.model == IANUS_POTTS4_PERM) return launch_sweep_perm(lat, colour, t);
  PottsParams p;
  p.spins = (uint32_t*)lat.spins;
  p.J = (const uint32_t*)lat.J;
  p.ptab = lat.ptab;
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
  const void* k = lat.D == 3 ? (const void*)k_sweep_potts<3> : (const void*)k_sweep_potts<2>;
  return launch_dependent(k, grid, dim3(kBlock), args, 0, lat.stream);
}

cudaError_t launch_measure_potts(Lattice& lat, int want_q) {
  if (lat.model == IANUS_POTTS4_PERM) return launch_measure_perm(lat, want_q);
  cudaError_t e = cudaMemsetAsync(lat.acc, 0, (size_t)lat.S * lat.slots * kAccStride * sizeof(int64_t), lat.stream);
  if (e != cudaSuccess) return e;
  const uint32_t per_block = kBlock * kPottsMeasIters;
  dim3 grid((lat.N + per_block - 1) / per_block, (unsigned)(lat.slots * lat.Q4));
  if (lat.D == 3)
    k_measure_potts<3><<<grid, kBlock, 0, lat.stream>>>((const uint32_t*)lat.spins, (const uint32_t*)lat.J,
                                                         lat.acc, lat.geom, lat.S, lat.Q4, lat.slots);
  else
    k_measure_potts<2><<<grid, kBlock, 0, lat.stream>>>((const uint32_t*)lat.spins, (const uint32_t*)lat.J,
                                                         lat.acc, lat.geom, lat.S, lat.Q4, lat.slots);
  if (want_q && lat.R >= 2) return launch_overlap_potts(lat);
  return cudaGetLastError();
}

cudaError_t launch_overlap_potts(Lattice& lat) {
  const uint32_t per_block = kBlock * kPottsMeasIters;
  dim3 gq((lat.N + per_block - 1) / per_block, (unsigned)(lat.Q4 * lat.K));
  k_overlap_potts<<<gq, kBlock, 0, lat.stream>>>((const uint32_t*)lat.spins, lat.slot_at, lat.acc, lat.N, lat.S,
                                                 lat.R, lat.K, lat.Q4, lat.slots);
  return cudaGetLastError();
}

cudaError_t launch_get_spins_potts(Lattice& lat, int8_t* dev_out) {
  if (lat.model == IANUS_POTTS4_PERM) return launch_get_spins_perm(lat, dev_out);
  k_get_spins_potts<<<grid_for((uint64_t)lat.S * lat.slots * lat.N), 256, 0, lat.stream>>>(
      (const uint32_t*)lat.spins, dev_out, lat.geom, lat.S, lat.Q4, lat.slots);
  return cudaGetLastError();
}

cudaError_t launch_set_spins_potts(Lattice& lat, const int8_t* dev_in) {
  if (lat.model == IANUS_POTTS4_PERM) return launch_set_spins_perm(lat, dev_in);
  k_set_spins_potts<<<grid_for((uint64_t)lat.slots * lat.Q4 * lat.N), 256, 0, lat.stream>>>(
      (uint32_t*)lat.spins, dev_in, lat.geom, lat.S, lat.Q4, lat.slots);
  return cudaGetLastError();
}

cudaError_t launch_get_couplings_potts(Lattice& lat, int8_t* dev_out) {
  if (lat.model == IANUS_POTTS4_PERM) return launch_get_couplings_perm(lat, dev_out);
  k_get_couplings_potts<<<grid_for((uint64_t)lat.S * lat.D * lat.N), 256, 0, lat.stream>>>(
      (const uint32_t*)lat.J, dev_out, lat.geom, lat.S);
  return cudaGetLastError();
}

cudaError_t launch_set_couplings_potts(Lattice& lat, const int8_t* dev_in) {
  if (lat.model == IANUS_POTTS4_PERM) return launch_set_couplings_perm(lat, dev_in);
  k_set_couplings_potts<<<grid_for((uint64_t)lat.Q4 * lat.D * lat.N), 256, 0, lat.stream>>>(
      (uint32_t*)lat.J, dev_in, lat.geom, lat.S, lat.Q4);
  return cudaGetLastError();
}

}  // namespace ianus
