// k_resident_bits.cu -- resident sweeps of small bit-sliced lattices: many
// sweeps per launch, the lattice held in shared memory.
//
// A sweep is colour 0 then colour 1 over every site (Sec. 2.2, Sec. 3.1).  A
// small lattice (a serving job, a pool of small jobs) does too little work
// per colour pass to fill the GPU, so one launch per colour pass leaves it
// bound by launch latency.  Here one block holds everything one
// configuration set needs -- its spin words, its group's coupling words and
// its per-lane threshold planes -- in shared memory and runs every sweep up
// to the next measurement point, the two colours separated by block
// barriers; the spins go back to global memory at the end.  The update of a
// word is the one of the per-lane-plane sweep (sweep_planes.cuh, Sec. 3.2 in
// bit-sliced form) with the same random stream, so the trajectory is the
// same bit for bit.
//
// k_resident_bits: one block per (group, temperature slot), its R replicas.
// k_resident_fused: one block per group of a fused serving pool, with the
// pool's segments (jobs) and their sweep counters kept in shared memory and
// advanced after every sweep, as the per-pass pool kernels do.
#include "lattice.h"
#include "sweep_planes.cuh"

namespace ianus {

namespace {

constexpr int kResThreads = 512;
// dynamic shared memory a block may use (the fused kernel adds its segment
// table, under 3 KB, as static shared memory)
constexpr size_t kResSmemMax = 220u * 1024u;

uint32_t res_threads(uint32_t half) {
  uint32_t t = (half + 31u) & ~31u;
  return t < 32u ? 32u : (t > (uint32_t)kResThreads ? (uint32_t)kResThreads : t);
}

// Coupling words of a colour-c word's 2D bonds: bond d of a site is stored
// at the site (x+, y+, z+); the minus bonds are the plus bonds of the
// neighbours.
template <int D>
__device__ __forceinline__ void bond_words(const uint64_t* sJ, uint32_t N, const Nbr& n, uint64_t* jw) {
  jw[0] = sJ[n.self];
  jw[1] = sJ[n.xm];
  jw[2] = sJ[N + n.self];
  jw[3] = sJ[N + n.ym];
  if (D == 3) {
    jw[4] = sJ[2u * N + n.self];
    jw[5] = sJ[2u * N + n.zm];
  }
}

template <int D, int ALGO, bool P2>
__global__ void __launch_bounds__(kResThreads, 1) k_resident_bits(const BitsParams p, uint32_t nsweeps) {
  extern __shared__ uint64_t sm[];
  const uint32_t R = (uint32_t)p.R, N = p.geom.N, half = p.geom.half;
  const int g = (int)blockIdx.x / p.K, tslot = (int)blockIdx.x - g * p.K;
  uint64_t* s_sp = sm;                          // [R][N]
  uint64_t* s_J = s_sp + (size_t)R * N;         // [D][N]
  uint64_t* s_tp = s_J + (size_t)D * N;         // [R][kPlanes][kMaxClasses]
  uint4* s_u = reinterpret_cast<uint4*>(s_tp + (size_t)R * kPlanes * kMaxClasses);  // [R][16] Philox parts
  uint64_t* g_sp = p.spins + ((size_t)g * p.slots + (size_t)tslot * R) * N;
  const uint64_t* g_J = p.J + (size_t)g * D * N;
  const uint64_t* g_tp = p.tp + ((size_t)g * p.slots + (size_t)tslot * R) * kPlanes * kMaxClasses;
  for (uint32_t i = threadIdx.x; i < R * N; i += blockDim.x) s_sp[i] = g_sp[i];
  for (uint32_t i = threadIdx.x; i < (uint32_t)D * N; i += blockDim.x) s_J[i] = __ldg(g_J + i);
  for (uint32_t i = threadIdx.x; i < R * kPlanes * kMaxClasses; i += blockDim.x) s_tp[i] = g_tp[i];
  __syncthreads();
  const uint64_t t0 = ((uint64_t)p.t_hi << 32) | p.t_lo;
#pragma unroll 1
  for (uint32_t s = 0; s < nsweeps; ++s) {
    const uint64_t t = t0 + s;
    const Tick tk{(uint32_t)t, (uint32_t)(t >> 32)};
    // this sweep's Philox parts shared by the block (the previous sweep's
    // last barrier has passed every reader of the old ones)
    planes::plane_uniform_table(s_u, (int)R, tslot * (int)R, (uint32_t)g, tk, p.keys);
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
#pragma unroll 1
      for (uint32_t w = threadIdx.x; w < half; w += blockDim.x) {
        const Nbr n = split_neighbours_t<P2>(p.geom, c, w);
        uint64_t jw[2 * D];
        bond_words<D>(s_J, N, n, jw);
        const planes::PlaneSiteKey sk = planes::plane_site_key(n.site, tk, p.keys);
#pragma unroll 1
        for (uint32_t a = 0; a < R; ++a) {
          uint64_t* sp = s_sp + (size_t)a * N;
          const uint64_t* tpa = s_tp + (size_t)a * kPlanes * kMaxClasses;
          uint64_t b, u0, u1, u2;
          planes::bits_class_planes<D>(sp, n, jw, b, u0, u1, u2);
          planes::LazyWord lw = planes::bits_word_start<D, ALGO>(tpa, u0, u1, u2);
          planes::bits_plane_pairs<D, ALGO>(lw, tpa, s_u + 16u * a, sk, p.keys, 0u, tk, 0u, 16u);
          const uint64_t flip = ALGO == 0 ? lw.lt : ~lw.lt;
          if (flip) sp[n.self] = b ^ flip;
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < R * N; i += blockDim.x) g_sp[i] = s_sp[i];
}

template <int D, bool P2>
__global__ void __launch_bounds__(kResThreads, 1) k_resident_fused(const BitsParams p, Segment* segs,
                                                                   const uint32_t* __restrict__ nseg,
                                                                   uint32_t nsweeps) {
  extern __shared__ uint64_t sm[];
  __shared__ uint64_t s_mask[kMaxSegs], s_t[kMaxSegs], s_tend[kMaxSegs];
  __shared__ uint32_t s_klo[kMaxSegs], s_khi[kMaxSegs], s_lane0[kMaxSegs], s_c2[kMaxSegs], s_inv[kMaxSegs];
  __shared__ uint64_t s_live, s_invm;
  __shared__ int s_n;
  const int g = (int)blockIdx.x;
  const uint32_t N = p.geom.N, half = p.geom.half;
  uint64_t* s_sp = sm;                  // [N] (one slot per group)
  uint64_t* s_J = s_sp + N;             // [D][N]
  uint64_t* tpa = s_J + (size_t)D * N;  // [kPlanes][kMaxClasses]
  uint64_t* g_sp = p.spins + (size_t)g * N;
  const uint64_t* g_J = p.J + (size_t)g * D * N;
  for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) s_sp[i] = g_sp[i];
  for (uint32_t i = threadIdx.x; i < (uint32_t)D * N; i += blockDim.x) s_J[i] = __ldg(g_J + i);
  for (uint32_t i = threadIdx.x; i < kPlanes * kMaxClasses; i += blockDim.x)
    tpa[i] = p.tp[(size_t)g * kPlanes * kMaxClasses + i];
  if (threadIdx.x == 0) {
    const uint32_t ns = min(nseg[g], (uint32_t)kMaxSegs);
    for (uint32_t j = 0; j < ns; ++j) {
      const Segment sg = segs[(size_t)g * kMaxSegs + j];
      s_mask[j] = sg.mask;
      s_t[j] = sg.t;
      s_tend[j] = sg.t_end;
      s_klo[j] = sg.key_lo;
      s_khi[j] = sg.key_hi;
      s_lane0[j] = sg.lane0;
      s_c2[j] = (TAG_SPIN << 28) | sg.jgroup;  // slot 0, the job's own group
      s_inv[j] = sg.inv;
    }
    s_n = (int)ns;
  }
#pragma unroll 1
  for (uint32_t s = 0; s < nsweeps; ++s) {
    __syncthreads();
    if (threadIdx.x == 0) {  // the segments still running this sweep
      uint64_t live = 0, inv = 0;
      for (int j = 0; j < s_n; ++j)
        if (s_mask[j] != 0ull && s_t[j] < s_tend[j]) {
          live |= s_mask[j];
          if (s_inv[j]) inv |= s_mask[j];
        }
      s_live = live;
      s_invm = inv;
    }
    __syncthreads();
    const uint64_t live = s_live, inv = s_invm;
    if (live == 0ull) break;  // every job done: later sweeps change nothing
    const int nsg = s_n;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
#pragma unroll 1
      for (uint32_t w = threadIdx.x; w < half; w += blockDim.x) {
        const Nbr n = split_neighbours_t<P2>(p.geom, c, w);
        uint64_t jw[2 * D];
        bond_words<D>(s_J, N, n, jw);
        uint64_t b, u0, u1, u2;
        planes::bits_class_planes<D>(s_sp, n, jw, b, u0, u1, u2);
        // a segment's lanes may hold either algorithm's planes: select over all classes
        const uint64_t always = planes::class_select<D, 1>(tpa + 32 * kMaxClasses, u0, u1, u2);
        uint64_t lt = always;
        uint64_t und = ~always & live;
#pragma unroll 1
        for (uint32_t mm = 0; mm < 16u && und != 0ull; ++mm) {
          uint64_t r0 = 0, r1 = 0;
#pragma unroll 1
          for (int j = 0; j < nsg; ++j) {
            const uint64_t mk = s_mask[j];
            if (!(und & mk)) continue;
            const uint64_t tj = s_t[j];
            const uint4 x = philox10_key(n.site, (uint32_t)tj, s_c2[j] | (mm << 24), (uint32_t)(tj >> 32), s_klo[j],
                                         s_khi[j]);
            const uint32_t sh = s_lane0[j];
            r0 |= (((uint64_t)x.x | ((uint64_t)x.y << 32)) << sh) & mk;
            r1 |= (((uint64_t)x.z | ((uint64_t)x.w << 32)) << sh) & mk;
          }
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const uint64_t r = q == 0 ? r0 : r1;
            const uint64_t tb = planes::class_select<D, 1>(tpa + (2u * mm + (uint32_t)q) * kMaxClasses, u0, u1, u2);
            lt |= und & ~r & tb;
            und &= ~(r ^ tb);
          }
        }
        const uint64_t flip = (lt ^ inv) & live;
        if (flip) s_sp[n.self] = b ^ flip;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0)  // every running segment has done one more sweep
      for (int j = 0; j < s_n; ++j)
        if (s_mask[j] != 0ull && s_t[j] < s_tend[j]) s_t[j] += 1;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) g_sp[i] = s_sp[i];
  if (threadIdx.x == 0)
    for (int j = 0; j < s_n; ++j) segs[(size_t)g * kMaxSegs + j].t = s_t[j];
}

template <typename K>
cudaError_t allow_smem(K kern, bool& done) {
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResSmemMax);
  if (e == cudaSuccess) done = true;
  return e;
}

template <int D, int ALGO, bool P2>
cudaError_t launch_bits_t(Lattice& lat, const BitsParams& p, uint32_t nsweeps, size_t smem) {
  static bool ok = false;
  cudaError_t e = allow_smem(k_resident_bits<D, ALGO, P2>, ok);
  if (e != cudaSuccess) return e;
  k_resident_bits<D, ALGO, P2><<<(unsigned)(lat.G * lat.K), res_threads(lat.geom.half), smem, lat.stream>>>(p, nsweeps);
  return cudaGetLastError();
}

template <int D, bool P2>
cudaError_t launch_fused_t(Lattice& lat, const BitsParams& p, uint32_t nsweeps, size_t smem) {
  static bool ok = false;
  cudaError_t e = allow_smem(k_resident_fused<D, P2>, ok);
  if (e != cudaSuccess) return e;
  k_resident_fused<D, P2><<<(unsigned)lat.G, res_threads(lat.geom.half), smem, lat.stream>>>(p, lat.segs, lat.nseg,
                                                                                            nsweeps);
  return cudaGetLastError();
}

size_t resident_bits_smem(const Lattice& lat) {
  return ((size_t)lat.R * lat.N + (size_t)lat.D * lat.N + (size_t)lat.R * kPlanes * kMaxClasses) * sizeof(uint64_t) +
         (size_t)lat.R * 16 * sizeof(uint4);
}

size_t resident_fused_smem(const Lattice& lat) {
  return ((size_t)lat.N + (size_t)lat.D * lat.N + (size_t)kPlanes * kMaxClasses) * sizeof(uint64_t);
}

BitsParams resident_params(const Lattice& lat, uint64_t t0) {
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
  return p;
}

}  // namespace

// One block sweeps its R N words in about 5.5 ns each on GB300 (3D heat
// bath), while a sweep of two launches costs about 4.5 us of launch latency
// when the lattice is small: the block wins up to about 512 words per sweep,
// and up to 1024 when there are enough blocks (32 or more) that the
// launch-per-colour sweep has real work to spread.  Measured on 3D L = 8..16
// and 2D L = 32, 64, 1 to 152 groups, one and two replicas.
static bool resident_pays(uint64_t words, uint64_t blocks, int mode) {
  return mode >= 2 || words <= 512u || (words <= 1024u && blocks >= 32u);
}

bool resident_bits_fits(const Lattice& lat) {
  return lat.layout == IANUS_LAYOUT_BITS64 && lat.model == IANUS_EA_PM_J && !lat.field && !lat.pool &&
         (lat.D == 2 || lat.D == 3) && resident_bits_smem(lat) <= kResSmemMax &&
         resident_pays((uint64_t)lat.R * lat.N, (uint64_t)lat.G * lat.K, lat.resident_mode);
}

bool resident_fused_fits(const Lattice& lat) {
  return lat.layout == IANUS_LAYOUT_BITS64 && lat.pool && lat.segs && (lat.D == 2 || lat.D == 3) &&
         resident_fused_smem(lat) <= kResSmemMax && resident_pays(lat.N, (uint64_t)lat.G, lat.resident_mode);
}

cudaError_t launch_resident_bits(Lattice& lat, int inv, uint64_t t0, uint32_t nsweeps) {
  const BitsParams p = resident_params(lat, t0);
  const size_t smem = resident_bits_smem(lat);
  const bool p2 = lat.geom.lL > 0;
  if (lat.D == 3) {
    if (inv) return p2 ? launch_bits_t<3, 1, true>(lat, p, nsweeps, smem) : launch_bits_t<3, 1, false>(lat, p, nsweeps, smem);
    return p2 ? launch_bits_t<3, 0, true>(lat, p, nsweeps, smem) : launch_bits_t<3, 0, false>(lat, p, nsweeps, smem);
  }
  if (inv) return p2 ? launch_bits_t<2, 1, true>(lat, p, nsweeps, smem) : launch_bits_t<2, 1, false>(lat, p, nsweeps, smem);
  return p2 ? launch_bits_t<2, 0, true>(lat, p, nsweeps, smem) : launch_bits_t<2, 0, false>(lat, p, nsweeps, smem);
}

cudaError_t launch_resident_fused(Lattice& lat, uint32_t nsweeps) {
  BitsParams p = resident_params(lat, 0);
  p.R = p.K = p.slots = 1;
  const size_t smem = resident_fused_smem(lat);
  const bool p2 = lat.geom.lL > 0;
  if (lat.D == 3) return p2 ? launch_fused_t<3, true>(lat, p, nsweeps, smem) : launch_fused_t<3, false>(lat, p, nsweeps, smem);
  return p2 ? launch_fused_t<2, true>(lat, p, nsweeps, smem) : launch_fused_t<2, false>(lat, p, nsweeps, smem);
}

}  // namespace ianus
