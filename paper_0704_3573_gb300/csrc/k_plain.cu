// k_plain.cu -- the plain one-byte-per-spin layout (IANUS_LAYOUT_I8).
//
// One thread updates one site of the active colour of one configuration
// (Sec. 3.1: all sites of one colour are independent).  The update cell of
// Sec. 3.2 becomes: count the unsatisfied bonds u among the 2D bonds, look
// up the class threshold T(u), compare against the site's 32-bit random
// number, write the new spin.  The random number is produced lazily, two
// bit-planes per Philox call, from the most significant bit down, and the
// comparison stops at the first plane where r and T differ.
#include <algorithm>
#include <cmath>

#include <cooperative_groups.h>

#include "lattice.h"
#include "sweep_planes.cuh"

namespace ianus {

namespace {

struct I8Params {
  int8_t* spins;            // [slots][S][N]
  const int8_t* J;          // [S][D][N]
  const uint64_t* thr;      // [K][kMaxClasses]
  const int32_t* temp_of;   // [S][R][K]
  int S, R, K, slots, L;
  uint32_t N, half;
  int colour, inv;
  uint32_t t_lo, t_hi;
  PhiloxKeys keys;
  const uint64_t* t_dev;  // non-null in captured graphs
};

// r < T for the random r of (sample, slot, site, sweep), decided from the
// most significant plane down.  T in [0, 2^32].
__device__ __forceinline__ bool lazy_less(uint64_t T, const I8Params& p, const Tick& tk, int s, int sigma,
                                          uint32_t site) {
  if (T >= kTwo32) return true;
  const uint32_t T32 = (uint32_t)T;
  const uint32_t lane = (uint32_t)s & 63u, g = (uint32_t)s >> 6;
  const uint32_t c2base = (TAG_SPIN << 28) | ((uint32_t)sigma << 12) | g;
#pragma unroll 1
  for (uint32_t m = 0; m < 16u; ++m) {
    const uint4 x = philox10(site, tk.lo, c2base | (m << 24), tk.hi, p.keys);
    const uint32_t w0 = lane < 32u ? (x.x >> lane) : (x.y >> (lane - 32u));
    const uint32_t w1 = lane < 32u ? (x.z >> lane) : (x.w >> (lane - 32u));
    const uint32_t r0 = w0 & 1u, t0 = (T32 >> (31u - 2u * m)) & 1u;
    if (r0 != t0) return r0 < t0;
    const uint32_t r1 = w1 & 1u, t1 = (T32 >> (30u - 2u * m)) & 1u;
    if (r1 != t1) return r1 < t1;
  }
  return false;  // r == T
}

template <int D>
__global__ void __launch_bounds__(256) k_sweep_i8(const I8Params p) {
  const uint64_t total = (uint64_t)p.slots * p.S * p.half;
  const uint32_t L = (uint32_t)p.L, h = L / 2u;
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t lat = (uint32_t)(idx / p.half);
    const uint32_t w = (uint32_t)(idx - (uint64_t)lat * p.half);
    const int sigma = (int)(lat / (uint32_t)p.S);
    const int s = (int)(lat - (uint32_t)sigma * (uint32_t)p.S);
    const uint32_t row = w / h, k = w - row * h;
    const uint32_t y = row % L, z = row / L;
    const uint32_t x = 2u * k + ((uint32_t)(p.colour ^ (int)(y + z)) & 1u);
    const uint32_t i = x + L * (y + L * z);
    int8_t* sp = p.spins + (size_t)lat * p.N;
    const int8_t* Jp = p.J + (size_t)s * D * p.N;
    const int si = sp[i];
    // neighbours along each axis (periodic)
    const uint32_t xp = (x + 1u == L ? 0u : x + 1u) + L * (y + L * z);
    const uint32_t xm = (x == 0u ? L - 1u : x - 1u) + L * (y + L * z);
    const uint32_t yp = x + L * ((y + 1u == L ? 0u : y + 1u) + L * z);
    const uint32_t ym = x + L * ((y == 0u ? L - 1u : y - 1u) + L * z);
    int u = 0;
    u += (Jp[i] * si * sp[xp]) < 0;
    u += (Jp[xm] * si * sp[xm]) < 0;
    u += (Jp[p.N + i] * si * sp[yp]) < 0;
    u += (Jp[p.N + ym] * si * sp[ym]) < 0;
    if (D == 3) {
      const uint32_t zp = x + L * (y + L * (z + 1u == L ? 0u : z + 1u));
      const uint32_t zm = x + L * (y + L * (z == 0u ? L - 1u : z - 1u));
      u += (Jp[2u * p.N + i] * si * sp[zp]) < 0;
      u += (Jp[2u * p.N + zm] * si * sp[zm]) < 0;
    }
    const int tslot = sigma / p.R, a = sigma - tslot * p.R;
    const int kt = p.temp_of[((size_t)s * p.R + a) * p.K + tslot];
    const uint64_t T = p.thr[(size_t)kt * kMaxClasses + u];
    const bool less = lazy_less(T, p, tk, s, sigma, i);
    if (less != (p.inv != 0)) sp[i] = (int8_t)(-si);
  }
}


// ---- plain layout, tiled: the random planes of a site shared by its group ----
//
// The random number of sample s at (site, sweep) is bit (s mod 64) of the
// 32 bit-planes drawn for the site and its group of 64 samples, so one
// Philox block serves 64 updates.  A block of kTileThreads threads takes a
// tile of up to kTileSites colour-c sites (consecutive colour words
// w = row * L/2 + k of one configuration slot) and one group:
//   phase A: one thread per site draws plane pairs 0..3 (planes 0..7) and
//     transposes them, 8 lanes at a time (an 8 x 8 bit transpose), into one
//     8-bit prefix of the random number per (site, lane) in shared memory;
//     the block also stages the class thresholds of its 64 samples;
//   phase B: thread t keeps site t and runs through the group's samples, so
//     the 32 threads of a warp read 32 neighbouring sites of one sample;
//     each update compares the 8-bit prefix with the top 8 bits of its
//     threshold and is decided there unless the two are equal (probability
//     1/256), in which case it continues with pairs 4.. on its own.
constexpr int kTileThreads = 256;
constexpr int kTileSites = 256;
constexpr int kTileRow = 68;  // bytes per site of prefixes: 64 lanes + 4 of padding (no bank conflicts)

// 8 x 8 bit transpose: element (i, j) = bit 8 i + j goes to bit 8 j + i.
__device__ __forceinline__ uint64_t transpose8(uint64_t x) {
  uint64_t t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
  x = x ^ t ^ (t << 7);
  t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
  x = x ^ t ^ (t << 14);
  t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
  return x ^ t ^ (t << 28);
}

// r < T decided from plane pairs m0.. of the lane's random number (the
// planes before m0 equal those of T).
__device__ __noinline__ bool lazy_less_from(uint32_t T32, uint32_t m0, const I8Params& p, const Tick& tk, int sigma,
                                            uint32_t g, uint32_t lane, uint32_t site) {
  const uint32_t c2base = (TAG_SPIN << 28) | ((uint32_t)sigma << 12) | g;
  for (uint32_t m = m0; m < 16u; ++m) {
    const uint4 x = philox10(site, tk.lo, c2base | (m << 24), tk.hi, p.keys);
    const uint32_t w0 = lane < 32u ? (x.x >> lane) : (x.y >> (lane - 32u));
    const uint32_t w1 = lane < 32u ? (x.z >> lane) : (x.w >> (lane - 32u));
    const uint32_t r0 = w0 & 1u, t0 = (T32 >> (31u - 2u * m)) & 1u;
    if (r0 != t0) return r0 < t0;
    const uint32_t r1 = w1 & 1u, t1 = (T32 >> (30u - 2u * m)) & 1u;
    if (r1 != t1) return r1 < t1;
  }
  return false;  // r == T
}

// grid: (tiles of kTileSites colour words, groups, slots)
template <int D>
__global__ void __launch_bounds__(kTileThreads) k_sweep_i8_tiled(const I8Params p) {
  __shared__ __align__(16) uint8_t s_r8[kTileSites * kTileRow];
  __shared__ uint64_t s_thr[64][kMaxClasses];
  const uint32_t g = blockIdx.y;
  const int sigma = (int)blockIdx.z;
  const uint32_t L = (uint32_t)p.L, h = L / 2u;
  const uint32_t w0 = blockIdx.x * (uint32_t)kTileSites;
  const uint32_t nsites = min((uint32_t)kTileSites, p.half - w0);
  const uint32_t t = threadIdx.x;
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  // the site of this thread: colour word w -> row, k -> natural index
  const bool has_site = t < nsites;
  uint32_t i = 0, xp = 0, xm = 0, yp = 0, ym = 0, zp = 0, zm = 0;
  if (has_site) {
    const uint32_t w = w0 + t;
    const uint32_t row = w / h, k = w - row * h;
    const uint32_t y = row % L, z = row / L;
    const uint32_t x = 2u * k + ((uint32_t)(p.colour ^ (int)(y + z)) & 1u);
    i = x + L * row;
    xp = (x + 1u == L ? 0u : x + 1u) + L * row;
    xm = (x == 0u ? L - 1u : x - 1u) + L * row;
    yp = x + L * ((y + 1u == L ? 0u : y + 1u) + L * z);
    ym = x + L * ((y == 0u ? L - 1u : y - 1u) + L * z);
    if (D == 3) {
      zp = x + L * (y + L * (z + 1u == L ? 0u : z + 1u));
      zm = x + L * (y + L * (z == 0u ? L - 1u : z - 1u));
    }
  }
  // phase A: planes 0..7 of the site for the group's 64 lanes, as 8-bit prefixes
  if (has_site) {
    const uint32_t c2base = (TAG_SPIN << 28) | ((uint32_t)sigma << 12) | g;
    uint32_t pw[8][2];  // plane p: lanes 0..31, 32..63
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const uint4 x = philox10(i, tk.lo, c2base | ((uint32_t)m << 24), tk.hi, p.keys);
      pw[2 * m][0] = x.x;
      pw[2 * m][1] = x.y;
      pw[2 * m + 1][0] = x.z;
      pw[2 * m + 1][1] = x.w;
    }
    uint8_t* dst = s_r8 + t * kTileRow;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      // byte 7 - p of M = byte c of plane p's 64-bit word (lanes 8c .. 8c+7)
      const int hw = c >> 2, sh = 8 * (c & 3);
      uint64_t M = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) M |= (uint64_t)((pw[q][hw] >> sh) & 0xFFu) << (8 * (7 - q));
      const uint64_t r = transpose8(M);  // byte j: lane 8c + j, bit 7 - p = plane p
      *reinterpret_cast<uint32_t*>(dst + 8 * c) = (uint32_t)r;
      *reinterpret_cast<uint32_t*>(dst + 8 * c + 4) = (uint32_t)(r >> 32);
    }
  }
  // thresholds of the group's samples (their temperatures may differ)
  for (uint32_t e = t; e < 64u * kMaxClasses; e += kTileThreads) {
    const uint32_t lane = e / kMaxClasses, u = e - lane * kMaxClasses;
    const uint32_t s = 64u * g + lane;
    uint64_t T = 0;
    if (s < (uint32_t)p.S) {
      const int tslot = sigma / p.R, a = sigma - tslot * p.R;
      const int kt = p.temp_of[((size_t)s * p.R + a) * p.K + tslot];
      T = p.thr[(size_t)kt * kMaxClasses + u];
    }
    s_thr[lane][u] = T;
  }
  __syncthreads();
  if (!has_site) return;
  // phase B: site t, every sample of the group
  const uint32_t lanes = min(64u, (uint32_t)p.S - 64u * g);
  const uint32_t N = p.N;
  const int8_t* r8row = reinterpret_cast<const int8_t*>(s_r8 + t * kTileRow);
  for (uint32_t lane = 0; lane < lanes; ++lane) {
    const uint32_t s = 64u * g + lane;
    int8_t* sp = p.spins + ((size_t)sigma * p.S + s) * N;
    const int8_t* Jp = p.J + (size_t)s * D * N;
    const int si = sp[i];
    int u = (Jp[i] * si * sp[xp] < 0) + (Jp[xm] * si * sp[xm] < 0) + (Jp[N + i] * si * sp[yp] < 0) +
            (Jp[N + ym] * si * sp[ym] < 0);
    if (D == 3) u += (Jp[2u * N + i] * si * sp[zp] < 0) + (Jp[2u * N + zm] * si * sp[zm] < 0);
    const uint64_t T = s_thr[lane][u];
    bool less;
    if (T >= kTwo32) {
      less = true;
    } else {
      const uint32_t r8 = (uint8_t)r8row[lane], T8 = (uint32_t)(T >> 24);
      if (r8 != T8)
        less = r8 < T8;
      else
        less = lazy_less_from((uint32_t)T, 4u, p, tk, sigma, g, lane, i);
    }
    if (less != (p.inv != 0)) sp[i] = (int8_t)(-si);
  }
}

// The same with each thread on one aligned 4-byte word of a row (sites
// x0 .. x0+3, two of them of the active colour), for L a multiple of 4.  The
// local fields of the word's four sites come out together: per direction
// the sign bits of s_i ^ s_j ^ J_ij (bytes of +-1) mark the unsatisfied
// bonds, x-neighbours by funnel shifts with the adjacent words, and the
// per-byte counts are summed in the word.  Thread t takes word q0 + t of
// every sample of the group, loading the next sample's words while it
// updates the current one (the sweep waits on memory, not on arithmetic).
// Its two active sites are rows j kWordThreads + t of the prefix table.
constexpr int kWordThreads = 128;

// the words one update of a 4-byte word reads
template <int D>
struct WordLoads {
  uint32_t self, prev, next, yp, ym, zp, zm;
  uint32_t j0s, j0p, j1s, j1m, j2s, j2m;
};

struct WordOffsets {
  uint32_t self, prev, next, yp, ym, zp, zm;
};

template <int D>
__device__ __forceinline__ void load_word(WordLoads<D>& w, const int8_t* sp, const int8_t* Jp, uint32_t N,
                                          const WordOffsets& o) {
  w.self = *reinterpret_cast<const uint32_t*>(sp + o.self);
  w.prev = *reinterpret_cast<const uint32_t*>(sp + o.prev);
  w.next = *reinterpret_cast<const uint32_t*>(sp + o.next);
  w.yp = *reinterpret_cast<const uint32_t*>(sp + o.yp);
  w.ym = *reinterpret_cast<const uint32_t*>(sp + o.ym);
  w.j0s = __ldg(reinterpret_cast<const uint32_t*>(Jp + o.self));
  w.j0p = __ldg(reinterpret_cast<const uint32_t*>(Jp + o.prev));
  w.j1s = __ldg(reinterpret_cast<const uint32_t*>(Jp + N + o.self));
  w.j1m = __ldg(reinterpret_cast<const uint32_t*>(Jp + N + o.ym));
  if (D == 3) {
    w.zp = *reinterpret_cast<const uint32_t*>(sp + o.zp);
    w.zm = *reinterpret_cast<const uint32_t*>(sp + o.zm);
    w.j2s = __ldg(reinterpret_cast<const uint32_t*>(Jp + 2u * N + o.self));
    w.j2m = __ldg(reinterpret_cast<const uint32_t*>(Jp + 2u * N + o.zm));
  }
}

template <int D>
__global__ void __launch_bounds__(kWordThreads, 6) k_sweep_i8_words(const I8Params p) {
  __shared__ __align__(16) uint8_t s_r8[2 * kWordThreads * kTileRow];
  __shared__ uint32_t s_thr[64][kMaxClasses];  // low 32 bits of T (the lazy path)
  __shared__ uint16_t s_t8[64][kMaxClasses];   // top 8 bits of T, 256 for T = 2^32 (always below)
  const uint32_t g = blockIdx.y;
  const int sigma = (int)blockIdx.z;
  const uint32_t L = (uint32_t)p.L, N = p.N, nq = N / 4u, qrow = L / 4u;
  const uint32_t q0 = blockIdx.x * (uint32_t)kWordThreads;
  const uint32_t t = threadIdx.x;
  const bool has = q0 + t < nq;
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  uint32_t row = 0, x0 = 0, y = 0, z = 0, b0 = 0;
  if (has) {
    const uint32_t q = q0 + t;
    row = q / qrow;
    x0 = 4u * (q - row * qrow);
    y = row % L;
    z = row / L;
    b0 = (uint32_t)(p.colour ^ (int)(y + z)) & 1u;  // byte of the first active site
  }
  // phase A: planes 0..7 of the two active sites for the group's 64 lanes
  if (has) {
    const uint32_t c2base = (TAG_SPIN << 28) | ((uint32_t)sigma << 12) | g;
#pragma unroll 1
    for (int j = 0; j < 2; ++j) {
      const uint32_t i = x0 + b0 + 2u * (uint32_t)j + L * row;
      uint32_t pw[8][2];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const uint4 x = philox10(i, tk.lo, c2base | ((uint32_t)m << 24), tk.hi, p.keys);
        pw[2 * m][0] = x.x;
        pw[2 * m][1] = x.y;
        pw[2 * m + 1][0] = x.z;
        pw[2 * m + 1][1] = x.w;
      }
      uint8_t* dst = s_r8 + ((uint32_t)j * kWordThreads + t) * kTileRow;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int hw = c >> 2, sh = 8 * (c & 3);
        uint64_t M = 0;
#pragma unroll
        for (int qq = 0; qq < 8; ++qq) M |= (uint64_t)((pw[qq][hw] >> sh) & 0xFFu) << (8 * (7 - qq));
        const uint64_t r = transpose8(M);
        *reinterpret_cast<uint32_t*>(dst + 8 * c) = (uint32_t)r;
        *reinterpret_cast<uint32_t*>(dst + 8 * c + 4) = (uint32_t)(r >> 32);
      }
    }
  }
  for (uint32_t e = t; e < 64u * kMaxClasses; e += kWordThreads) {
    const uint32_t lane = e / kMaxClasses, u = e - lane * kMaxClasses;
    const uint32_t s = 64u * g + lane;
    uint64_t T = 0;
    if (s < (uint32_t)p.S) {
      const int tslot = sigma / p.R, a = sigma - tslot * p.R;
      const int kt = p.temp_of[((size_t)s * p.R + a) * p.K + tslot];
      T = p.thr[(size_t)kt * kMaxClasses + u];
    }
    s_thr[lane][u] = (uint32_t)T;
    s_t8[lane][u] = T >= kTwo32 ? (uint16_t)256u : (uint16_t)(T >> 24);
  }
  __syncthreads();
  if (!has) return;
  // word offsets within a configuration (bytes), all multiples of 4
  WordOffsets o;
  o.self = L * row + x0;
  o.prev = L * row + (x0 == 0u ? L - 4u : x0 - 4u);
  o.next = L * row + (x0 + 4u == L ? 0u : x0 + 4u);
  o.yp = L * ((y + 1u == L ? 0u : y + 1u) + L * z) + x0;
  o.ym = L * ((y == 0u ? L - 1u : y - 1u) + L * z) + x0;
  o.zp = o.zm = 0u;
  if (D == 3) {
    o.zp = L * (y + L * (z + 1u == L ? 0u : z + 1u)) + x0;
    o.zm = L * (y + L * (z == 0u ? L - 1u : z - 1u)) + x0;
  }
  const uint32_t lanes = min(64u, (uint32_t)p.S - 64u * g);
  const uint32_t sh1 = 8u * b0, sh2 = 8u * (b0 + 2u);
  int8_t* spl = p.spins + ((size_t)sigma * p.S + 64u * g) * N;
  const int8_t* Jl = p.J + (size_t)64u * g * D * N;
  WordLoads<D> cur, nxt;
  load_word<D>(cur, spl, Jl, N, o);
#pragma unroll 1
  for (uint32_t lane = 0; lane < lanes; ++lane) {
    if (lane + 1u < lanes) load_word<D>(nxt, spl + (size_t)(lane + 1u) * N, Jl + (size_t)(lane + 1u) * D * N, N, o);
    // sign bit 7 of each byte: bond unsatisfied
    const uint32_t self = cur.self;
    uint32_t cnt = ((self ^ __funnelshift_r(self, cur.next, 8) ^ cur.j0s) >> 7) & 0x01010101u;  // x + 1
    cnt += ((self ^ __funnelshift_l(cur.prev, self, 8) ^ __funnelshift_l(cur.j0p, cur.j0s, 8)) >> 7) &
           0x01010101u;  // x - 1
    cnt += ((self ^ cur.yp ^ cur.j1s) >> 7) & 0x01010101u;
    cnt += ((self ^ cur.ym ^ cur.j1m) >> 7) & 0x01010101u;
    if (D == 3) {
      cnt += ((self ^ cur.zp ^ cur.j2s) >> 7) & 0x01010101u;
      cnt += ((self ^ cur.zm ^ cur.j2m) >> 7) & 0x01010101u;
    }
    uint32_t flip = 0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint32_t shj = j == 0 ? sh1 : sh2;
      const uint32_t u = (cnt >> shj) & 0xFFu;
      const uint32_t t8 = s_t8[lane][u];
      const uint32_t r8 = s_r8[((uint32_t)j * kWordThreads + t) * kTileRow + lane];
      bool less = r8 < t8;  // decided by the first 8 planes unless equal (then T < 2^32)
      if (r8 == t8)
        less = lazy_less_from(s_thr[lane][u], 4u, p, tk, sigma, g, lane, x0 + b0 + 2u * (uint32_t)j + L * row);
      if (less != (p.inv != 0)) flip |= 0xFEu << shj;  // +1 (0x01) <-> -1 (0xFF)
    }
    if (flip) *reinterpret_cast<uint32_t*>(spl + (size_t)lane * N + o.self) = self ^ flip;
    cur = nxt;
  }
}

// Field models (Eq. 2 with fields h_i = +-|h| and occupations x_i): an empty
// site is skipped; for an occupied one v = s_i sum_j J_ij x_j s_j and
// f = [s_i h_i > 0] select the threshold of class (v + 2D) * 2 + f.
struct FieldI8Params {
  I8Params b;
  const int8_t* hs;    // [S][N]
  const int8_t* occ;   // [S][N]
  const uint64_t* fthr;  // [K][kFieldClasses]
};

template <int D>
__global__ void __launch_bounds__(256) k_sweep_field_i8(const FieldI8Params fp) {
  const I8Params& p = fp.b;
  const uint64_t total = (uint64_t)p.slots * p.S * p.half;
  const uint32_t L = (uint32_t)p.L, h = L / 2u;
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t lat = (uint32_t)(idx / p.half);
    const uint32_t w = (uint32_t)(idx - (uint64_t)lat * p.half);
    const int sigma = (int)(lat / (uint32_t)p.S);
    const int s = (int)(lat - (uint32_t)sigma * (uint32_t)p.S);
    const uint32_t row = w / h, k = w - row * h;
    const uint32_t y = row % L, z = row / L;
    const uint32_t x = 2u * k + ((uint32_t)(p.colour ^ (int)(y + z)) & 1u);
    const uint32_t i = x + L * (y + L * z);
    const int8_t* xo = fp.occ + (size_t)s * p.N;
    if (!xo[i]) continue;
    int8_t* sp = p.spins + (size_t)lat * p.N;
    const int8_t* Jp = p.J + (size_t)s * D * p.N;
    const int si = sp[i];
    const uint32_t xp = (x + 1u == L ? 0u : x + 1u) + L * (y + L * z);
    const uint32_t xm = (x == 0u ? L - 1u : x - 1u) + L * (y + L * z);
    const uint32_t yp = x + L * ((y + 1u == L ? 0u : y + 1u) + L * z);
    const uint32_t ym = x + L * ((y == 0u ? L - 1u : y - 1u) + L * z);
    int phi = Jp[i] * xo[xp] * sp[xp] + Jp[xm] * xo[xm] * sp[xm] + Jp[p.N + i] * xo[yp] * sp[yp] +
              Jp[p.N + ym] * xo[ym] * sp[ym];
    if (D == 3) {
      const uint32_t zp = x + L * (y + L * (z + 1u == L ? 0u : z + 1u));
      const uint32_t zm = x + L * (y + L * (z == 0u ? L - 1u : z - 1u));
      phi += Jp[2u * p.N + i] * xo[zp] * sp[zp] + Jp[2u * p.N + zm] * xo[zm] * sp[zm];
    }
    const int v = si * phi;
    const int f = si * fp.hs[(size_t)s * p.N + i] > 0;
    const int tslot = sigma / p.R, a = sigma - tslot * p.R;
    const int kt = p.temp_of[((size_t)s * p.R + a) * p.K + tslot];
    const uint64_t T = fp.fthr[(size_t)kt * kFieldClasses + (v + 2 * D) * 2 + f];
    const bool less = lazy_less(T, p, tk, s, sigma, i);
    if (less != (p.inv != 0)) sp[i] = (int8_t)(-si);
  }
}

// ---- Parisi-Rapuano wheels (Sec. 3.3, Eq. 5) ----
//
// One thread per (configuration, row) walks the colour-c sites of its row in
// increasing x, drawing R(k) = I(k) ^ I(k-61), I(k) = I(k-24) + I(k-55), from
// the row's wheel; k = t L/2 + j for the j-th site.  The ring of 64 words
// (I(k) at index k mod 64) sits in shared memory for the launch, ring index
// major so that the threads of a warp, which share k, hit 32 banks.
constexpr int kWheelBlock = 128;

struct WheelParams {
  I8Params b;
  uint32_t* wheels;      // [slots * S][2][64][rows]
  uint32_t rows;
  const int8_t* hs;      // field models: [S][N], else null
  const int8_t* occ;
  const uint64_t* fthr;  // field models: [K][kFieldClasses]
};

template <int D, bool FIELD>
__global__ void __launch_bounds__(kWheelBlock) k_sweep_wheel_i8(const WheelParams wp) {
  __shared__ uint32_t ring[64 * kWheelBlock];
  const I8Params& p = wp.b;
  const uint32_t L = (uint32_t)p.L, h = L / 2u, rows = wp.rows;
  const uint64_t total = (uint64_t)p.slots * p.S * rows;
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  const uint32_t k0 = tk.lo * h;  // t L/2 mod 2^32; only k mod 64 is used
  const uint32_t tid = threadIdx.x;
  for (uint64_t base = (uint64_t)blockIdx.x * kWheelBlock; base < total; base += (uint64_t)gridDim.x * kWheelBlock) {
    const uint64_t idx = base + tid;
    const bool active = idx < total;
    const uint32_t lat = active ? (uint32_t)(idx / rows) : 0u;
    const uint32_t row = active ? (uint32_t)(idx - (uint64_t)lat * rows) : 0u;
    uint32_t* wg = wp.wheels + ((size_t)lat * 2 + (size_t)p.colour) * 64 * rows + row;
    if (active)
      for (int m = 0; m < 64; ++m) ring[m * kWheelBlock + tid] = wg[(size_t)m * rows];
    if (active) {
      const int sigma = (int)(lat / (uint32_t)p.S);
      const int s = (int)(lat - (uint32_t)sigma * (uint32_t)p.S);
      const uint32_t y = row % L, z = row / L;  // D = 2: z = 0
      const uint32_t x0 = (uint32_t)(p.colour ^ (int)(y + z)) & 1u;
      int8_t* sp = p.spins + (size_t)lat * p.N;
      const int8_t* Jp = p.J + (size_t)s * D * p.N;
      const int8_t* xo = FIELD ? wp.occ + (size_t)s * p.N : nullptr;
      const int tslot = sigma / p.R, a = sigma - tslot * p.R;
      const int kt = p.temp_of[((size_t)s * p.R + a) * p.K + tslot];
      // rows of the neighbours along y and z
      const uint32_t yp = (y + 1u == L ? 0u : y + 1u) + L * z, ym = (y == 0u ? L - 1u : y - 1u) + L * z;
      const uint32_t zp = y + L * (z + 1u == L ? 0u : z + 1u), zm = y + L * (z == 0u ? L - 1u : z - 1u);
      for (uint32_t j = 0; j < h; ++j) {
        const uint32_t k = k0 + j;
        const uint32_t Ik = ring[((k - 24u) & 63u) * kWheelBlock + tid] + ring[((k - 55u) & 63u) * kWheelBlock + tid];
        const uint32_t r = Ik ^ ring[((k - 61u) & 63u) * kWheelBlock + tid];
        ring[(k & 63u) * kWheelBlock + tid] = Ik;
        const uint32_t x = 2u * j + x0;
        const uint32_t i = x + L * row;
        if (FIELD && !xo[i]) continue;
        const uint32_t xp = (x + 1u == L ? 0u : x + 1u) + L * row;
        const uint32_t xm = (x == 0u ? L - 1u : x - 1u) + L * row;
        const uint32_t iyp = x + L * yp, iym = x + L * ym;
        const int si = sp[i];
        uint64_t T;
        if (FIELD) {
          int phi = Jp[i] * xo[xp] * sp[xp] + Jp[xm] * xo[xm] * sp[xm] + Jp[p.N + i] * xo[iyp] * sp[iyp] +
                    Jp[p.N + iym] * xo[iym] * sp[iym];
          if (D == 3) {
            const uint32_t izp = x + L * zp, izm = x + L * zm;
            phi += Jp[2u * p.N + i] * xo[izp] * sp[izp] + Jp[2u * p.N + izm] * xo[izm] * sp[izm];
          }
          const int v = si * phi;
          const int f = si * wp.hs[(size_t)s * p.N + i] > 0;
          T = wp.fthr[(size_t)kt * kFieldClasses + (v + 2 * D) * 2 + f];
        } else {
          int u = (Jp[i] * si * sp[xp] < 0) + (Jp[xm] * si * sp[xm] < 0) + (Jp[p.N + i] * si * sp[iyp] < 0) +
                  (Jp[p.N + iym] * si * sp[iym] < 0);
          if (D == 3) {
            const uint32_t izp = x + L * zp, izm = x + L * zm;
            u += (Jp[2u * p.N + i] * si * sp[izp] < 0) + (Jp[2u * p.N + izm] * si * sp[izm] < 0);
          }
          T = p.thr[(size_t)kt * kMaxClasses + u];
        }
        const bool less = (uint64_t)r < T;
        if (less != (p.inv != 0)) sp[i] = (int8_t)(-si);
      }
      for (int m = 0; m < 64; ++m) wg[(size_t)m * rows] = ring[m * kWheelBlock + tid];
    }
  }
}

// Starting values: I(-61 + n) = word n of the WHEEL stream of the wheel, at
// ring index (n + 3) mod 64; I(-61) made odd.
__global__ void k_init_wheels(uint32_t* wheels, int S, int slots, uint32_t rows, PhiloxKeys keys) {
  const uint64_t total = (uint64_t)slots * S * 2u * rows;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t row = (uint32_t)(idx % rows);
    const uint64_t rest = idx / rows;
    const uint32_t c = (uint32_t)(rest & 1u), lat = (uint32_t)(rest >> 1);
    const uint32_t sigma = lat / (uint32_t)S, s = lat - sigma * (uint32_t)S;
    uint32_t* w = wheels + ((size_t)lat * 2 + c) * 64 * rows + row;
    for (uint32_t blk = 0; blk < 16u; ++blk) {
      const uint4 x = philox10(row, s, (TAG_WHEEL << 28) | (blk << 24) | (sigma << 12) | c, 0u, keys);
      const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
      for (uint32_t e = 0; e < 4u; ++e) {
        const uint32_t n = 4u * blk + e;
        if (n < 61u) w[(size_t)((n + 3u) & 63u) * rows] = n == 0u ? (xs[e] | 1u) : xs[e];
      }
    }
    for (uint32_t m = 0; m < 3u; ++m) w[(size_t)m * rows] = 0u;
  }
}

// ---- resident mode: a whole configuration in shared memory ----
//
// One block per configuration (n_temps == 1) keeps the spins and the
// couplings in shared memory and runs many sweeps in one launch, with a block
// barrier between the two colours (Sec. 3.1) instead of a kernel boundary,
// and records E and M into the series ring after every measured sweep.  The
// per-site update is the one of k_sweep_i8.

struct ResidentParams {
  int8_t* spins;            // [slots][S][N]
  const int8_t* J;          // [S][D][N]
  const uint64_t* thr;      // [1][kMaxClasses]
  int S, R, slots, L, inv;
  uint32_t N, half;
  uint64_t t0;              // absolute index of the first sweep
  uint32_t nsweeps;
  uint32_t measure_every;   // 0 = none
  uint64_t row0;            // series rows recorded before this launch
  uint32_t cap;             // series capacity
  int64_t* ser_E;           // [cap][S*R]
  int64_t* ser_M;
  uint64_t* ser_sweep;      // [cap]
  PhiloxKeys keys;
};

template <int D>
__global__ void __launch_bounds__(1024) k_resident_i8(const ResidentParams p) {
  extern __shared__ int8_t sm[];  // spins[N], then J[D][N]
  __shared__ long long red[2][32];
  int8_t* sp = sm;
  int8_t* Js = sm + p.N;
  const uint32_t lat = blockIdx.x;  // sigma * S + s
  const int sigma = (int)(lat / (uint32_t)p.S), s = (int)(lat - (uint32_t)sigma * (uint32_t)p.S);
  int8_t* gsp = p.spins + (size_t)lat * p.N;
  const int8_t* gJ = p.J + (size_t)s * D * p.N;
  for (uint32_t i = threadIdx.x; i < p.N; i += blockDim.x) sp[i] = gsp[i];
  for (uint32_t i = threadIdx.x; i < (uint32_t)D * p.N; i += blockDim.x) Js[i] = gJ[i];
  __syncthreads();
  const uint32_t L = (uint32_t)p.L, h = L / 2u;
  I8Params q;  // the fields lazy_less reads
  q.keys = p.keys;
  uint32_t nmeas = 0;
  for (uint32_t it = 0; it < p.nsweeps; ++it) {
    const uint64_t t = p.t0 + it;
    const Tick tk{(uint32_t)t, (uint32_t)(t >> 32)};
    for (int colour = 0; colour < 2; ++colour) {
      for (uint32_t w = threadIdx.x; w < p.half; w += blockDim.x) {
        const uint32_t row = w / h, k = w - row * h;
        const uint32_t y = row % L, z = row / L;
        const uint32_t x = 2u * k + ((uint32_t)(colour ^ (int)(y + z)) & 1u);
        const uint32_t i = x + L * (y + L * z);
        const int si = sp[i];
        const uint32_t xp = (x + 1u == L ? 0u : x + 1u) + L * (y + L * z);
        const uint32_t xm = (x == 0u ? L - 1u : x - 1u) + L * (y + L * z);
        const uint32_t yp = x + L * ((y + 1u == L ? 0u : y + 1u) + L * z);
        const uint32_t ym = x + L * ((y == 0u ? L - 1u : y - 1u) + L * z);
        int u = 0;
        u += (Js[i] * si * sp[xp]) < 0;
        u += (Js[xm] * si * sp[xm]) < 0;
        u += (Js[p.N + i] * si * sp[yp]) < 0;
        u += (Js[p.N + ym] * si * sp[ym]) < 0;
        if (D == 3) {
          const uint32_t zp = x + L * (y + L * (z + 1u == L ? 0u : z + 1u));
          const uint32_t zm = x + L * (y + L * (z == 0u ? L - 1u : z - 1u));
          u += (Js[2u * p.N + i] * si * sp[zp]) < 0;
          u += (Js[2u * p.N + zm] * si * sp[zm]) < 0;
        }
        const bool less = lazy_less(p.thr[u], q, tk, s, sigma, i);
        if (less != (p.inv != 0)) sp[i] = (int8_t)(-si);
      }
      __syncthreads();
    }
    if (p.measure_every && (t + 1) % p.measure_every == 0) {
      long long e = 0, m = 0;
      for (uint32_t i = threadIdx.x; i < p.N; i += blockDim.x) {
        const uint32_t x = i % L, y = (i / L) % L, z = D == 3 ? i / (L * L) : 0u;
        const int si = sp[i];
        e -= Js[i] * si * sp[(x + 1u == L ? 0u : x + 1u) + L * (y + L * z)];
        e -= Js[p.N + i] * si * sp[x + L * ((y + 1u == L ? 0u : y + 1u) + L * z)];
        if (D == 3) e -= Js[2u * p.N + i] * si * sp[x + L * (y + L * (z + 1u == L ? 0u : z + 1u))];
        m += si;
      }
      for (int off = 16; off > 0; off >>= 1) {
        e += __shfl_down_sync(0xffffffffu, e, off);
        m += __shfl_down_sync(0xffffffffu, m, off);
      }
      if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = e;
        red[1][threadIdx.x >> 5] = m;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        long long E = 0, M = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
          E += red[0][w];
          M += red[1][w];
        }
        const uint64_t row = (p.row0 + nmeas) % p.cap;
        const size_t at = (size_t)row * p.S * p.R + (size_t)s * p.R + (size_t)sigma;  // one temperature: slot = replica
        p.ser_E[at] = E;
        p.ser_M[at] = M;
        if (lat == 0) p.ser_sweep[row] = t + 1;
      }
      __syncthreads();
      ++nmeas;
    }
  }
  for (uint32_t i = threadIdx.x; i < p.N; i += blockDim.x) gsp[i] = sp[i];
}

// ---- cluster-resident mode: one configuration across a thread-block cluster ----
//
// When there are few configurations, one block each leaves most SMs idle and
// every colour pass is as long as the slowest of a block's many sites.  Here
// a cluster of C blocks (C divides L) holds one configuration: block r owns
// the slab of P = L/C planes along the last axis (z in 3D, y in 2D), its
// spins and forward couplings in shared memory, the plane of last-axis
// couplings just below the slab, and halo copies of the neighbouring blocks'
// face planes.  A flip on a face is also stored into the neighbour's halo
// (distributed shared memory), so every read is local, and the two colours
// are separated by cluster barriers (Sec. 3.1) whose release/acquire makes
// those stores visible.  The random stream and the update rule are those of
// k_sweep_i8, so the results are the same bit for bit.  E and M are measured
// once per launch and then carried by the flips; per-block changes are
// summed in block 0's shared memory at each measured sweep.

// Sum of (e, m) over the block, valid in thread 0; red holds one pair per warp.
__device__ __forceinline__ void block_sum2(long long (*red)[32], long long e, long long m, long long& E,
                                           long long& M) {
  for (int off = 16; off > 0; off >>= 1) {
    e += __shfl_down_sync(0xffffffffu, e, off);
    m += __shfl_down_sync(0xffffffffu, m, off);
  }
  __syncthreads();  // red may still be read from the previous sum
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = e;
    red[1][threadIdx.x >> 5] = m;
  }
  __syncthreads();
  E = M = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) {
      E += red[0][w];
      M += red[1][w];
    }
}

// The first eight planes of a site's random number (plane 0 in bit 7), from
// four Philox blocks computed together: they do not depend on the spins, so
// a block draws them for its next pass while it waits at the cluster barrier.
__device__ __forceinline__ uint32_t first_planes(const PhiloxKeys& keys, const Tick& tk, int s, int sigma,
                                                 uint32_t site) {
  const uint32_t lane = (uint32_t)s & 63u, g = (uint32_t)s >> 6;
  const uint32_t c2base = (TAG_SPIN << 28) | ((uint32_t)sigma << 12) | g;
  uint4 x[4];
#pragma unroll
  for (uint32_t m = 0; m < 4u; ++m) x[m] = philox10(site, tk.lo, c2base | (m << 24), tk.hi, keys);
  uint32_t r8 = 0;
#pragma unroll
  for (uint32_t m = 0; m < 4u; ++m) {
    const uint32_t w0 = lane < 32u ? (x[m].x >> lane) : (x[m].y >> (lane - 32u));
    const uint32_t w1 = lane < 32u ? (x[m].z >> lane) : (x[m].w >> (lane - 32u));
    r8 |= ((w0 & 1u) << (7u - 2u * m)) | ((w1 & 1u) << (6u - 2u * m));
  }
  return r8;
}

// r < T (as lazy_less) given the first eight planes r8; planes 8.. drawn
// one Philox block at a time when those agree with T.
__device__ __forceinline__ bool less_from(uint64_t T, uint32_t r8, const PhiloxKeys& keys, const Tick& tk, int s,
                                          int sigma, uint32_t site) {
  if (T >= kTwo32) return true;
  const uint32_t T32 = (uint32_t)T;
  const uint32_t t8 = T32 >> 24;
  if (r8 != t8) return r8 < t8;
  const uint32_t lane = (uint32_t)s & 63u, g = (uint32_t)s >> 6;
  const uint32_t c2base = (TAG_SPIN << 28) | ((uint32_t)sigma << 12) | g;
#pragma unroll 1
  for (uint32_t m = 4; m < 16u; ++m) {
    const uint4 y = philox10(site, tk.lo, c2base | (m << 24), tk.hi, keys);
    const uint32_t w0 = lane < 32u ? (y.x >> lane) : (y.y >> (lane - 32u));
    const uint32_t w1 = lane < 32u ? (y.z >> lane) : (y.w >> (lane - 32u));
    const uint32_t r0 = w0 & 1u, t0 = (T32 >> (31u - 2u * m)) & 1u;
    if (r0 != t0) return r0 < t0;
    const uint32_t r1 = w1 & 1u, t1 = (T32 >> (30u - 2u * m)) & 1u;
    if (r1 != t1) return r1 < t1;
  }
  return false;  // r == T
}

// Split cluster barrier: arrive (release: this block's shared-memory writes
// become visible) and wait (acquire).  Not the .aligned forms, so that they
// need no warp convergence.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory"); }

constexpr unsigned kClusterBlockMax = 512;  // threads per block of the cluster-resident kernel

// Sum of (e, m) over the block into thread 0 (64-bit), from 32-bit thread
// values: one warp reduction each, one word per warp in red.  The caller
// makes sure red is not still being read from an earlier sum.
__device__ __forceinline__ void block_sum2_i32(int (*red)[32], int e, int m, long long& E, long long& M) {
  e = __reduce_add_sync(0xffffffffu, e);
  m = __reduce_add_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = e;
    red[1][threadIdx.x >> 5] = m;
  }
  __syncthreads();
  E = M = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) {
      E += red[0][w];
      M += red[1][w];
    }
}

// E and M of a block's slab (forward bonds of its own sites; the plane above
// the slab from the halo), summed over the block by thread 0.
template <int D>
__device__ __forceinline__ void slab_energy(const int8_t* sp, const int8_t* Js, const int8_t* halo_up, uint32_t L,
                                            uint32_t A, uint32_t P, long long (*red)[32], long long& E,
                                            long long& M) {
  const uint32_t PA = P * A;
  long long e = 0, m = 0;
  for (uint32_t j = threadIdx.x; j < PA; j += blockDim.x) {
    const uint32_t zl = j / A, ip = j - zl * A;
    const uint32_t x = ip % L;
    const int si = sp[j];
    e -= Js[j] * si * sp[j - x + (x + 1u == L ? 0u : x + 1u)];
    if (D == 3) {
      const uint32_t y = ip / L;
      e -= Js[PA + j] * si * sp[j - L * y + L * (y + 1u == L ? 0u : y + 1u)];
    }
    const int8_t s_up = zl + 1u < P ? sp[j + A] : halo_up[ip];
    e -= Js[(D - 1) * PA + j] * si * s_up;
    m += si;
  }
  block_sum2(red, e, m, E, M);
}

// One colour-c site of a slab: where it is, where its 2D neighbours are (in
// this block's slab or halo planes), its 2D coupling values, and the halo
// cells of the neighbouring blocks that mirror it (null when it is inside
// the slab).
template <int D>
struct SlabSite {
  uint32_t j, i;            // slab index, natural site index
  uint32_t n[2 * D - 2];    // in-slab neighbours (x+, x-, y+, y-)
  const int8_t* up;         // last axis +1
  const int8_t* dn;         // last axis -1
  int8_t* mirror_prev;      // the previous block's upper halo cell (bottom plane)
  int8_t* mirror_next;      // the next block's lower halo cell (top plane)
  int8_t J[2 * D];          // couplings in the order x+, x-, (y+, y-,) up, dn
};

// Shared memory of one block: spins[P*A], J[D][P*A], the plane of last-axis
// couplings below the slab, and the halos: copies of the next block's bottom
// plane (up) and of the previous block's top plane (dn), kept current by
// their owners' stores.
struct SlabMem {
  int8_t *sp, *Js, *Jh, *halo_up, *halo_dn;
  int8_t *prev_halo_up, *next_halo_dn;  // in the neighbouring blocks
};

template <int D>
__device__ __forceinline__ SlabSite<D> slab_site(uint32_t w, int colour, uint32_t L, uint32_t A, uint32_t P,
                                                 uint32_t z0, const SlabMem& sm) {
  const uint32_t h = L / 2u, PA = P * A;
  const uint32_t row = w / h, k = w - row * h;  // local row of the slab
  uint32_t y, z, zl;
  if (D == 3) {
    y = row % L;
    zl = row / L;
    z = z0 + zl;
  } else {
    zl = row;
    y = z0 + zl;
    z = 0;
  }
  const uint32_t x = 2u * k + ((uint32_t)(colour ^ (int)(y + z)) & 1u);
  const uint32_t ip = D == 3 ? x + L * y : x;  // index within the plane
  SlabSite<D> q;
  q.j = ip + A * zl;
  q.i = ip + A * (z0 + zl);
  const uint32_t xm = q.j - x + (x == 0u ? L - 1u : x - 1u);
  q.n[0] = q.j - x + (x + 1u == L ? 0u : x + 1u);
  q.n[1] = xm;
  q.J[0] = sm.Js[q.j];
  q.J[1] = sm.Js[xm];
  if constexpr (D == 3) {
    const uint32_t ym = (y == 0u ? L - 1u : y - 1u) * L + x + A * zl;
    q.n[2] = (y + 1u == L ? 0u : y + 1u) * L + x + A * zl;
    q.n[3] = ym;
    q.J[2] = sm.Js[PA + q.j];
    q.J[3] = sm.Js[PA + ym];
  }
  q.up = zl + 1u < P ? sm.sp + q.j + A : sm.halo_up + ip;
  q.dn = zl > 0u ? sm.sp + q.j - A : sm.halo_dn + ip;
  q.mirror_prev = zl == 0u ? sm.prev_halo_up + ip : nullptr;
  q.mirror_next = zl + 1u == P ? sm.next_halo_dn + ip : nullptr;
  q.J[2 * D - 2] = sm.Js[(D - 1) * PA + q.j];
  q.J[2 * D - 1] = zl > 0u ? sm.Js[(D - 1) * PA + q.j - A] : sm.Jh[ip];
  return q;
}

// One site's update: unsatisfied bonds (J s_i s_j < 0), the decision, and on
// a flip the new spin in the slab and in the neighbours' halos, with the
// changes of E and M.
template <int D>
__device__ __forceinline__ void slab_update(const SlabSite<D>& q, int8_t* sp, const uint64_t* thr, uint32_t r8,
                                            const PhiloxKeys& keys, const Tick& tk, int s, int sigma, int inv,
                                            int& dE, int& dM) {
  const int si = sp[q.j];
  int u = 0;
#pragma unroll
  for (int b = 0; b < 2 * D - 2; ++b) u += (q.J[b] * si * sp[q.n[b]]) < 0;
  u += (q.J[2 * D - 2] * si * *q.up) < 0;
  u += (q.J[2 * D - 1] * si * *q.dn) < 0;
  const uint64_t T = thr[u];
  if (T < kTwo32 && r8 == 0xFFFFFFFFu) r8 = first_planes(keys, tk, s, sigma, q.i);
  if (less_from(T, r8, keys, tk, s, sigma, q.i) != (inv != 0)) {
    const int8_t ns = (int8_t)(-si);
    sp[q.j] = ns;
    if (q.mirror_prev) *q.mirror_prev = ns;
    if (q.mirror_next) *q.mirror_next = ns;
    dE += 4 * D - 4 * u;
    dM -= 2 * si;
  }
}

// ONE: every block has at most one site of each colour per thread; the
// sites' neighbourhoods are then worked out once per launch and the first
// eight random planes of the next pass are drawn during each barrier wait.
// E and M are measured once at the start of a launch and then carried by the
// flips: a flip of a site with u unsatisfied bonds changes E by 4D - 4u and
// M by -2 s_i.  A launch runs at most 65536 sweeps, so a thread's changes
// between two measurements fit 32 bits.
template <int D, bool ONE>
__global__ void __launch_bounds__(kClusterBlockMax) k_resident_cluster_i8(const ResidentParams p, int C) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ int8_t smem[];
  __shared__ long long red[2][32];
  __shared__ int red32[2][32];
  __shared__ long long part[2][16];  // per-block sums, read in block 0
  __shared__ uint64_t thr_s[kMaxClasses];
  const uint32_t L = (uint32_t)p.L;
  const uint32_t A = D == 3 ? L * L : L;  // sites per plane of the last axis
  const uint32_t P = L / (uint32_t)C;     // planes per block
  const uint32_t PA = P * A;
  const uint32_t rank = cl.block_rank();
  const uint32_t prev = (rank + (uint32_t)C - 1u) % (uint32_t)C, next = (rank + 1u) % (uint32_t)C;
  const uint32_t z0 = rank * P;  // first plane of this block's slab
  SlabMem sm;
  sm.sp = smem;
  sm.Js = smem + PA;
  sm.Jh = sm.Js + (size_t)D * PA;
  sm.halo_up = sm.Jh + A;
  sm.halo_dn = sm.halo_up + A;
  sm.prev_halo_up = cl.map_shared_rank(sm.halo_up, prev);
  sm.next_halo_dn = cl.map_shared_rank(sm.halo_dn, next);
  int8_t* sp = sm.sp;
  const uint32_t lat = blockIdx.x / (uint32_t)C;  // sigma * S + s
  const int sigma = (int)(lat / (uint32_t)p.S), s = (int)(lat - (uint32_t)sigma * (uint32_t)p.S);
  int8_t* gsp = p.spins + (size_t)lat * p.N + (size_t)z0 * A;
  const int8_t* gJ = p.J + (size_t)s * D * p.N;
  cl.sync();  // every block of the cluster running before any store into another's shared memory
  for (uint32_t j = threadIdx.x; j < PA; j += blockDim.x) {
    const int8_t v = gsp[j];
    sp[j] = v;
    if (j < A) sm.prev_halo_up[j] = v;                  // bottom plane
    if (j >= PA - A) sm.next_halo_dn[j - (PA - A)] = v;  // top plane
  }
  for (uint32_t d = 0; d < (uint32_t)D; ++d)
    for (uint32_t j = threadIdx.x; j < PA; j += blockDim.x) sm.Js[d * PA + j] = gJ[(size_t)d * p.N + z0 * A + j];
  const uint32_t zb = (z0 + L - 1u) % L;  // plane below the slab
  for (uint32_t j = threadIdx.x; j < A; j += blockDim.x) sm.Jh[j] = gJ[(size_t)(D - 1) * p.N + zb * A + j];
  if (threadIdx.x < (unsigned)kMaxClasses) thr_s[threadIdx.x] = p.thr[threadIdx.x];
  long long* part0 = cl.map_shared_rank(&part[0][0], 0u);
  const uint32_t nw = PA / 2u;  // sites of one colour in the slab
  const bool mine = threadIdx.x < nw;
  __syncthreads();  // couplings staged before the sites read them
  SlabSite<D> site[2];
  uint32_t r8 = 0;  // first planes of this thread's site in the next pass
  if (ONE && mine) {
    site[0] = slab_site<D>(threadIdx.x, 0, L, A, P, z0, sm);
    site[1] = slab_site<D>(threadIdx.x, 1, L, A, P, z0, sm);
  }
  cluster_arrive();
  if (ONE && mine && p.nsweeps > 0)
    r8 = first_planes(p.keys, Tick{(uint32_t)p.t0, (uint32_t)(p.t0 >> 32)}, s, sigma, site[0].i);
  cluster_wait();  // slabs and halos loaded
  long long E_run = 0, M_run = 0;  // block 0, thread 0
  if (p.measure_every) {
    long long E, M;
    slab_energy<D>(sp, sm.Js, sm.halo_up, L, A, P, red, E, M);
    if (threadIdx.x == 0) {
      part0[rank] = E;
      part0[16 + rank] = M;
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0)
      for (int r = 0; r < C; ++r) {
        E_run += part[0][r];
        M_run += part[1][r];
      }
  }
  int dE = 0, dM = 0;  // this thread's flips since the last measurement
  uint64_t row = p.cap ? p.row0 % p.cap : 0;  // series row of the next measurement
  // sweeps until the next measured one: sweep t is measured when (t + 1) % every == 0
  uint32_t left = p.measure_every ? (uint32_t)(p.measure_every - p.t0 % p.measure_every) : 0u;
  for (uint32_t it = 0; it < p.nsweeps; ++it) {
    const uint64_t t = p.t0 + it;
    const Tick tk{(uint32_t)t, (uint32_t)(t >> 32)};
    const bool measured = left == 1u;
    if (p.measure_every) left = measured ? p.measure_every : left - 1u;
#pragma unroll
    for (int colour = 0; colour < 2; ++colour) {
      if (ONE) {
        if (mine) slab_update<D>(site[colour], sp, thr_s, r8, p.keys, tk, s, sigma, p.inv, dE, dM);
      } else {
        for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x)
          slab_update<D>(slab_site<D>(w, colour, L, A, P, z0, sm), sp, thr_s, 0xFFFFFFFFu, p.keys, tk, s, sigma,
                         p.inv, dE, dM);
      }
      if (colour == 1 && measured) {  // this sweep's changes, into block 0 before the barrier
        long long bE, bM;
        block_sum2_i32(red32, dE, dM, bE, bM);
        dE = dM = 0;
        if (threadIdx.x == 0) {
          part0[rank] = bE;
          part0[16 + rank] = bM;
        }
      }
      cluster_arrive();
      if (ONE && mine) {  // the next pass: the other colour, or colour 0 of the next sweep
        if (colour == 0)
          r8 = first_planes(p.keys, tk, s, sigma, site[1].i);
        else if (it + 1 < p.nsweeps)
          r8 = first_planes(p.keys, Tick{(uint32_t)(t + 1), (uint32_t)((t + 1) >> 32)}, s, sigma, site[0].i);
      }
      cluster_wait();
    }
    if (measured) {
      if (rank == 0 && threadIdx.x == 0) {
        for (int r = 0; r < C; ++r) {
          E_run += part[0][r];
          M_run += part[1][r];
        }
        const size_t at = (size_t)row * p.S * p.R + (size_t)s * p.R + (size_t)sigma;  // one temperature
        p.ser_E[at] = E_run;
        p.ser_M[at] = M_run;
        if (lat == 0) p.ser_sweep[row] = t + 1;
      }
      row = row + 1u == p.cap ? 0u : row + 1u;
    }
  }
  for (uint32_t j = threadIdx.x; j < PA; j += blockDim.x) gsp[j] = sp[j];
  cl.sync();  // no block leaves while another may still write into its shared memory
}

struct InitParams {
  int8_t* spins;
  int8_t* J;
  int S, D, slots;
  uint32_t N;
  int jmode;  // 0 = J stream, 1 = every J = +1, 2 = every J = -1
  PhiloxKeys keys;
};

__device__ __forceinline__ uint32_t lane_bit(const uint4& x, uint32_t lane) {
  return (lane < 32u ? (x.x >> lane) : (x.y >> (lane - 32u))) & 1u;
}

__global__ void k_init_i8(const InitParams p) {
  const uint64_t total = (uint64_t)p.S * p.N;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = (uint32_t)(idx / p.N), i = (uint32_t)(idx - (uint64_t)s * p.N);
    const uint32_t g = s >> 6, lane = s & 63u;
    for (int d = 0; d < p.D; ++d) {
      const uint4 x = philox10(i, (uint32_t)d, (TAG_J << 28) | g, 0u, p.keys);
      p.J[((size_t)s * p.D + d) * p.N + i] = p.jmode == 2 ? -1 : ((p.jmode == 1 || !lane_bit(x, lane)) ? 1 : -1);
    }
    for (int sg = 0; sg < p.slots; ++sg) {
      const uint4 x = philox10(i, 0u, (TAG_INIT << 28) | ((uint32_t)sg << 12) | g, 0u, p.keys);
      p.spins[((size_t)sg * p.S + s) * p.N + i] = lane_bit(x, lane) ? -1 : 1;
    }
  }
}

// Site disorder: sign of h_i from the H stream (RFIM) and x_i = [r_x < T_occ]
// with r_x assembled from the 32 bit-planes of the X stream (DAFF).
__global__ void k_init_sites_i8(int8_t* hs, int8_t* occ, int S, uint32_t N, int rfim, int daff, uint64_t T_occ,
                                PhiloxKeys keys) {
  const uint64_t total = (uint64_t)S * N;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = (uint32_t)(idx / N), i = (uint32_t)(idx - (uint64_t)s * N);
    const uint32_t g = s >> 6, lane = s & 63u;
    int8_t h = 1, xo = 1;
    if (rfim) {
      const uint4 x = philox10(i, 0u, (TAG_H << 28) | g, 0u, keys);
      h = lane_bit(x, lane) ? -1 : 1;
    }
    if (daff) {
      uint32_t r = 0;
      for (uint32_t m = 0; m < 16u; ++m) {
        const uint4 x = philox10(i, 0u, (TAG_X << 28) | (m << 24) | g, 0u, keys);
        const uint32_t b0 = lane_bit(x, lane);
        const uint32_t b1 = (lane < 32u ? (x.z >> lane) : (x.w >> (lane - 32u))) & 1u;
        r |= (b0 << (31u - 2u * m)) | (b1 << (30u - 2u * m));
      }
      xo = (uint64_t)r < T_occ ? 1 : 0;
    }
    hs[idx] = h;
    occ[idx] = xo;
  }
}

// Field models, block per configuration: E_J = -sum_bonds J x x s s,
// M = sum x s, F = sum sign(h) x s (Sec. 4.1 observables of Eq. 2).
template <int D>
__global__ void __launch_bounds__(256) k_measure_field_i8(const int8_t* __restrict__ spins,
                                                          const int8_t* __restrict__ J,
                                                          const int8_t* __restrict__ hs,
                                                          const int8_t* __restrict__ occ, int64_t* acc, int S,
                                                          int slots, int L, uint32_t N) {
  __shared__ long long red[3][8];
  for (uint32_t lat = blockIdx.x; lat < (uint32_t)(slots * S); lat += gridDim.x) {
    const int sigma = (int)(lat / (uint32_t)S), s = (int)(lat - (uint32_t)sigma * S);
    const int8_t* sp = spins + (size_t)lat * N;
    const int8_t* Jp = J + (size_t)s * D * N;
    const int8_t* xo = occ + (size_t)s * N;
    const int8_t* hp = hs + (size_t)s * N;
    long long e = 0, m = 0, f = 0;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
      const uint32_t x = i % (uint32_t)L, y = (i / (uint32_t)L) % (uint32_t)L;
      const uint32_t z = D == 3 ? i / ((uint32_t)L * (uint32_t)L) : 0u;
      const int si = xo[i] * sp[i];
      const uint32_t xp = (x + 1u == (uint32_t)L ? 0u : x + 1u) + (uint32_t)L * (y + (uint32_t)L * z);
      const uint32_t yp = x + (uint32_t)L * ((y + 1u == (uint32_t)L ? 0u : y + 1u) + (uint32_t)L * z);
      e -= Jp[i] * si * xo[xp] * sp[xp];
      e -= Jp[N + i] * si * xo[yp] * sp[yp];
      if (D == 3) {
        const uint32_t zp = x + (uint32_t)L * (y + (uint32_t)L * (z + 1u == (uint32_t)L ? 0u : z + 1u));
        e -= Jp[2u * N + i] * si * xo[zp] * sp[zp];
      }
      m += si;
      f += hp[i] * si;
    }
    for (int off = 16; off > 0; off >>= 1) {
      e += __shfl_down_sync(0xffffffffu, e, off);
      m += __shfl_down_sync(0xffffffffu, m, off);
      f += __shfl_down_sync(0xffffffffu, f, off);
    }
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      red[0][wid] = e;
      red[1][wid] = m;
      red[2][wid] = f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long E = 0, M = 0, F = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        E += red[0][w];
        M += red[1][w];
        F += red[2][w];
      }
      int64_t* a = acc + ((size_t)s * slots + sigma) * kAccStride;
      a[0] = E;
      a[1] = M;
      a[2] = F;
    }
    __syncthreads();
  }
}

// One temperature, R = 1 or 2 replicas, L a multiple of 16: block per
// sample, E and M of each replica and (R = 2) the overlap Q of the two
// (Sec. 4.1) in one pass that reads the sample's couplings once.  16 sites
// of a row per step: a bond (i, j) is unsatisfied iff the sign bits (bit 7)
// of s_i, J_ij and s_j XOR to 1, so E = 2 U - D N, M = N - 2 n_- and
// Q = N - 2 n_differ, with U, n_- and n_differ counted by popcounts of
// sign-bit masks.
template <int D, int R>
__global__ void __launch_bounds__(256) k_measure_i8_k1(const int8_t* __restrict__ spins,
                                                       const int8_t* __restrict__ J, int64_t* acc, int S, int L,
                                                       uint32_t N, int want_q) {
  __shared__ long long red[2 * R + 1][8];
  const uint32_t qrow = (uint32_t)L / 16u, nq = N / 16u, uL = (uint32_t)L;
  for (uint32_t s = blockIdx.x; s < (uint32_t)S; s += gridDim.x) {
    const int8_t* Jp = J + (size_t)s * D * N;
    uint32_t un[R], ng[R], df = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) un[r] = ng[r] = 0;
    for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
      const uint32_t row = q / qrow, k = q - row * qrow;
      const uint32_t y = row % uL, z = row / uL;
      const uint32_t base = row * uL + 16u * k;
      const uint32_t nxo = row * uL + (k + 1u == qrow ? 0u : 16u * (k + 1u));
      const uint32_t yb = ((D == 3 ? z * uL : 0u) + (y + 1u == uL ? 0u : y + 1u)) * uL + 16u * k;
      const uint32_t zb = D == 3 ? ((z + 1u == uL ? 0u : z + 1u) * uL + y) * uL + 16u * k : 0u;
      const uint4 jx = __ldg(reinterpret_cast<const uint4*>(Jp + base));
      const uint4 jy = __ldg(reinterpret_cast<const uint4*>(Jp + N + base));
      uint4 jz = make_uint4(0u, 0u, 0u, 0u);
      if (D == 3) jz = __ldg(reinterpret_cast<const uint4*>(Jp + 2u * N + base));
      const uint32_t jxs[4] = {jx.x, jx.y, jx.z, jx.w}, jys[4] = {jy.x, jy.y, jy.z, jy.w};
      const uint32_t jzs[4] = {jz.x, jz.y, jz.z, jz.w};
      uint32_t w0[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int8_t* sp = spins + ((size_t)r * S + s) * N;  // slot r = replica r at the one temperature
        const uint4 w = *reinterpret_cast<const uint4*>(sp + base);
        const uint32_t nx = *reinterpret_cast<const uint32_t*>(sp + nxo);
        const uint4 wy = *reinterpret_cast<const uint4*>(sp + yb);
        uint4 wz = make_uint4(0u, 0u, 0u, 0u);
        if (D == 3) wz = *reinterpret_cast<const uint4*>(sp + zb);
        const uint32_t ws[5] = {w.x, w.y, w.z, w.w, nx};
        const uint32_t ys[4] = {wy.x, wy.y, wy.z, wy.w}, zs[4] = {wz.x, wz.y, wz.z, wz.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const uint32_t right = __funnelshift_r(ws[t], ws[t + 1], 8);  // byte j: the site at x + 1
          un[r] += __popc((ws[t] ^ right ^ jxs[t]) & 0x80808080u) + __popc((ws[t] ^ ys[t] ^ jys[t]) & 0x80808080u);
          if (D == 3) un[r] += __popc((ws[t] ^ zs[t] ^ jzs[t]) & 0x80808080u);
          ng[r] += __popc(ws[t] & 0x80808080u);
          if (R == 2) {
            if (r == 0) w0[t] = ws[t];
            else df += __popc((w0[t] ^ ws[t]) & 0x80808080u);
          }
        }
      }
    }
    long long v[2 * R + 1];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      v[2 * r] = un[r];
      v[2 * r + 1] = ng[r];
    }
    v[2 * R] = df;
#pragma unroll
    for (int i = 0; i < 2 * R + 1; ++i)
      for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
      for (int i = 0; i < 2 * R + 1; ++i) red[i][wid] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
      long long t[2 * R + 1];
      for (int i = 0; i < 2 * R + 1; ++i) {
        t[i] = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t[i] += red[i][w];
      }
      for (int r = 0; r < R; ++r) {
        int64_t* a = acc + ((size_t)s * R + r) * kAccStride;
        a[0] = 2ll * t[2 * r] - (long long)D * N;
        a[1] = (long long)N - 2ll * t[2 * r + 1];
      }
      if (R == 2 && want_q) acc[(size_t)s * R * kAccStride + 6] = (long long)N - 2ll * t[2 * R];
    }
    __syncthreads();
  }
}

// Block per configuration: E = -sum_bonds J s s and M = sum s (Sec. 4.1).
template <int D>
__global__ void __launch_bounds__(256) k_measure_i8(const int8_t* __restrict__ spins,
                                                    const int8_t* __restrict__ J, int64_t* acc, int S,
                                                    int R, int slots, int L, uint32_t N) {
  __shared__ long long red[3][8];
  for (uint32_t lat = blockIdx.x; lat < (uint32_t)(slots * S); lat += gridDim.x) {
    const int sigma = (int)(lat / (uint32_t)S), s = (int)(lat - (uint32_t)sigma * S);
    const int8_t* sp = spins + (size_t)lat * N;
    const int8_t* Jp = J + (size_t)s * D * N;
    long long e = 0, m = 0;
    if ((L & 15) == 0) {
      // 16 sites of a row per step: the sign bit of a +-1 byte is bit 7, a
      // bond (i, j) is unsatisfied iff s_i J_ij s_j = -1, i.e. the three
      // sign bits XOR to 1, so E = 2 U - D N and M = N - 2 n_-, with U and
      // n_- counted by popcounts of sign-bit masks
      const uint32_t qrow = (uint32_t)L / 16u, nq = N / 16u;
      uint32_t un = 0, ng = 0;
      for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
        const uint32_t row = q / qrow, k = q - row * qrow;
        const uint32_t y = row % (uint32_t)L, z = row / (uint32_t)L;
        const uint32_t base = row * (uint32_t)L + 16u * k;
        const uint4 w = *reinterpret_cast<const uint4*>(sp + base);
        const uint32_t nx = *reinterpret_cast<const uint32_t*>(sp + row * (uint32_t)L + (k + 1u == qrow ? 0u : 16u * (k + 1u)));
        const uint32_t yb = ((D == 3 ? z * (uint32_t)L : 0u) + (y + 1u == (uint32_t)L ? 0u : y + 1u)) * (uint32_t)L + 16u * k;
        const uint4 wy = *reinterpret_cast<const uint4*>(sp + yb);
        const uint4 jx = __ldg(reinterpret_cast<const uint4*>(Jp + base));
        const uint4 jy = __ldg(reinterpret_cast<const uint4*>(Jp + N + base));
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w}, wn[5] = {w.x, w.y, w.z, w.w, nx};
        const uint32_t ys[4] = {wy.x, wy.y, wy.z, wy.w}, jxs[4] = {jx.x, jx.y, jx.z, jx.w}, jys[4] = {jy.x, jy.y, jy.z, jy.w};
        uint32_t zs[4] = {0u, 0u, 0u, 0u}, jzs[4] = {0u, 0u, 0u, 0u};
        if (D == 3) {
          const uint32_t zb = ((z + 1u == (uint32_t)L ? 0u : z + 1u) * (uint32_t)L + y) * (uint32_t)L + 16u * k;
          const uint4 wz = *reinterpret_cast<const uint4*>(sp + zb);
          const uint4 jz = __ldg(reinterpret_cast<const uint4*>(Jp + 2u * N + base));
          zs[0] = wz.x; zs[1] = wz.y; zs[2] = wz.z; zs[3] = wz.w;
          jzs[0] = jz.x; jzs[1] = jz.y; jzs[2] = jz.z; jzs[3] = jz.w;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const uint32_t right = __funnelshift_r(wn[t], wn[t + 1], 8);  // byte j: the site at x + 1
          un += __popc((ws[t] ^ right ^ jxs[t]) & 0x80808080u);
          un += __popc((ws[t] ^ ys[t] ^ jys[t]) & 0x80808080u);
          if (D == 3) un += __popc((ws[t] ^ zs[t] ^ jzs[t]) & 0x80808080u);
          ng += __popc(ws[t] & 0x80808080u);
        }
      }
      e = 2ll * un;  // - D N added once per configuration below
      m = -2ll * ng;
    } else
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
      const uint32_t x = i % (uint32_t)L, y = (i / (uint32_t)L) % (uint32_t)L;
      const uint32_t z = D == 3 ? i / ((uint32_t)L * (uint32_t)L) : 0u;
      const int si = sp[i];
      const uint32_t xp = (x + 1u == (uint32_t)L ? 0u : x + 1u) + (uint32_t)L * (y + (uint32_t)L * z);
      const uint32_t yp = x + (uint32_t)L * ((y + 1u == (uint32_t)L ? 0u : y + 1u) + (uint32_t)L * z);
      e -= Jp[i] * si * sp[xp];
      e -= Jp[N + i] * si * sp[yp];
      if (D == 3) {
        const uint32_t zp = x + (uint32_t)L * (y + (uint32_t)L * (z + 1u == (uint32_t)L ? 0u : z + 1u));
        e -= Jp[2u * N + i] * si * sp[zp];
      }
      m += si;
    }
    for (int off = 16; off > 0; off >>= 1) {
      e += __shfl_down_sync(0xffffffffu, e, off);
      m += __shfl_down_sync(0xffffffffu, m, off);
    }
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      red[0][wid] = e;
      red[1][wid] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long E = 0, M = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        E += red[0][w];
        M += red[1][w];
      }
      if ((L & 15) == 0) {
        E -= (long long)D * N;
        M += (long long)N;
      }
      int64_t* a = acc + ((size_t)s * slots + sigma) * kAccStride;
      a[0] = E;
      a[1] = M;
    }
    __syncthreads();
  }
}

// Block per (sample, temperature k): Q = sum_i s_i^0 s_i^1 between the
// configurations of replicas 0 and 1 that currently hold temperature k
// (Sec. 4.1 overlap).  Stored in acc[s][k*R][6].
__global__ void __launch_bounds__(256) k_overlap_i8(const int8_t* __restrict__ spins, const int32_t* slot_at,
                                                    const int8_t* __restrict__ occ, int64_t* acc, int S, int R,
                                                    int K, int slots, uint32_t N) {
  __shared__ long long red[8];
  for (uint32_t sk = blockIdx.x; sk < (uint32_t)(S * K); sk += gridDim.x) {
    const int s = (int)(sk / (uint32_t)K), k = (int)(sk - (uint32_t)s * K);
    const int s0 = slot_at[((size_t)s * R + 0) * K + k] * R + 0;
    const int s1 = slot_at[((size_t)s * R + 1) * K + k] * R + 1;
    const int8_t* a0 = spins + ((size_t)s0 * S + s) * N;
    const int8_t* a1 = spins + ((size_t)s1 * S + s) * N;
    long long q = 0;
    if (occ) {  // Q = sum_i x_i s_i^0 s_i^1
      const int8_t* xo = occ + (size_t)s * N;
      for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) q += xo[i] * a0[i] * a1[i];
    } else if ((N & 15u) == 0u) {  // 16 sites per step: s0 s1 = -1 iff the sign bits differ
      uint32_t d = 0;
      for (uint32_t i = 16u * threadIdx.x; i < N; i += 16u * blockDim.x) {
        const uint4 u = *reinterpret_cast<const uint4*>(a0 + i), v = *reinterpret_cast<const uint4*>(a1 + i);
        d += __popc((u.x ^ v.x) & 0x80808080u) + __popc((u.y ^ v.y) & 0x80808080u) +
             __popc((u.z ^ v.z) & 0x80808080u) + __popc((u.w ^ v.w) & 0x80808080u);
      }
      q = -2ll * d;  // N added once below
    } else {
      for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) q += a0[i] * a1[i];
    }
    for (int off = 16; off > 0; off >>= 1) q += __shfl_down_sync(0xffffffffu, q, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long Q = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) Q += red[w];
      if (!occ && (N & 15u) == 0u) Q += (long long)N;
      acc[((size_t)s * slots + (size_t)k * R) * kAccStride + 6] = Q;
    }
    __syncthreads();
  }
}

// natural-order conversions: device [S][slots][N] <-> [slots][S][N]
__global__ void k_copy_spins_i8(int8_t* spins, int8_t* out, const int8_t* in, int S, int slots, uint32_t N) {
  const uint64_t total = (uint64_t)S * slots * N;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = idx % N, rest = idx / N;
    const uint64_t sg = rest % slots, s = rest / slots;
    int8_t* v = spins + (sg * S + s) * N + i;
    if (out) out[idx] = *v;
    else *v = in[idx];
  }
}

inline unsigned grid_for(uint64_t total, unsigned block = 256, unsigned cap = 152u * 16u) {
  uint64_t g = (total + block - 1) / block;
  if (g > cap) g = cap;
  if (g == 0) g = 1;
  return (unsigned)g;
}

// ---- the plain layout swept bit-sliced in shared memory ----
//
// The random number of sample s at (site, sweep) is bit (s mod 64) of the
// plane stream drawn for the site and its group of 64 samples: the stream
// the bit-sliced layout draws once per 64-lane word.  So a block takes a
// tile of sites of one group and its configuration slots (two when the
// lattice has an even number of slots, so the couplings they share are read
// and converted once), reads the tile and its halo for the group's 64
// samples as bytes, turns them into 64-lane words in shared memory (bit l =
// sign of sample 64 g + l), runs the bit-sliced update of Sec. 3.2 on those
// words (one Philox block and one compare chain per 64 updates), and writes
// the tile's rows back as bytes.  The spins stay one byte each in global
// memory before and after every colour pass.
//
// Tile: kSlZ planes (3D) x kSlY rows x the L sites of a row (L = 32, 64 or
// 128).  Shared memory, 64-bit words; a row is stored by x parity (even x
// at x/2, odd x at L/2 + x/2), so the active sites of a warp are adjacent:
//   box [SB][NB][L]   each slot's spins: planes z0-1 and z0+kSlZ with rows
//                     y0..y0+kSlY-1 only (sl_zm_row, sl_zp_row), planes
//                     z0..z0+kSlZ-1 with rows y0-1..y0+kSlY (sl_own_row)
//   jx  [kSlZ][kSlY][L]          x+ couplings of the tile's sites
//   jy  [kSlZ][kSlY + 1][L]      y+ couplings of rows y0-1..y0+kSlY-1
//   jz  [kSlZ + 1][kSlY][L]      z+ couplings of planes z0-1..z0+kSlZ-1
//   tp  [SB][kPlanes][kMaxClasses]  threshold planes of each slot's 64 lanes
//   u   [SB][16] (uint4)         the slots' Philox parts shared by the block
//   staging, per warp [64][L/32] (uint32): 32-site sign masks per sample
// In 2D the box is one plane of kSlY + 2 rows and there is no jz.
constexpr int kSlThreads = 256;
constexpr uint32_t kSlZ = 2, kSlY = 4;

// Rows a block reads: the spin box without its four corner rows (no site of
// the tile has them as neighbours), then the coupling rows.
template <int D>
__host__ __device__ constexpr uint32_t sl_box_rows() {
  return D == 3 ? 2 * kSlY + kSlZ * (kSlY + 2) : kSlY + 2;
}
template <int D>
__host__ __device__ constexpr uint32_t sl_rows(uint32_t) {
  return sl_box_rows<D>() + (D == 3 ? kSlZ * kSlY + kSlZ * (kSlY + 1) + (kSlZ + 1) * kSlY : kSlY + (kSlY + 1));
}
// Words of the tile's shared-memory arrays (the box keeps room for its
// corner rows, unused).
template <int D>
__host__ __device__ constexpr uint32_t sl_smem_rows() {
  return D == 3 ? (kSlZ + 2) * (kSlY + 2) + kSlZ * kSlY + kSlZ * (kSlY + 1) + (kSlZ + 1) * kSlY
                : (kSlY + 2) + kSlY + (kSlY + 1);
}

__device__ __forceinline__ uint32_t sl_index(uint32_t x, uint32_t hL) { return (x & 1u) * hL + (x >> 1); }

// Site (within a 32-site chunk) whose bit sits at position q of a packed
// mask: site 4k + b at bit 8b + 7 - k (sl_pack).
__device__ __forceinline__ uint32_t sl_site_of_bit(uint32_t q) { return 4u * (7u - (q & 7u)) + (q >> 3); }

// Signs of 32 consecutive +-1 bytes (words k = 0..7 of a and b, byte b of
// word k = site 4k + b) as one 32-bit mask.  Every bit of a +-1 byte but
// bit 0 is its sign, so word k gives bit 7 - k of each of its bytes (word
// 7 gives bit 1, moved down to bit 0): site 4k + b lands at bit 8b + 7 - k.
__device__ __forceinline__ uint32_t sl_pack(const uint4& a, const uint4& b) {
  uint32_t m = a.x & 0x80808080u;
  m |= a.y & 0x40404040u;
  m |= a.z & 0x20202020u;
  m |= a.w & 0x10101010u;
  m |= b.x & 0x08080808u;
  m |= b.y & 0x04040404u;
  m |= b.z & 0x02020202u;
  m |= (b.w >> 1) & 0x01010101u;
  return m;
}

// Signs of 16 consecutive +-1 bytes (words k = 0..3 of v, byte b of word k
// = site 4k + b): site 4k + b at bit 8b + 7 - k (bits 4..7 of each byte).
__device__ __forceinline__ uint32_t sl_pack16(const uint4& v) {
  return (v.x & 0x80808080u) | (v.y & 0x40404040u) | (v.z & 0x20202020u) | (v.w & 0x10101010u);
}

// Two sl_pack16 masks of sites 0..15 (lo) and 16..31 (hi) of a chunk as one
// 32-bit mask: byte b holds lo's bits in its low nibble, hi's in its high
// nibble, so bit j is site 16 ((j >> 2) & 1) + 4 (3 - (j & 3)) + (j >> 3).
__device__ __forceinline__ uint32_t sl_merge16(uint32_t lo, uint32_t hi) {
  return ((lo >> 4) & 0x0F0F0F0Fu) | (hi & 0xF0F0F0F0u);
}

__device__ __forceinline__ uint32_t sl_site_of_bit16(uint32_t j) {
  return 16u * ((j >> 2) & 1u) + 4u * (3u - (j & 3u)) + (j >> 3);
}

// Word k of the 32 bytes a mask packs: sign of byte b from bit 8b + 7 - k,
// byte = +1 (0x01) or -1 (0xFF) = 1 + 0xFE sign.
__device__ __forceinline__ uint32_t sl_unpack_word(uint32_t m, int k) {
  return ((m >> (7 - k)) & 0x01010101u) * 0xFEu + 0x01010101u;
}

// 32 x 32 bit transpose across a warp: lane i holds row i on entry (bit j
// = element (i, j)) and column i on return (bit j = element (j, i)).  Stage
// s swaps bit s of the row index with bit s of the column index: the lane
// with bit s of its index clear keeps its bits j with bit s clear and takes
// the partner's bits with bit s clear shifted up by s; the other lane keeps
// the bits with bit s set and takes the partner's shifted down by s.  A
// rotation stands in for either shift: the bits it wraps around land where
// the keep-mask discards them.  The per-lane rotations and keep-masks of the
// five stages are constants.
struct SlTranspose {
  uint32_t rot[5], keep[5];
  __device__ __forceinline__ SlTranspose() {
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const uint32_t s = 16u >> i;
      const uint32_t m = i == 0 ? 0x0000FFFFu : i == 1 ? 0x00FF00FFu : i == 2 ? 0x0F0F0F0Fu : i == 3 ? 0x33333333u
                                                                                                      : 0x55555555u;
      const bool up = (lane & s) != 0u;
      rot[i] = up ? 32u - s : s;  // rotate left: down by s, or up by s
      keep[i] = up ? ~m : m;
    }
  }
  __device__ __forceinline__ uint32_t operator()(uint32_t x) const {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const uint32_t y = __shfl_xor_sync(0xffffffffu, x, 16u >> i);
      const uint32_t yr = __funnelshift_l(y, y, rot[i]);
      x = (x & keep[i]) | (yr & ~keep[i]);
    }
    return x;
  }
};

// Row of the compact spin box (the corner rows are not stored): 3D planes 0
// and kSlZ + 1 hold rows 1..kSlY of the box only, planes 1..kSlZ all kSlY +
// 2 rows; 2D one plane of kSlY + 2 rows.  own(zi, yi): the row of tile
// site row yi (0..kSlY-1) of tile plane zi (0..kSlZ-1).
template <int D>
__device__ __forceinline__ uint32_t sl_own_row(uint32_t zi, uint32_t yi) {
  return D == 3 ? kSlY + zi * (kSlY + 2) + yi + 1u : yi + 1u;
}
template <int D>
__device__ __forceinline__ uint32_t sl_zm_row(uint32_t zi, uint32_t yi) {  // the same row one plane down
  return zi == 0u ? yi : sl_own_row<D>(zi - 1u, yi);
}
template <int D>
__device__ __forceinline__ uint32_t sl_zp_row(uint32_t zi, uint32_t yi) {  // the same row one plane up
  return zi + 1u == kSlZ ? kSlY + kSlZ * (kSlY + 2) + yi : sl_own_row<D>(zi + 1u, yi);
}

// SB configuration slots (1, or 2 when the lattice has an even number) per
// block: the slots share the group's couplings, which are converted once.
template <int D, int ALGO, int C, int SB>
__global__ void __launch_bounds__(kSlThreads, 3) k_sweep_i8_sliced(const I8Params p) {
  extern __shared__ uint64_t sl[];
  constexpr uint32_t TZ = D == 3 ? kSlZ : 1u, BY = kSlY + 2;
  constexpr uint32_t NB = sl_box_rows<D>();  // rows of one slot's compact box
  const uint32_t L = (uint32_t)p.L, hL = L >> 1, N = p.N, S = (uint32_t)p.S;
  uint64_t* box = sl;                        // [SB][NB][L]
  uint64_t* jx = box + SB * NB * L;           // [TZ][kSlY][L]
  uint64_t* jy = jx + TZ * kSlY * L;          // [TZ][kSlY + 1][L]
  uint64_t* jz = jy + TZ * (kSlY + 1) * L;    // [TZ + 1][kSlY][L] (3D)
  uint64_t* tp = jz + (D == 3 ? (TZ + 1) * kSlY * L : 0u);  // [SB][kPlanes][kMaxClasses]
  // grid (slot pairs, tiles, groups): the slots of one tile and group run
  // side by side, so the couplings they share are read from DRAM once
  const uint32_t tiles_y = L / kSlY;
  const uint32_t y0 = (blockIdx.y % tiles_y) * kSlY, z0 = (blockIdx.y / tiles_y) * TZ;
  const uint32_t g = blockIdx.z;
  const int sigma0 = (int)blockIdx.x * SB;
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const Tick tk = sweep_tick(p.t_lo, p.t_hi, p.t_dev);
  auto wrap = [L](uint32_t v) { return v == 0xFFFFFFFFu ? L - 1u : (v == L ? 0u : v); };  // v in [-1, L]
  constexpr uint32_t kWarps = kSlThreads / 32;
  // the boxes and the couplings, one row (L sites) of the group's 64
  // samples per warp task.  A sample's row is read as P = L/16 pieces of 16
  // bytes by P consecutive lanes, 32/P samples per load instruction, so a
  // load touches 32/P lines instead of 32; each lane packs its piece's 16
  // signs, neighbouring lanes merge their halves of a 32-site chunk into the
  // warp's staging row [sample][chunk], and the row's words are then formed
  // chunk by chunk: lane l reads the 32-site mask of sample 32 h + l and the
  // warp transposes.  Warp w takes rows w, w + 8, ... of the block's list:
  // the SB compact boxes, then the coupling rows.
  constexpr int P = 2 * C;          // pieces of 16 sites per row
  constexpr int SPI = 32 / P;       // samples per load instruction
  constexpr int NI = 64 / SPI;      // load instructions per row
  constexpr int SW = C;             // staging words (32-site masks) per sample
  constexpr uint32_t n_box = SB * NB, n_jx = TZ * kSlY, n_jy = TZ * (kSlY + 1);
  const uint32_t n_rows = n_box + sl_rows<D>(L) - NB;
  const uint32_t xq = sl_site_of_bit16(lane);
  const uint32_t dq = sl_index(xq, hL);  // chunk c adds 16 c: each 32-site chunk is 16 words of each parity
  uint4* su = reinterpret_cast<uint4*>(tp + SB * kPlanes * kMaxClasses);  // [SB][16] Philox parts
  uint32_t* stage = reinterpret_cast<uint32_t*>(su + SB * 16) + warp * (64 * SW);
  const uint32_t grp = lane / P, piece = lane - grp * P;
  // row r of the list: issue this lane's loads (v) and return the row's
  // shared-memory words
  uint4 v[NI];
  auto issue = [&](uint32_t r) -> uint64_t* {
    uint32_t z, y, d = 0;
    const int8_t* src0;
    size_t stride;
    if (r < n_box) {
      const uint32_t as = r / NB, rb = r - as * NB;
      // 3D: rows 1..kSlY of box plane 0, all rows of planes 1..kSlZ, rows
      // 1..kSlY of plane kSlZ + 1
      uint32_t zi = 0u, yi = rb;
      if (D == 3) {
        if (rb < kSlY) {
          yi = rb + 1u;
        } else if (rb < kSlY + kSlZ * BY) {
          zi = 1u + (rb - kSlY) / BY;
          yi = rb - kSlY - (zi - 1u) * BY;
        } else {
          zi = kSlZ + 1u;
          yi = rb - kSlY - kSlZ * BY + 1u;
        }
      }
      z = D == 3 ? wrap(z0 + zi - 1u) : 0u;
      y = wrap(y0 + yi - 1u);
      stride = (size_t)N;
      src0 = p.spins + ((size_t)(sigma0 + (int)as) * S + 64u * g) * N;
    } else {
      const uint32_t rj = r - n_box;
      if (rj < n_jx) {
        const uint32_t zi = rj / kSlY, yi = rj - zi * kSlY;
        z = z0 + zi;
        y = y0 + yi;
      } else if (rj < n_jx + n_jy) {
        const uint32_t rr = rj - n_jx, zi = rr / (kSlY + 1), yi = rr - zi * (kSlY + 1);
        z = z0 + zi;
        y = wrap(y0 + yi - 1u);
        d = 1;
      } else {
        const uint32_t rr = rj - n_jx - n_jy, zi = rr / kSlY, yi = rr - zi * kSlY;
        z = wrap(z0 + zi - 1u);
        y = y0 + yi;
        d = 2;
      }
      stride = (size_t)D * N;
      src0 = p.J + (size_t)64u * g * D * N + (size_t)d * N;
    }
    // lane's sample for instruction i: 64 g + SPI i + grp
    const int8_t* base = src0 + ((size_t)z * L + y) * L + 16u * piece + (size_t)grp * stride;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      v[i] = make_uint4(0u, 0u, 0u, 0u);
      if (64u * g + (uint32_t)(SPI * i) + grp < S) v[i] = *reinterpret_cast<const uint4*>(base + (size_t)(SPI * i) * stride);
    }
    return box + r * L;  // the boxes and coupling arrays follow the row list
  };
  // the first row's loads are in flight while the threshold planes are built
  uint64_t* dst = warp < n_rows ? issue(warp) : nullptr;
  const SlTranspose tr;
  // threshold planes of the 64 lanes of each slot: one warp per (slot,
  // class u).  Plane q is bit 31 - q of each lane's threshold (0 for a
  // threshold of 2^32), i.e. a row of the transposed 32 x 32 bit matrix of
  // the thresholds of 32 lanes; plane 32 marks the thresholds of 2^32.
#pragma unroll 1
  for (uint32_t task = warp; task < SB * (2u * D + 1u); task += kWarps) {
    const uint32_t as = task / (2u * D + 1u), u = task - as * (2u * D + 1u);
    const int sigma = sigma0 + (int)as, tslot = sigma / p.R, rep = sigma - tslot * p.R;
    uint64_t T[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t s = 64u * g + 32u * (uint32_t)h + lane;
      const int k = s < S ? p.temp_of[((size_t)s * p.R + rep) * p.K + tslot] : tslot;
      T[h] = p.thr[(size_t)k * kMaxClasses + u];
    }
    const uint64_t always = (uint64_t)__ballot_sync(0xffffffffu, T[0] >= kTwo32) |
                            ((uint64_t)__ballot_sync(0xffffffffu, T[1] >= kTwo32) << 32);
    // after the transpose lane j holds bit j of the 32 lanes' thresholds
    const uint32_t lo = tr(T[0] >= kTwo32 ? 0u : (uint32_t)T[0]);
    const uint32_t hi = tr(T[1] >= kTwo32 ? 0u : (uint32_t)T[1]);
    uint64_t* tpa = tp + as * kPlanes * kMaxClasses;
    tpa[(31u - lane) * kMaxClasses + u] = (uint64_t)lo | ((uint64_t)hi << 32);
    if (lane == 0) tpa[32 * kMaxClasses + u] = always;
  }
  planes::plane_uniform_table(su, SB, sigma0, g, tk, p.keys);
  // each row: its signs packed and staged, the next row's loads issued,
  // then the staged chunks transposed into the row's words
#pragma unroll 1
  for (uint32_t r = warp; r < n_rows; r += kWarps) {
    // pieces 2c and 2c + 1 of a sample sit in neighbouring lanes: the even
    // lane merges them into the chunk's 32-site mask and stages it
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const uint32_t mine = sl_pack16(v[i]);
      const uint32_t other = __shfl_xor_sync(0xffffffffu, mine, 1);
      if ((piece & 1u) == 0u) stage[((uint32_t)(SPI * i) + grp) * SW + (piece >> 1)] = sl_merge16(mine, other);
    }
    __syncwarp();
    uint64_t* const cur = dst;
    if (r + kWarps < n_rows) dst = issue(r + kWarps);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const uint32_t lo = tr(stage[lane * SW + c]);
      const uint32_t hi = tr(stage[(32u + lane) * SW + c]);
      cur[dq + 16u * c] = (uint64_t)lo | ((uint64_t)hi << 32);
    }
    __syncwarp();
  }
  __syncthreads();
  // the colour pass on the tile's words, every slot of the block per word
  const uint32_t n_act = TZ * kSlY * hL;
#pragma unroll 1
  for (uint32_t w = threadIdx.x; w < n_act; w += kSlThreads) {
    const uint32_t k = w % hL, rest = w / hL, yi = rest % kSlY, zi = rest / kSlY;
    const uint32_t y = y0 + yi, z = D == 3 ? z0 + zi : 0u;
    const uint32_t par = (uint32_t)(p.colour ^ (int)(y + z)) & 1u;
    const uint32_t x = 2u * k + par;
    const uint32_t is = par * hL + k;                                        // the site (parity par)
    const uint32_t ip = par ? (k + 1u == hL ? 0u : k + 1u) : hL + k;          // x + 1
    const uint32_t im = par ? k : hL + (k == 0u ? hL - 1u : k - 1u);          // x - 1
    const uint32_t ro = sl_own_row<D>(zi, yi) * L, rzp = sl_zp_row<D>(zi, yi) * L, rzm = sl_zm_row<D>(zi, yi) * L;
    uint64_t jw[2 * D];
    jw[0] = jx[(zi * kSlY + yi) * L + is];
    jw[1] = jx[(zi * kSlY + yi) * L + im];
    jw[2] = jy[(zi * (kSlY + 1) + yi + 1u) * L + is];
    jw[3] = jy[(zi * (kSlY + 1) + yi) * L + is];
    if (D == 3) {
      jw[4] = jz[((zi + 1u) * kSlY + yi) * L + is];
      jw[5] = jz[(zi * kSlY + yi) * L + is];
    }
    const planes::PlaneSiteKey sk = planes::plane_site_key(x + L * (y + L * z), tk, p.keys);
#pragma unroll
    for (int as = 0; as < SB; ++as) {
      uint64_t* bx = box + (uint32_t)as * NB * L;
      const uint64_t b = bx[ro + is];
      uint64_t e[2 * D];
      e[0] = b ^ bx[ro + ip] ^ jw[0];
      e[1] = b ^ bx[ro + im] ^ jw[1];
      e[2] = b ^ bx[ro + L + is] ^ jw[2];
      e[3] = b ^ bx[ro - L + is] ^ jw[3];
      if (D == 3) {
        e[4] = b ^ bx[rzp + is] ^ jw[4];
        e[5] = b ^ bx[rzm + is] ^ jw[5];
      }
      uint64_t u0, u1, u2;
      count_unsat<D>(e, u0, u1, u2);
      const uint64_t* tpa = tp + (uint32_t)as * kPlanes * kMaxClasses;
      planes::LazyWord lw = planes::bits_word_start<D, ALGO>(tpa, u0, u1, u2);
      planes::bits_plane_pairs<D, ALGO>(lw, tpa, su + 16 * as, sk, p.keys, 0u, tk, 0u, 16u);
      const uint64_t flip = ALGO == 0 ? lw.lt : ~lw.lt;
      if (flip) bx[ro + is] = b ^ flip;
    }
  }
  __syncthreads();
  // the tile's rows back to global memory, a row of the group's 64 samples
  // per warp task: lane q takes the word of the site whose sign lands at
  // bit q of the 32-byte packing (sl_pack), so after the transpose lane l
  // holds sample 32 h + l's 32 signs in the order sl_unpack_word expects
  const uint32_t dq3 = sl_index(sl_site_of_bit(lane), hL);
#pragma unroll 1
  for (uint32_t r = warp; r < SB * TZ * kSlY; r += kWarps) {
    const uint32_t as = r / (TZ * kSlY), ro = r - as * (TZ * kSlY), zi = ro / kSlY, yi = ro - zi * kSlY;
    const uint32_t y = y0 + yi, z = D == 3 ? z0 + zi : 0u;
    const uint64_t* src = box + (as * NB + sl_own_row<D>(zi, yi)) * L + dq3;
    const size_t row_off = ((size_t)z * L + y) * L;
    const uint32_t s_0 = 64u * g + lane, s_1 = s_0 + 32u;
    const size_t sl0 = (size_t)(sigma0 + (int)as) * S;
    int8_t* d0 = p.spins + (sl0 + s_0) * N + row_off;
    int8_t* d1 = p.spins + (sl0 + s_1) * N + row_off;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const uint64_t wv = src[16 * c];
      const uint32_t m0 = tr((uint32_t)wv), m1 = tr((uint32_t)(wv >> 32));
      if (s_0 < S) {
        *reinterpret_cast<uint4*>(d0 + 32 * c) =
            make_uint4(sl_unpack_word(m0, 0), sl_unpack_word(m0, 1), sl_unpack_word(m0, 2), sl_unpack_word(m0, 3));
        *reinterpret_cast<uint4*>(d0 + 32 * c + 16) =
            make_uint4(sl_unpack_word(m0, 4), sl_unpack_word(m0, 5), sl_unpack_word(m0, 6), sl_unpack_word(m0, 7));
      }
      if (s_1 < S) {
        *reinterpret_cast<uint4*>(d1 + 32 * c) =
            make_uint4(sl_unpack_word(m1, 0), sl_unpack_word(m1, 1), sl_unpack_word(m1, 2), sl_unpack_word(m1, 3));
        *reinterpret_cast<uint4*>(d1 + 32 * c + 16) =
            make_uint4(sl_unpack_word(m1, 4), sl_unpack_word(m1, 5), sl_unpack_word(m1, 6), sl_unpack_word(m1, 7));
      }
    }
  }
}

// Shared memory of a block: SB compact spin boxes, the coupling rows, SB
// threshold-plane tables, SB tables of shared Philox parts and the warps'
// staging rows.
size_t sl_smem_bytes(int D, uint32_t L, int SB) {
  const uint32_t box = D == 3 ? sl_box_rows<3>() : sl_box_rows<2>();
  const uint32_t jrows = (D == 3 ? sl_rows<3>(L) : sl_rows<2>(L)) - box;
  const size_t stage = (size_t)(kSlThreads / 32) * 64 * (L / 32) * sizeof(uint32_t);  // per warp [64][L/32] masks
  return ((size_t)(SB * box + jrows) * L + (size_t)SB * kPlanes * kMaxClasses) * sizeof(uint64_t) +
         (size_t)SB * 16 * sizeof(uint4) + stage;
}

// The shared-memory bit-sliced sweep takes rows of 1, 2 or 4 whole 32-site
// chunks, read by 2, 4 or 8 lanes per sample: L = 32, 64 or 128 (3D tiles
// of 98 L words, 2D of 27 L, plus 1 KiB L/16 of staging).
bool i8_sliced_fits(const Lattice& lat) {
  return (lat.D == 2 || lat.D == 3) && (lat.L == 32 || lat.L == 64 || lat.L == 128) && !lat.field &&
         lat.rng != IANUS_RNG_WHEEL;
}

template <int D, int ALGO, int C, int SB>
cudaError_t launch_sliced_c(Lattice& lat, const I8Params& p, dim3 grid, size_t smem) {
  static bool ok = false;
  if (!ok) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_i8_sliced<D, ALGO, C, SB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    ok = true;
  }
  k_sweep_i8_sliced<D, ALGO, C, SB><<<grid, kSlThreads, smem, lat.stream>>>(p);
  return cudaGetLastError();
}

// Two configuration slots per block when the lattice has an even number of
// slots, else one.
template <int D, int ALGO>
cudaError_t launch_sliced(Lattice& lat, const I8Params& p) {
  const int SB = lat.slots % 2 == 0 ? 2 : 1;
  const size_t smem = sl_smem_bytes(D, (uint32_t)lat.L, SB);
  const uint32_t tiles = (uint32_t)lat.L / kSlY * (D == 3 ? (uint32_t)lat.L / kSlZ : 1u);
  const dim3 grid((unsigned)(lat.slots / SB), tiles, (unsigned)lat.G);
  switch (lat.L / 32 * 2 + (SB - 1)) {
    case 2: return launch_sliced_c<D, ALGO, 1, 1>(lat, p, grid, smem);
    case 3: return launch_sliced_c<D, ALGO, 1, 2>(lat, p, grid, smem);
    case 4: return launch_sliced_c<D, ALGO, 2, 1>(lat, p, grid, smem);
    case 5: return launch_sliced_c<D, ALGO, 2, 2>(lat, p, grid, smem);
    case 8: return launch_sliced_c<D, ALGO, 4, 1>(lat, p, grid, smem);
    default: return launch_sliced_c<D, ALGO, 4, 2>(lat, p, grid, smem);
  }
}

}  // namespace

cudaError_t launch_init_i8(Lattice& lat, int jmode) {
  InitParams p{(int8_t*)lat.spins, (int8_t*)lat.J, lat.S, lat.D, lat.slots, lat.N, jmode, lat.keys};
  k_init_i8<<<grid_for((uint64_t)lat.S * lat.N), 256, 0, lat.stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_sweep_i8(Lattice& lat, int colour, uint64_t t, int inv) {
  I8Params p;
  p.spins = (int8_t*)lat.spins;
  p.J = (const int8_t*)lat.J;
  p.thr = lat.thr;
  p.temp_of = lat.temp_of;
  p.S = lat.S;
  p.R = lat.R;
  p.K = lat.K;
  p.slots = lat.slots;
  p.L = lat.L;
  p.N = lat.N;
  p.half = lat.N / 2;
  p.colour = colour;
  p.inv = inv;
  p.t_lo = (uint32_t)(t & 0xffffffffu);
  p.t_hi = (uint32_t)(t >> 32);
  p.keys = lat.keys;
  p.t_dev = lat.capturing ? lat.t_dev : nullptr;
  if (lat.rng == IANUS_RNG_WHEEL) {
    const WheelParams wp{p, lat.wheels, lat.rows, lat.hs, lat.occ, lat.fthr};
    const unsigned wgrid = grid_for((uint64_t)lat.slots * lat.S * lat.rows, kWheelBlock, 152u * 12u);
    if (lat.field)
      lat.D == 3 ? k_sweep_wheel_i8<3, true><<<wgrid, kWheelBlock, 0, lat.stream>>>(wp)
                 : k_sweep_wheel_i8<2, true><<<wgrid, kWheelBlock, 0, lat.stream>>>(wp);
    else
      lat.D == 3 ? k_sweep_wheel_i8<3, false><<<wgrid, kWheelBlock, 0, lat.stream>>>(wp)
                 : k_sweep_wheel_i8<2, false><<<wgrid, kWheelBlock, 0, lat.stream>>>(wp);
    return cudaGetLastError();
  }
  const uint64_t total = (uint64_t)lat.slots * lat.S * p.half;
  const unsigned grid = grid_for(total, 256, 152u * 8u);
  if (lat.field) {
    const FieldI8Params fp{p, lat.hs, lat.occ, lat.fthr};
    if (lat.D == 3)
      k_sweep_field_i8<3><<<grid, 256, 0, lat.stream>>>(fp);
    else
      k_sweep_field_i8<2><<<grid, 256, 0, lat.stream>>>(fp);
    return cudaGetLastError();
  }
  if (lat.variant == 0 && i8_sliced_fits(lat)) {  // bit-sliced in shared memory, the automatic choice
    if (lat.D == 3) return inv ? launch_sliced<3, 1>(lat, p) : launch_sliced<3, 0>(lat, p);
    return inv ? launch_sliced<2, 1>(lat, p) : launch_sliced<2, 0>(lat, p);
  }
  if (lat.variant != 1 && lat.L % 4 == 0) {  // the word kernel: 4-byte words, planes shared by the group
    const dim3 wgrid((lat.N / 4u + kWordThreads - 1) / kWordThreads, (unsigned)lat.G, (unsigned)lat.slots);
    if (lat.D == 3)
      k_sweep_i8_words<3><<<wgrid, kWordThreads, 0, lat.stream>>>(p);
    else
      k_sweep_i8_words<2><<<wgrid, kWordThreads, 0, lat.stream>>>(p);
    return cudaGetLastError();
  }
  if (lat.variant != 1) {  // the tiled kernel (planes shared by the group); variant 1: one thread per update
    const dim3 tgrid((p.half + kTileSites - 1) / kTileSites, (unsigned)lat.G, (unsigned)lat.slots);
    if (lat.D == 3)
      k_sweep_i8_tiled<3><<<tgrid, kTileThreads, 0, lat.stream>>>(p);
    else
      k_sweep_i8_tiled<2><<<tgrid, kTileThreads, 0, lat.stream>>>(p);
    return cudaGetLastError();
  }
  if (lat.D == 3)
    k_sweep_i8<3><<<grid, 256, 0, lat.stream>>>(p);
  else
    k_sweep_i8<2><<<grid, 256, 0, lat.stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_measure_i8(Lattice& lat, int want_q) {
  const unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)lat.slots * lat.S, 152u * 8u);
  if (lat.field && lat.D == 3)
    k_measure_field_i8<3><<<grid, 256, 0, lat.stream>>>((const int8_t*)lat.spins, (const int8_t*)lat.J, lat.hs,
                                                         lat.occ, lat.acc, lat.S, lat.slots, lat.L, lat.N);
  else if (lat.field)
    k_measure_field_i8<2><<<grid, 256, 0, lat.stream>>>((const int8_t*)lat.spins, (const int8_t*)lat.J, lat.hs,
                                                         lat.occ, lat.acc, lat.S, lat.slots, lat.L, lat.N);
  else if (lat.K == 1 && lat.R <= 2 && lat.L % 16 == 0) {  // E, M (and Q) in one pass per sample
    const unsigned gs = (unsigned)std::min<uint64_t>((uint64_t)lat.S, 152u * 8u);
    const int8_t* sp = (const int8_t*)lat.spins;
    const int8_t* J = (const int8_t*)lat.J;
    if (lat.D == 3) {
      if (lat.R == 2) k_measure_i8_k1<3, 2><<<gs, 256, 0, lat.stream>>>(sp, J, lat.acc, lat.S, lat.L, lat.N, want_q);
      else k_measure_i8_k1<3, 1><<<gs, 256, 0, lat.stream>>>(sp, J, lat.acc, lat.S, lat.L, lat.N, want_q);
    } else {
      if (lat.R == 2) k_measure_i8_k1<2, 2><<<gs, 256, 0, lat.stream>>>(sp, J, lat.acc, lat.S, lat.L, lat.N, want_q);
      else k_measure_i8_k1<2, 1><<<gs, 256, 0, lat.stream>>>(sp, J, lat.acc, lat.S, lat.L, lat.N, want_q);
    }
    return cudaGetLastError();
  } else if (lat.D == 3)
    k_measure_i8<3><<<grid, 256, 0, lat.stream>>>((const int8_t*)lat.spins, (const int8_t*)lat.J, lat.acc,
                                                   lat.S, lat.R, lat.slots, lat.L, lat.N);
  else
    k_measure_i8<2><<<grid, 256, 0, lat.stream>>>((const int8_t*)lat.spins, (const int8_t*)lat.J, lat.acc,
                                                   lat.S, lat.R, lat.slots, lat.L, lat.N);
  if (want_q && lat.R >= 2) {
    const unsigned gq = (unsigned)std::min<uint64_t>((uint64_t)lat.S * lat.K, 152u * 8u);
    k_overlap_i8<<<gq, 256, 0, lat.stream>>>((const int8_t*)lat.spins, lat.slot_at, lat.field ? lat.occ : nullptr,
                                            lat.acc, lat.S, lat.R, lat.K, lat.slots, lat.N);
  }
  return cudaGetLastError();
}

bool resident_i8_fits(const Lattice& lat) {
  return lat.layout == IANUS_LAYOUT_I8 && !lat.field && lat.rng == IANUS_RNG_PHILOX && lat.K == 1 && (size_t)lat.N * (1 + lat.D) <= kResidentSmemMax;
}

// Launch geometry of the cluster-resident kernel for cluster size C.
struct ClusterShape {
  uint32_t PA, A;    // sites of a slab, of a plane
  unsigned threads;  // per block
  size_t smem;
  bool one;          // at most one site of each colour per thread
};

inline ClusterShape cluster_shape(const Lattice& lat, int C) {
  ClusterShape c;
  const uint32_t L = (uint32_t)lat.L;
  c.A = lat.D == 3 ? L * L : L;
  c.PA = (L / (uint32_t)C) * c.A;
  c.threads = std::min(kClusterBlockMax, ((c.PA / 2u + 31u) / 32u) * 32u);
  c.smem = (size_t)c.PA * (1 + lat.D) + 3u * c.A;
  c.one = c.PA / 2u <= c.threads;
  return c;
}

template <int D, bool ONE>
cudaError_t cluster_launch(const Lattice& lat, const ResidentParams* p, unsigned configs, int C, bool query, int* n) {
  const ClusterShape sh = cluster_shape(lat, C);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(configs * (unsigned)C);
  cfg.blockDim = dim3(sh.threads);
  cfg.dynamicSmemBytes = sh.smem;
  cfg.stream = query ? 0 : lat.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (query) {
    if (C > 8) {
      const cudaError_t e =
          cudaFuncSetAttribute(k_resident_cluster_i8<D, ONE>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveClusters(n, k_resident_cluster_i8<D, ONE>, &cfg);
  }
  return cudaLaunchKernelEx(&cfg, k_resident_cluster_i8<D, ONE>, *p, C);
}

template <int D>
cudaError_t cluster_dispatch(const Lattice& lat, const ResidentParams* p, unsigned configs, int C, bool query,
                             int* n) {
  return cluster_shape(lat, C).one ? cluster_launch<D, true>(lat, p, configs, C, query, n)
                                   : cluster_launch<D, false>(lat, p, configs, C, query, n);
}

// Cluster-resident launch shape of one configuration: the largest divisor C
// of L with 2 <= C <= 16 that keeps the grid within two blocks per SM (unless
// forced) and for which a cluster can be scheduled; 0 = one block per
// configuration.
int resident_cluster_size(const Lattice& lat, unsigned configs, bool force) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  const uint32_t L = (uint32_t)lat.L;
  for (int C = 16; C >= 2; --C) {
    if (L % (uint32_t)C != 0u || (!force && (uint64_t)configs * (uint64_t)C > 2ull * (uint64_t)sms)) continue;
    int n = 0;
    const cudaError_t e = lat.D == 3 ? cluster_dispatch<3>(lat, nullptr, configs, C, true, &n)
                                     : cluster_dispatch<2>(lat, nullptr, configs, C, true, &n);
    if (e != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (n >= 1) return C;
  }
  return 0;
}

cudaError_t launch_resident_i8(Lattice& lat, int inv, uint32_t nsweeps, uint32_t measure_every) {
  ResidentParams p;
  p.spins = (int8_t*)lat.spins;
  p.J = (const int8_t*)lat.J;
  p.thr = lat.thr;
  p.S = lat.S;
  p.R = lat.R;
  p.slots = lat.slots;
  p.L = lat.L;
  p.inv = inv;
  p.N = lat.N;
  p.half = lat.N / 2;
  p.t0 = lat.sweeps;
  p.nsweeps = nsweeps;
  p.measure_every = measure_every;
  p.row0 = lat.ser_count;
  p.cap = lat.cap;
  p.ser_E = lat.ser_E;
  p.ser_M = lat.ser_M;
  p.ser_sweep = lat.ser_sweep;
  p.keys = lat.keys;
  const size_t smem = (size_t)lat.N * (1 + lat.D);
  const unsigned blocks = (unsigned)(lat.slots * lat.S);
  if (lat.resident_mode == 1 || lat.resident_mode == 3) {
    const int C = resident_cluster_size(lat, blocks, lat.resident_mode == 3);
    if (C > 0)
      return lat.D == 3 ? cluster_dispatch<3>(lat, &p, blocks, C, false, nullptr)
                        : cluster_dispatch<2>(lat, &p, blocks, C, false, nullptr);
  }
  cudaError_t e;
  if (lat.D == 3) {
    e = cudaFuncSetAttribute(k_resident_i8<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResidentSmemMax);
    if (e == cudaSuccess) k_resident_i8<3><<<blocks, 1024, smem, lat.stream>>>(p);
  } else {
    e = cudaFuncSetAttribute(k_resident_i8<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResidentSmemMax);
    if (e == cudaSuccess) k_resident_i8<2><<<blocks, 1024, smem, lat.stream>>>(p);
  }
  return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t launch_get_spins_i8(Lattice& lat, int8_t* dev_out) {
  k_copy_spins_i8<<<grid_for((uint64_t)lat.S * lat.slots * lat.N), 256, 0, lat.stream>>>(
      (int8_t*)lat.spins, dev_out, nullptr, lat.S, lat.slots, lat.N);
  return cudaGetLastError();
}

cudaError_t launch_set_spins_i8(Lattice& lat, const int8_t* dev_in) {
  k_copy_spins_i8<<<grid_for((uint64_t)lat.S * lat.slots * lat.N), 256, 0, lat.stream>>>(
      (int8_t*)lat.spins, nullptr, dev_in, lat.S, lat.slots, lat.N);
  return cudaGetLastError();
}

cudaError_t launch_get_couplings_i8(Lattice& lat, int8_t* dev_out) {
  return cudaMemcpyAsync(dev_out, lat.J, (size_t)lat.S * lat.D * lat.N, cudaMemcpyDeviceToDevice, lat.stream);
}

cudaError_t launch_set_couplings_i8(Lattice& lat, const int8_t* dev_in) {
  return cudaMemcpyAsync(lat.J, dev_in, (size_t)lat.S * lat.D * lat.N, cudaMemcpyDeviceToDevice, lat.stream);
}

cudaError_t launch_init_wheels(Lattice& lat) {
  k_init_wheels<<<grid_for((uint64_t)lat.slots * lat.S * 2u * lat.rows), 256, 0, lat.stream>>>(
      lat.wheels, lat.S, lat.slots, lat.rows, lat.keys);
  return cudaGetLastError();
}

cudaError_t launch_init_sites_i8(Lattice& lat, double occupation) {
  const uint64_t T_occ = (uint64_t)std::floor(std::ldexp(occupation, 32));
  k_init_sites_i8<<<grid_for((uint64_t)lat.S * lat.N), 256, 0, lat.stream>>>(
      lat.hs, lat.occ, lat.S, lat.N, lat.disorder == IANUS_DISORDER_RFIM, lat.disorder == IANUS_DISORDER_DAFF, T_occ,
      lat.keys);
  return cudaGetLastError();
}

cudaError_t launch_get_sites_i8(Lattice& lat, int8_t* dev_hs, int8_t* dev_occ) {
  const size_t n = (size_t)lat.S * lat.N;
  cudaError_t e = cudaMemcpyAsync(dev_hs, lat.hs, n, cudaMemcpyDeviceToDevice, lat.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dev_occ, lat.occ, n, cudaMemcpyDeviceToDevice, lat.stream);
  return e;
}

cudaError_t launch_set_sites_i8(Lattice& lat, const int8_t* dev_hs, const int8_t* dev_occ) {
  const size_t n = (size_t)lat.S * lat.N;
  cudaError_t e = cudaMemcpyAsync(lat.hs, dev_hs, n, cudaMemcpyDeviceToDevice, lat.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(lat.occ, dev_occ, n, cudaMemcpyDeviceToDevice, lat.stream);
  return e;
}

}  // namespace ianus
