// common.cuh -- device-side definitions shared by the library's kernels:
// the counter-based random stream, lattice geometry and launch parameters.
//
// Everything here follows the definitions stated in include/ianus.h:
// Philox4x32-10 (Salmon et al., SC'11) replaces the paper's Parisi-Rapuano
// wheel (Sec. 3.3, Eq. (5)); the lattice and checkerboard are those of
// Sec. 2.1 and Sec. 3.1.
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>

#include <cuda_runtime.h>
#else  // runtime compilation (jit.cu) provides no standard headers
typedef unsigned char uint8_t;
typedef signed char int8_t;
typedef unsigned int uint32_t;
typedef int int32_t;
typedef unsigned long long uint64_t;
typedef long long int64_t;
#endif

namespace ianus {

enum : uint32_t { TAG_SPIN = 1, TAG_J = 2, TAG_INIT = 3, TAG_POTTS = 4, TAG_PINIT = 5, TAG_PT = 6, TAG_H = 7, TAG_X = 8,
                   TAG_PERM = 9, TAG_WHEEL = 10 };

// Per-lane threshold planes of the bit-sliced layout: per class u = 0..2D
// (padded to 8), 32 bit-planes of the threshold, most significant first, and
// the "always" mask (threshold 2^32).
constexpr int kMaxClasses = 8;
constexpr int kPlanes = 33;

// Round keys of Philox4x32-10 for one seed: k[r] = key + r * (W0, W1) mod 2^32.
// Passed by value inside kernel parameters so that the XOR with the round key
// reads the constant bank.
struct PhiloxKeys {
  uint32_t k0[10];
  uint32_t k1[10];
};

#ifndef __CUDACC_RTC__
inline PhiloxKeys make_keys(uint64_t seed) {
  PhiloxKeys K;
  uint32_t a = (uint32_t)(seed & 0xffffffffu), b = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    K.k0[r] = a;
    K.k1[r] = b;
    a += 0x9E3779B9u;
    b += 0xBB67AE85u;
  }
  return K;
}
#endif

// One Philox4x32-10 block: ten rounds of two 32x32->64 products; the high
// halves are XORed with the other counter words and the round key.
__device__ __forceinline__ uint4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          const PhiloxKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
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

// The same block with the key (lo, hi) bumped by the Weyl constants each
// round, for keys that differ per thread (several jobs in one kernel).
__device__ __forceinline__ uint4 philox10_key(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Geometry of a periodic D-dimensional cube (D = 2 or 3) of even side L.
// Natural site index i = x + L*(y + L*z).  The checkerboard-split index puts
// the sites of one colour in one row (y, z) next to each other:
//   split(x, y, z) = (2*(y + L*z) + colour) * (L/2) + x/2.
struct Geom {
  int D, L, h;    // h = L/2
  uint32_t N;     // L^D
  uint32_t half;  // N/2 sites per colour
  int lh, lL;     // log2(h), log2(L) when L is a power of two (else 0)
};

#ifdef IANUS_JIT_L
// Kernels compiled at run time for one lattice get its geometry as constants
// (IANUS_JIT_D, IANUS_JIT_L, and IANUS_JIT_LH, IANUS_JIT_LL as above), so
// that the index arithmetic folds and words N apart are constant offsets.
constexpr uint32_t kJitSites = IANUS_JIT_D == 3 ? (uint32_t)IANUS_JIT_L * IANUS_JIT_L * IANUS_JIT_L
                                                : (uint32_t)IANUS_JIT_L * IANUS_JIT_L;
constexpr Geom kJitGeom = {IANUS_JIT_D, IANUS_JIT_L, IANUS_JIT_L / 2, kJitSites, kJitSites / 2, IANUS_JIT_LH,
                           IANUS_JIT_LL};
#endif

__host__ __device__ __forceinline__ uint32_t split_index(const Geom& g, int x, int y, int z) {
  const int c = (x + y + z) & 1;
  const uint32_t row = (uint32_t)y + (uint32_t)g.L * (uint32_t)z;
  return (2u * row + (uint32_t)c) * (uint32_t)g.h + (uint32_t)(x >> 1);
}

// Colour-c word w of the split layout -> coordinates and the split indices of
// the site and of its 2D neighbours (which all have colour 1-c).
struct Nbr {
  uint32_t self;
  uint32_t site;     // natural index (drives the random stream)
  uint32_t xp, xm;   // x+1, x-1
  uint32_t yp, ym;
  uint32_t zp, zm;
};

template <bool P2>
__device__ __forceinline__ Nbr split_neighbours_t(const Geom& g, int c, uint32_t w) {
  const uint32_t h = (uint32_t)g.h, L = (uint32_t)g.L;
  uint32_t row, k, y, z;
  if (P2) {  // L a power of two: shifts and masks
    row = w >> g.lh;
    k = w & (h - 1u);
    y = row & (L - 1u);
    z = row >> g.lL;
  } else {
    row = w / h;
    k = w - row * h;
    y = row % L;
    z = row / L;  // z = 0 for D = 2 (row < L)
  }
  const uint32_t xpar = (uint32_t)(c ^ (int)(y + z)) & 1u;
  const uint32_t x = 2u * k + xpar;
  const uint32_t oc = 1u - (uint32_t)c;
  Nbr n;
  n.self = (2u * row + (uint32_t)c) * h + k;
  n.site = x + L * (y + L * z);
  const uint32_t base_o = (2u * row + oc) * h;
  const uint32_t kp = xpar ? (k + 1u == h ? 0u : k + 1u) : k;  // (x+1)/2 mod h
  const uint32_t km = xpar ? k : (k == 0u ? h - 1u : k - 1u);  // (x-1)/2 mod h
  n.xp = base_o + kp;
  n.xm = base_o + km;
  const uint32_t yp = (y + 1u == L) ? 0u : y + 1u, ym = (y == 0u) ? L - 1u : y - 1u;
  n.yp = (2u * (yp + L * z) + oc) * h + k;
  n.ym = (2u * (ym + L * z) + oc) * h + k;
  if (g.D == 3) {
    const uint32_t zp = (z + 1u == L) ? 0u : z + 1u, zm = (z == 0u) ? L - 1u : z - 1u;
    n.zp = (2u * (y + L * zp) + oc) * h + k;
    n.zm = (2u * (y + L * zm) + oc) * h + k;
  } else {
    n.zp = n.zm = 0u;
  }
  return n;
}

__device__ __forceinline__ Nbr split_neighbours(const Geom& g, int c, uint32_t w) {
  return split_neighbours_t<false>(g, c, w);
}

// Launch parameters of the bit-sliced sweep kernels (k_msc.cu and the
// runtime-specialised kernel of jit_sweep.cuh).
struct BitsParams {
  uint64_t* spins;        // [G][slots][N]
  const uint64_t* J;      // [G][D][N]
  const uint64_t* tp;     // [G][slots][kPlanes][kMaxClasses] per-lane threshold planes
  Geom geom;
  int G, R, K, slots;
  int colour;
  uint32_t t_lo, t_hi;
  uint32_t words_per_block;  // colour-c words handled by one block (a multiple of 32)
  PhiloxKeys keys;
  const uint64_t* t_dev;     // non-null in captured graphs: sweep = *t_dev + t_lo
};

// Launch parameters of the persistent form of the lane-queue sweep
// (jit_sweep_lt.cuh with IANUS_JIT_PERSIST): one launch runs npass colour
// passes (colour 0 first) of sweeps t0, t0 + 1, ...  Block b owns rows
// [j R_g / cpg, (j + 1) R_g / cpg) of group g = b / cpg, j = b % cpg
// (R_g = N / L rows of L/2 words per colour).  flags[b] counts the passes b
// has completed in this launch (zeroed before the launch); a block starts a
// pass once the blocks owning the rows its sites' neighbours live in have
// completed the previous one, waiting at most timeout_ns.  On a wait that
// runs out the block sets ERR_TIMEOUT in *err and returns.  skip_block >= 0
// makes that block return at once (a wait that nothing ends, for tests).
struct PersistParams {
  uint32_t* flags;
  uint32_t* err;
  uint32_t npass;
  uint32_t cpg;
  uint32_t t0_lo, t0_hi;
  uint64_t timeout_ns;
  int32_t skip_block;
};

// The absolute sweep index of a launch: the (t_hi, t_lo) parameters, or in a
// captured graph the device-resident counter plus the offset in t_lo.
struct Tick {
  uint32_t lo, hi;
};

__device__ __forceinline__ Tick sweep_tick(uint32_t t_lo, uint32_t t_hi, const uint64_t* t_dev) {
  if (t_dev) {
    const uint64_t t = *t_dev + (uint64_t)t_lo;
    return Tick{(uint32_t)t, (uint32_t)(t >> 32)};
  }
  return Tick{t_lo, t_hi};
}

// Entry of a kernel launched with programmatic stream serialisation: wait
// until the previous kernel on the stream has completed and its writes are
// visible (nothing of the previous grid is read or written before this),
// then allow the next such kernel's blocks onto the SMs this grid's tail
// leaves free.  Both are no-ops for a plain launch.
__device__ __forceinline__ void dependent_launch_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Number of unsatisfied bonds per lane as bit-planes (u2, u1, u0), from the
// 2D unsatisfied-bond words e[]: a carry-save adder tree.
template <int D>
__device__ __forceinline__ void count_unsat(const uint64_t* e, uint64_t& u0, uint64_t& u1, uint64_t& u2) {
  const uint64_t sa = e[0] ^ e[1] ^ e[2];
  const uint64_t ca = (e[0] & e[1]) | (e[0] & e[2]) | (e[1] & e[2]);
  if (D == 3) {
    const uint64_t sb = e[3] ^ e[4] ^ e[5];
    const uint64_t cb = (e[3] & e[4]) | (e[3] & e[5]) | (e[4] & e[5]);
    u0 = sa ^ sb;
    const uint64_t k = sa & sb;
    u1 = ca ^ cb ^ k;
    u2 = (ca & cb) | (ca & k) | (cb & k);
  } else {
    u0 = sa ^ e[3];
    const uint64_t k = sa & e[3];
    u1 = ca ^ k;
    u2 = ca & k;
  }
}

// Device error word bits (read by ianus_synchronize): a PT energy difference
// off the multiple-of-4 grid (k_pt.cu), a bounded wait of the persistent
// sweep that ran out (jit_sweep_lt.cuh).
enum : uint32_t { ERR_PT_PARITY = 2u, ERR_TIMEOUT = 4u };

}  // namespace ianus
