// k_pt.cu -- kernels shared by all layouts: turning the per-configuration
// measurement accumulators into per-temperature outputs (Sec. 4.1), and the
// parallel-tempering swap step that Sec. 2.2 names as an add-on without
// giving its rules; the rule used is the standard one, with the exact
// integer energies of the configurations and an integer acceptance table.
#include "lattice.h"

namespace ianus {

namespace {

// acc row of a configuration -> its energy, by layout.
__device__ __forceinline__ long long config_energy(const int64_t* row, int mode, int D, uint32_t N) {
  if (mode == IANUS_LAYOUT_BITS64) return 2 * (long long)row[0] - (long long)D * (long long)N;
  return (long long)row[0];
}

__global__ void k_finalize(const int64_t* __restrict__ acc, const int32_t* __restrict__ slot_at, int64_t* E,
                           int64_t* M, int64_t* Q, uint64_t* sweep_out, uint64_t sweep, int S, int R, int K,
                           int slots, int mode, int D, uint32_t N, int want_q, int field) {
  const int total = S * K * R;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int a = idx % R, sk = idx / R;
    const int k = sk % K, s = sk / K;
    const int tslot = slot_at[((size_t)s * R + a) * K + k];
    const int64_t* row = acc + ((size_t)s * slots + (size_t)tslot * R + a) * kAccStride;
    if (E) E[idx] = field ? row[0] : config_energy(row, mode, D, N);
    if (M) {
      if (field) {  // M = sum x s, F = sum sign(h) x s (values in both layouts)
        M[(size_t)idx * 2] = row[1];
        M[(size_t)idx * 2 + 1] = row[2];
      } else if (mode == IANUS_LAYOUT_U8X4) {
        for (int f = 0; f < 4; ++f) M[(size_t)idx * 4 + f] = row[2 + f];
      } else if (mode == IANUS_LAYOUT_BITS64) {
        M[idx] = (int64_t)N - 2 * row[1];
      } else {
        M[idx] = row[1];
      }
    }
    if (Q && want_q && a == 0) {
      const int64_t x = acc[((size_t)s * slots + (size_t)k * R) * kAccStride + 6];
      Q[sk] = mode == IANUS_LAYOUT_BITS64 && !field ? (int64_t)N - 2 * x : x;
    }
  }
  if (sweep_out && blockIdx.x == 0 && threadIdx.x == 0) *sweep_out = sweep;
}

// One thread per chain (sample s, replica a): pairs k = 0..K-2 in order.
// Swap iff db*d <= 0, else iff r < T_PT(|d|/4); d = E_B - E_A is a multiple
// of 4 in the +-J model (checked: a violation sets ERR_PT_PARITY and rejects).
__global__ void k_pt_swap(const int64_t* __restrict__ acc, int32_t* slot_at, int32_t* temp_of,
                          uint64_t* accepted, const uint64_t* __restrict__ pttab, const int8_t* __restrict__ pt_sign,
                          uint32_t pt_len, int S, int R, int K, int slots, int mode, int D, uint32_t N,
                          uint32_t tau_lo, uint32_t tau_hi, PhiloxKeys keys, uint32_t* err) {
  const int total = S * R;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int s = idx / R, a = idx - s * R;
    int32_t* sa = slot_at + (size_t)idx * K;
    int32_t* ta = temp_of + (size_t)idx * K;
    const uint32_t c2 = (TAG_PT << 28) | ((uint32_t)a << 16) | ((uint32_t)s >> 2);
    for (int k = 0; k + 1 < K; ++k) {
      const int A = sa[k], B = sa[k + 1];
      const long long EA = config_energy(acc + ((size_t)s * slots + (size_t)A * R + a) * kAccStride, mode, D, N);
      const long long EB = config_energy(acc + ((size_t)s * slots + (size_t)B * R + a) * kAccStride, mode, D, N);
      const long long d = EB - EA;
      const int sg = pt_sign[k];
      bool swap;
      if (d == 0 || sg == 0 || ((d > 0) != (sg > 0))) {
        swap = true;
      } else {
        const unsigned long long ad = (unsigned long long)(d > 0 ? d : -d);
        if (ad & 3ull) {
          atomicOr(err, ERR_PT_PARITY);
          swap = false;
        } else {
          const unsigned long long m = ad >> 2;
          const uint64_t T = (m <= pt_len) ? pttab[(size_t)k * pt_len + (m - 1)] : 0ull;
          const uint4 x = philox10((uint32_t)k, tau_lo, c2, tau_hi, keys);
          const uint32_t sel = (uint32_t)s & 3u;
          const uint32_t r = sel == 0 ? x.x : sel == 1 ? x.y : sel == 2 ? x.z : x.w;
          swap = (uint64_t)r < T;
        }
      }
      if (swap) {
        sa[k] = B;
        sa[k + 1] = A;
        ta[B] = k;
        ta[A] = k + 1;
        accepted[(size_t)idx * (K - 1) + k] += 1;
      }
    }
  }
}

// The same step with one warp per chain (K <= 32): thread j holds the slot
// at temperature j, the temperature of slot j and the energy of slot j; the
// random words of all pairs are drawn first, in parallel (they do not depend
// on the permutation); the pairs then go in order, each decided by thread k
// and broadcast.
__global__ void k_pt_swap_warp(const int64_t* __restrict__ acc, int32_t* slot_at, int32_t* temp_of,
                               uint64_t* accepted, const uint64_t* __restrict__ pttab,
                               const int8_t* __restrict__ pt_sign, uint32_t pt_len, int S, int R, int K, int slots,
                               int mode, int D, uint32_t N, uint32_t tau_lo, uint32_t tau_hi, PhiloxKeys keys,
                               uint32_t* err) {
  const int lane = (int)(threadIdx.x & 31u);
  const int idx = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);  // uniform across the warp
  if (idx >= S * R) return;
  const int s = idx / R, a = idx - s * R;
  int32_t* sa = slot_at + (size_t)idx * K;
  int32_t* ta = temp_of + (size_t)idx * K;
  int my_sa = 0, my_ta = 0;
  long long my_E = 0;
  if (lane < K) {
    my_sa = sa[lane];
    my_ta = ta[lane];
    my_E = config_energy(acc + ((size_t)s * slots + (size_t)lane * R + a) * kAccStride, mode, D, N);
  }
  uint32_t my_r = 0;
  int my_sg = 0;
  if (lane + 1 < K) {
    const uint32_t c2 = (TAG_PT << 28) | ((uint32_t)a << 16) | ((uint32_t)s >> 2);
    const uint4 x = philox10((uint32_t)lane, tau_lo, c2, tau_hi, keys);
    const uint32_t sel = (uint32_t)s & 3u;
    my_r = sel == 0 ? x.x : sel == 1 ? x.y : sel == 2 ? x.z : x.w;
    my_sg = pt_sign[lane];
  }
  uint64_t my_acc = 0;
  for (int k = 0; k + 1 < K; ++k) {
    const int A = __shfl_sync(0xffffffffu, my_sa, k), B = __shfl_sync(0xffffffffu, my_sa, k + 1);
    const long long EA = __shfl_sync(0xffffffffu, my_E, A), EB = __shfl_sync(0xffffffffu, my_E, B);
    int swap = 0;
    if (lane == k) {
      const long long d = EB - EA;
      if (d == 0 || my_sg == 0 || ((d > 0) != (my_sg > 0))) {
        swap = 1;
      } else {
        const unsigned long long ad = (unsigned long long)(d > 0 ? d : -d);
        if (ad & 3ull) {
          atomicOr(err, ERR_PT_PARITY);
        } else {
          const unsigned long long m = ad >> 2;
          const uint64_t T = (m <= pt_len) ? __ldg(pttab + (size_t)k * pt_len + (m - 1)) : 0ull;
          swap = (uint64_t)my_r < T ? 1 : 0;
        }
      }
    }
    if (__shfl_sync(0xffffffffu, swap, k)) {
      if (lane == k) {
        my_sa = B;
        my_acc += 1;
      }
      if (lane == k + 1) my_sa = A;
      if (lane == B) my_ta = k;
      if (lane == A) my_ta = k + 1;
    }
  }
  if (lane < K) {
    sa[lane] = my_sa;
    ta[lane] = my_ta;
  }
  if (lane + 1 < K && my_acc) accepted[(size_t)idx * (K - 1) + lane] += my_acc;
}

__global__ void k_set_tick(uint64_t* t, uint64_t v) { *t = v; }
__global__ void k_advance_tick(uint64_t* t, uint64_t by) { *t += by; }

}  // namespace

cudaError_t launch_set_tick(Lattice& lat, uint64_t value) {
  k_set_tick<<<1, 1, 0, lat.stream>>>(lat.t_dev, value);
  return cudaGetLastError();
}

cudaError_t launch_advance_tick(Lattice& lat, uint64_t by) {
  k_advance_tick<<<1, 1, 0, lat.stream>>>(lat.t_dev, by);
  return cudaGetLastError();
}

cudaError_t launch_finalize(Lattice& lat, int64_t* E, int64_t* M, int64_t* Q, uint64_t* sweep_out, int want_q) {
  const int total = lat.S * lat.K * lat.R;
  const unsigned grid = (unsigned)std::min(152 * 4, (total + 255) / 256);
  k_finalize<<<grid > 0 ? grid : 1, 256, 0, lat.stream>>>(lat.acc, lat.slot_at, E, M, Q, sweep_out, lat.sweeps,
                                                         lat.S, lat.R, lat.K, lat.slots, lat.layout, lat.D, lat.N,
                                                         want_q, lat.field ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_pt_swap(Lattice& lat) {
  const int total = lat.S * lat.R;
  if (lat.K <= 32) {  // one warp per chain
    const unsigned grid = (unsigned)((total + 7) / 8);
    k_pt_swap_warp<<<grid, 256, 0, lat.stream>>>(
        lat.acc, lat.slot_at, lat.temp_of, lat.accepted, lat.pttab, lat.pt_sign, lat.pt_len, lat.S, lat.R, lat.K,
        lat.slots, lat.layout, lat.D, lat.N, (uint32_t)(lat.steps & 0xffffffffu), (uint32_t)(lat.steps >> 32),
        lat.keys, lat.err);
    return cudaGetLastError();
  }
  const unsigned grid = (unsigned)((total + 127) / 128);
  k_pt_swap<<<grid, 128, 0, lat.stream>>>(lat.acc, lat.slot_at, lat.temp_of, lat.accepted, lat.pttab, lat.pt_sign,
                                          lat.pt_len, lat.S, lat.R, lat.K, lat.slots, lat.layout, lat.D, lat.N,
                                          (uint32_t)(lat.steps & 0xffffffffu), (uint32_t)(lat.steps >> 32), lat.keys,
                                          lat.err);
  return cudaGetLastError();
}

}  // namespace ianus
