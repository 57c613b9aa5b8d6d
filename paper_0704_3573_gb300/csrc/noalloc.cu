// noalloc.cu -- ianus_measure_bits64_noalloc: energy and magnetisation of
// bit-sliced configurations for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code that runs inside a host
// framework which owns every byte of device memory through its own pool (a
// direct cudaMalloc bypasses that accounting and can fail once the pool has
// reserved the device), and latency-critical serving loops in which
// cudaMalloc / cudaFree would synchronise the device and stall every other
// stream.  This entry point needs no allocation: its per-(sample, slot)
// counters live in a file-scope device array of fixed size, and the caller
// passes device pointers for the inputs and the outputs.
//
// The array below is a host-side stand-in when named in host code; its device
// address is fetched with cudaGetSymbolAddress once per device, the first
// time the entry point runs on that device (with that device current), and
// that address is what the kernels receive.
#include <mutex>

#include "lattice.h"

namespace ianus {
namespace {

constexpr int kBlockNA = 256;
constexpr int kItersNA = 64;  // sites per thread between counter flushes (3 bonds: 192 < 256)
constexpr int kCtrNA = 8;     // vertical counter planes
constexpr int kMaxDevicesNA = 64;

// Two counters per configuration: unsatisfied forward bonds U and spin-down
// sites B.  Every loaded GPU holds these 512 KiB until the process exits.
static __device__ __align__(256) unsigned long long g_measure_scratch[2 * IANUS_NOALLOC_MAX_CONFIGS];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevicesNA];
bool g_scratch_ready[kMaxDevicesNA];

cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevicesNA) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ready[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_measure_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
    g_scratch_ready[dev] = true;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

__device__ __forceinline__ void add_plane(uint64_t* c, uint64_t x) {
#pragma unroll
  for (int k = 0; k < kCtrNA; ++k) {
    const uint64_t t = c[k] & x;
    c[k] ^= x;
    x = t;
  }
}

// Per-lane totals of a warp's vertical counters; thread t gets lanes t, t+32.
__device__ __forceinline__ void warp_totals(const uint64_t* c, unsigned long long& lo, unsigned long long& hi) {
  const int lane = threadIdx.x & 31;
  lo = hi = 0;
#pragma unroll
  for (int k = 0; k < kCtrNA; ++k) {
    const uint32_t wl = (uint32_t)c[k], wh = (uint32_t)(c[k] >> 32);
    for (int j = 0; j < 32; ++j) {
      const uint32_t bl = __ballot_sync(0xffffffffu, (wl >> j) & 1u);
      const uint32_t bh = __ballot_sync(0xffffffffu, (wh >> j) & 1u);
      if (lane == j) {
        lo += (unsigned long long)__popc(bl) << k;
        hi += (unsigned long long)__popc(bh) << k;
      }
    }
  }
}

// blockIdx.y = group * slots + slot; each block covers kBlockNA * kItersNA sites.
template <int D>
__global__ void __launch_bounds__(kBlockNA) k_measure_bits_noalloc(const uint64_t* __restrict__ spins,
                                                                   const uint64_t* __restrict__ J,
                                                                   unsigned long long* scratch, Geom geom, int S,
                                                                   int slots) {
  const int gs = blockIdx.y;
  const int g = gs / slots, sigma = gs - g * slots;
  const uint32_t N = geom.N, L = (uint32_t)geom.L, h = (uint32_t)geom.h;
  const uint64_t* Jg = J + (size_t)g * D * N;
  const uint64_t* sp = spins + ((size_t)g * slots + sigma) * N;
  const uint32_t base = blockIdx.x * (uint32_t)(kBlockNA * kItersNA);
  uint64_t cu[kCtrNA], cb[kCtrNA];
#pragma unroll
  for (int k = 0; k < kCtrNA; ++k) cu[k] = cb[k] = 0;
  for (int it = 0; it < kItersNA; ++it) {
    const uint32_t j = base + (uint32_t)it * kBlockNA + threadIdx.x;
    if (j < N) {
      const uint32_t rc = j / h, k = j - rc * h;
      const uint32_t row = rc >> 1, c = rc & 1u;
      const uint32_t y = row % L, z = row / L;
      const uint32_t x = 2u * k + ((c ^ (y + z)) & 1u);
      const uint64_t bi = sp[j];
      const uint32_t xp = (x + 1u == L) ? 0u : x + 1u;
      const uint32_t yp = (y + 1u == L) ? 0u : y + 1u;
      add_plane(cu, bi ^ sp[split_index(geom, (int)xp, (int)y, (int)z)] ^ Jg[j]);
      add_plane(cu, bi ^ sp[split_index(geom, (int)x, (int)yp, (int)z)] ^ Jg[N + j]);
      if (D == 3) {
        const uint32_t zp = (z + 1u == L) ? 0u : z + 1u;
        add_plane(cu, bi ^ sp[split_index(geom, (int)x, (int)y, (int)zp)] ^ Jg[2u * N + j]);
      }
      add_plane(cb, bi);
    }
  }
  const int lane = threadIdx.x & 31;
  const int s_lo = 64 * g + lane, s_hi = 64 * g + 32 + lane;
  unsigned long long lo, hi;
  warp_totals(cu, lo, hi);
  if (s_lo < S) atomicAdd(&scratch[2 * ((size_t)s_lo * slots + sigma)], lo);
  if (s_hi < S) atomicAdd(&scratch[2 * ((size_t)s_hi * slots + sigma)], hi);
  warp_totals(cb, lo, hi);
  if (s_lo < S) atomicAdd(&scratch[2 * ((size_t)s_lo * slots + sigma) + 1], lo);
  if (s_hi < S) atomicAdd(&scratch[2 * ((size_t)s_hi * slots + sigma) + 1], hi);
}

// E = 2U - D N and M = N - 2B per (sample, slot).
__global__ void k_finalize_noalloc(const unsigned long long* scratch, int64_t* E, int64_t* M, int total, int D,
                                   uint32_t N) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const long long U = (long long)scratch[2 * idx], B = (long long)scratch[2 * idx + 1];
    E[idx] = 2 * U - (long long)D * (long long)N;
    M[idx] = (long long)N - 2 * B;
  }
}

}  // namespace
}  // namespace ianus

using namespace ianus;

extern "C" ianus_status ianus_measure_bits64_noalloc(const uint64_t* spins, const uint64_t* couplings, int32_t dim,
                                                     int32_t L, int32_t n_samples, int32_t n_slots, int64_t* energy,
                                                     int64_t* magnetisation, void* cuda_stream) {
  if (!spins || !couplings || !energy || !magnetisation) return IANUS_EINVAL;
  if ((dim != 2 && dim != 3) || L < 2 || (L & 1) || L > 4096 || n_samples < 1 || n_slots < 1) return IANUS_EINVAL;
  if ((long long)n_samples * n_slots > IANUS_NOALLOC_MAX_CONFIGS) return IANUS_EINVAL;
  uint64_t N = 1;
  for (int d = 0; d < dim; ++d) N *= (uint64_t)L;
  if (N >= (1ull << 31)) return IANUS_EINVAL;
  const int G = (n_samples + 63) / 64;
  if ((long long)G * n_slots > 65535) return IANUS_EINVAL;
  Geom geom{};
  geom.D = dim;
  geom.L = L;
  geom.h = L / 2;
  geom.N = (uint32_t)N;
  geom.half = (uint32_t)(N / 2);
  if ((L & (L - 1)) == 0) {  // power of two: log2 of L and L/2, as the other kernels expect
    while ((1 << geom.lL) < L) ++geom.lL;
    geom.lh = geom.lL - 1;
  }
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  void* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return IANUS_ECUDA;
  const int total = n_samples * n_slots;
  // the array keeps the previous call's counts: clear the part this call uses
  if (cudaMemsetAsync(scratch, 0, (size_t)total * 2 * sizeof(unsigned long long), stream) != cudaSuccess) {
    cudaGetLastError();
    return IANUS_ECUDA;
  }
  const uint32_t per_block = kBlockNA * kItersNA;
  dim3 grid((geom.N + per_block - 1) / per_block, (unsigned)(G * n_slots));
  unsigned long long* acc = (unsigned long long*)scratch;
  // Each launch's status is its own return value, so an error left pending
  // by unrelated earlier work is neither reported here nor cleared; a
  // refused launch is cleared so that it does not linger for the next caller.
  int ns = n_samples, nsl = n_slots;
  void* margs[] = {(void*)&spins, (void*)&couplings, (void*)&acc, (void*)&geom, (void*)&ns, (void*)&nsl};
  const void* mk = dim == 3 ? (const void*)k_measure_bits_noalloc<3> : (const void*)k_measure_bits_noalloc<2>;
  if (cudaLaunchKernel(mk, grid, dim3(kBlockNA), margs, 0, stream) != cudaSuccess) {
    cudaGetLastError();
    return IANUS_ECUDA;
  }
  const unsigned fin = (unsigned)std::min(1024, (total + 255) / 256);
  const unsigned long long* cacc = acc;
  int tot = total, D = dim;
  uint32_t Nn = geom.N;
  void* fargs[] = {(void*)&cacc, (void*)&energy, (void*)&magnetisation, (void*)&tot, (void*)&D, (void*)&Nn};
  if (cudaLaunchKernel((const void*)k_finalize_noalloc, dim3(fin), dim3(256), fargs, 0, stream) != cudaSuccess) {
    cudaGetLastError();
    return IANUS_ECUDA;
  }
  return IANUS_OK;
}
