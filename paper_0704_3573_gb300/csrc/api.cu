// api.cu -- the extern "C" entry points of libianus.so (declared and
// documented in include/ianus.h): lattice set-up, the sweep loop
// (Sec. 2.2 sweeps of the two-colour update of Sec. 3.1), acceptance-table
// uploads (Sec. 3.2), measurements (Sec. 4.1), parallel tempering,
// checkpoints and error reporting.  Host logic only; all per-site work runs
// in the kernels of k_plain.cu, k_msc.cu, k_potts.cu and k_pt.cu.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "lattice.h"

using namespace ianus;

namespace {

constexpr uint32_t kDefaultSeries = 1024;
constexpr uint32_t kPtCapMax = 4096;
constexpr uint64_t kStateMagic = 0x31534e4149ull;  // "IANS1"

struct Sizes {
  int model, D, L, S, R, K, slots, layout, G, Q4, mq;
  uint32_t N, cap, pt_cap;
  bool field;
  int fpc;
  uint32_t rows;
  size_t off_wheels, wheel_bytes;
  bool poolable;
  size_t off_segs, off_nseg;
  size_t off_spins, off_J, off_thr, off_tp, off_fthr, off_ftp, off_sites, off_ptab, off_pttab, off_ptsign, off_slot,
      off_temp, off_acc_pt, off_acc, off_oE, off_oM, off_oQ, off_sw, off_sE, off_sM, off_sQ, off_err, off_tdev, off_flags, total;
  size_t spins_bytes, J_bytes, sites_bytes;
};

constexpr size_t kMaxSmemPerBlock = 227 * 1024;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Validates cfg and lays out the device buffer.  Returns IANUS_OK or an error.
int plan(const ianus_config* c, Sizes& z) {
  if (!c) return IANUS_EINVAL;
  if (c->abi_version != IANUS_ABI_VERSION) return IANUS_EINVAL;
  if (c->model != IANUS_EA_PM_J && c->model != IANUS_POTTS4_J && c->model != IANUS_POTTS4_PERM) return IANUS_EINVAL;
  if (c->dim != 2 && c->dim != 3 && !(c->dim == 4 && c->model == IANUS_POTTS4_PERM)) return IANUS_EINVAL;
  if (c->L < 2 || (c->L & 1) || c->L > 4096) return IANUS_EINVAL;
  if (c->n_samples < 1 || c->n_samples >= (1 << 18)) return IANUS_EINVAL;
  if (c->n_replicas < 1 || c->n_temps < 1) return IANUS_EINVAL;
  if ((long long)c->n_replicas * c->n_temps >= 4096) return IANUS_EINVAL;
  if (c->disorder < IANUS_DISORDER_PM_J || c->disorder > IANUS_DISORDER_DAFF) return IANUS_EINVAL;
  const bool field = c->disorder == IANUS_DISORDER_RFIM || c->disorder == IANUS_DISORDER_DAFF;
  if (!std::isfinite(c->field) || c->field < 0.0) return IANUS_EINVAL;
  if (!field && c->field != 0.0) return IANUS_EINVAL;
  if (c->disorder == IANUS_DISORDER_DAFF && !(c->occupation >= 0.0 && c->occupation <= 1.0)) return IANUS_EINVAL;
  if (field && c->model != IANUS_EA_PM_J) return IANUS_EINVAL;
  if (c->rng != IANUS_RNG_PHILOX && c->rng != IANUS_RNG_WHEEL) return IANUS_EINVAL;
  uint64_t N = 1;
  for (int d = 0; d < c->dim; ++d) N *= (uint64_t)c->L;
  if (N >= (1ull << 31)) return IANUS_EINVAL;
  int layout = c->layout;
  const bool potts = c->model != IANUS_EA_PM_J;
  if (layout == IANUS_LAYOUT_AUTO)
    layout = potts ? IANUS_LAYOUT_U8X4
             : c->rng == IANUS_RNG_WHEEL ? IANUS_LAYOUT_I8
                                         : IANUS_LAYOUT_BITS64;
  if (layout < IANUS_LAYOUT_I8 || layout > IANUS_LAYOUT_U8X4) return IANUS_EINVAL;
  if (!potts && layout == IANUS_LAYOUT_U8X4) return IANUS_EUNSUPPORTED;
  if (potts && layout != IANUS_LAYOUT_U8X4) return IANUS_EUNSUPPORTED;
  if (c->rng == IANUS_RNG_WHEEL && (potts || layout != IANUS_LAYOUT_I8)) return IANUS_EUNSUPPORTED;
  if (layout == IANUS_LAYOUT_BITS64 &&  // the sweep stages one block's threshold planes in shared memory
      (!field ? sweep_bits_smem(c->n_replicas)
              : (size_t)c->n_replicas * kPlanes *
                    (c->disorder == IANUS_DISORDER_DAFF ? kDiluteClasses : kFieldPlaneClasses) * 8) > kMaxSmemPerBlock)
    return IANUS_EUNSUPPORTED;
  z.model = c->model;
  z.D = c->dim;
  z.L = c->L;
  z.S = c->n_samples;
  z.R = c->n_replicas;
  z.K = c->n_temps;
  z.slots = z.R * z.K;
  z.layout = layout;
  z.N = (uint32_t)N;
  z.G = (z.S + 63) / 64;
  z.Q4 = (z.S + 3) / 4;
  z.field = field;
  z.mq = potts ? 4 : (field ? 2 : 1);
  z.cap = c->series_capacity ? c->series_capacity : kDefaultSeries;
  z.pt_cap = z.K > 1 ? (uint32_t)std::min<uint64_t>((uint64_t)z.D * N / 2 + 1, kPtCapMax) : 0;
  if (layout == IANUS_LAYOUT_I8) {
    z.spins_bytes = (size_t)z.slots * z.S * N;
    z.J_bytes = (size_t)z.S * z.D * N;
  } else if (layout == IANUS_LAYOUT_BITS64) {
    z.spins_bytes = (size_t)z.G * z.slots * N * 8;
    z.J_bytes = (size_t)z.G * z.D * N * 8;
  } else {
    z.spins_bytes = (size_t)z.slots * z.Q4 * N * 4;
    z.J_bytes = (size_t)z.Q4 * z.D * N * 4;
  }
  // I8: hs, occ int8 [S][N]; BITS64: hbits, xbits u64 [G][N]
  z.sites_bytes = !field ? 0 : layout == IANUS_LAYOUT_I8 ? (size_t)2 * z.S * N : (size_t)2 * z.G * N * 8;
  z.fpc = c->disorder == IANUS_DISORDER_DAFF ? kDiluteClasses : kFieldPlaneClasses;
  z.rows = (uint32_t)(N / (uint64_t)c->L);
  z.wheel_bytes = c->rng == IANUS_RNG_WHEEL ? (size_t)z.slots * z.S * 2 * 64 * z.rows * 4 : 0;
  const size_t SKR = (size_t)z.S * z.K * z.R;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += align256(bytes);
    return at;
  };
  z.off_spins = take(z.spins_bytes);
  z.off_J = take(z.J_bytes);
  z.off_thr = take((size_t)z.K * kMaxClasses * 8 + sizeof(UniformLut));  // class thresholds, then the uniform tables
  z.off_tp = take(layout == IANUS_LAYOUT_BITS64 && !field ? (size_t)z.G * z.slots * kPlanes * kMaxClasses * 8 : 0);
  z.off_fthr = take(field ? (size_t)z.K * kFieldClasses * 8 + sizeof(FieldLut) : 0);  // then the uniform tables
  z.off_ftp = take(field && layout == IANUS_LAYOUT_BITS64 ? (size_t)z.G * z.slots * kPlanes * z.fpc * 8 : 0);
  z.off_sites = take(z.sites_bytes);
  z.off_wheels = take(z.wheel_bytes);
  // segment tables for fused serving: bit-sliced EA lattices with one replica
  // and one temperature
  z.poolable = !potts && !field && layout == IANUS_LAYOUT_BITS64 && z.R == 1 && z.K == 1;
  z.off_segs = take(z.poolable ? (size_t)z.G * kMaxSegs * sizeof(Segment) : 0);
  z.off_nseg = take(z.poolable ? (size_t)z.G * 4 : 0);
  z.off_ptab = take(layout != IANUS_LAYOUT_U8X4 ? 0
                    : c->model == IANUS_POTTS4_PERM ? (size_t)z.K * perm_table_entries(z.D) * 16
                                                    : (size_t)z.K * 65536 * 16);
  z.off_pttab = take((size_t)std::max(z.K - 1, 0) * z.pt_cap * 8);
  z.off_ptsign = take((size_t)std::max(z.K - 1, 1));
  z.off_slot = take((size_t)z.S * z.R * z.K * 4 * 2);  // slot_at then temp_of
  z.off_temp = z.off_slot + (size_t)z.S * z.R * z.K * 4;
  z.off_acc_pt = take((size_t)z.S * z.R * std::max(z.K - 1, 1) * 8);
  z.off_acc = take((size_t)z.S * z.slots * kAccStride * 8);
  z.off_oE = take(SKR * 8);
  z.off_oM = take(SKR * z.mq * 8);
  z.off_oQ = take((size_t)z.S * z.K * 8);
  z.off_sw = take((size_t)z.cap * 8);
  z.off_sE = take((size_t)z.cap * SKR * 8);
  z.off_sM = take((size_t)z.cap * SKR * z.mq * 8);
  z.off_sQ = take((size_t)z.cap * z.S * z.K * 8);
  z.off_err = take(8);
  z.off_tdev = take(8);
  // progress flags of the persistent one-temperature bit-sliced sweep
  z.off_flags = take(layout == IANUS_LAYOUT_BITS64 && !field && z.K == 1 ? (size_t)kMaxPersistBlocks * 4 : 0);
  z.total = o;
  return IANUS_OK;
}

// A failure code usable as the return value of both the int helpers and the
// ianus_status entry points.
struct Fail {
  int v;
  operator int() const { return v; }
  operator ianus_status() const { return (ianus_status)v; }
};

Fail fail(Lattice* lat, int st) {
  if (lat && st == IANUS_ECUDA) lat->sticky = IANUS_ESTATE;
  return Fail{st};
}

#define CK(expr)                                     \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return fail(lat, IANUS_ECUDA); \
  } while (0)

void drop_graphs(Lattice* lat);

}  // namespace

// Bit c of t[q] is bit 31 - q of class c's threshold; `always` marks the
// classes that flip whatever the random number (threshold 2^32), `need` the
// classes whose comparison decides the flip.
UniformLut ianus::uniform_lut(int dim, int algo, const uint64_t* thr) {
  UniformLut u{};
  uint32_t always = 0, cmp = 0;
  for (int c = 0; c <= 2 * dim; ++c) {
    const uint64_t T = thr[c];
    if (T >= kTwo32) always |= 1u << c;
    else if (algo == IANUS_HEATBATH || c < dim) cmp |= 1u << c;
    for (int q = 0; q < 32; ++q)
      if (T < kTwo32 && ((T >> (31 - q)) & 1ull)) u.t[q] |= (uint8_t)(1u << c);
  }
  u.always = (uint8_t)always;
  u.need = (uint8_t)cmp;
  return u;
}

namespace {

bool beta_ok(const double* beta, int K) {
  for (int k = 0; k < K; ++k)
    if (!std::isfinite(beta[k]) || beta[k] < 0.0) return false;
  return true;
}

// Rebuild and upload the acceptance tables for (algo, beta).
int upload_tables(Lattice* lat, int algo, const double* beta) {
  const int K = lat->K;
  if (lat->field) {
    std::vector<uint64_t> fthr((size_t)K * kFieldClasses);
    for (int k = 0; k < K; ++k) field_thresholds(lat->D, algo, beta[k], lat->hmag, &fthr[(size_t)k * kFieldClasses]);
    CK(cudaMemcpyAsync(lat->fthr, fthr.data(), fthr.size() * 8, cudaMemcpyHostToDevice, lat->stream));
    if (lat->layout == IANUS_LAYOUT_BITS64) CK(launch_build_field_planes(*lat));
    lat->ulut_ok = false;
    lat->jit = nullptr;
    lat->jit_algo = -1;
    lat->flut_ok = false;
    lat->jitf = nullptr;
    lat->jitf_algo = -1;
    if (K == 1 && lat->layout == IANUS_LAYOUT_BITS64) {
      // one temperature: the truth tables of the specialised field kernel.
      // Without dilution the class is (u, f), field class (v + 2D) * 2 + f
      // with v = 2D - 2u, tables [f][0] bit u.  With dilution it is (t, f),
      // t = v + 2D = 8 t3 + k, tables [f][t3] bit k.
      FieldLut fl{};
      for (int f = 0; f < 2; ++f)
        for (int cls = 0; cls <= (lat->dilute ? 4 * lat->D : 2 * lat->D); ++cls) {
          const int t = lat->dilute ? cls : 4 * lat->D - 2 * cls;
          const int hi = lat->dilute ? (cls >> 3) : 0, bit = lat->dilute ? (cls & 7) : cls;
          const uint64_t T = fthr[(size_t)t * 2 + f];
          if (T >= kTwo32) {
            fl.always[f][hi] |= (uint8_t)(1u << bit);
          } else {
            fl.need[f][hi] |= (uint8_t)(1u << bit);
            for (int q = 0; q < 32; ++q)
              if ((T >> (31 - q)) & 1ull) fl.t[f][hi][q] |= (uint8_t)(1u << bit);
          }
        }
      lat->flut = fl;
      CK(cudaMemcpyAsync(lat->fthr + (size_t)K * kFieldClasses, &lat->flut, sizeof(FieldLut), cudaMemcpyHostToDevice,
                         lat->stream));
      lat->flut_ok = true;
    }
  } else if (lat->model == IANUS_EA_PM_J) {
    std::vector<uint64_t> thr((size_t)K * kMaxClasses);
    for (int k = 0; k < K; ++k) class_thresholds(lat->D, algo, beta[k], &thr[(size_t)k * kMaxClasses]);
    CK(cudaMemcpyAsync(lat->thr, thr.data(), thr.size() * 8, cudaMemcpyHostToDevice, lat->stream));
    if (lat->layout == IANUS_LAYOUT_BITS64) CK(launch_build_planes(*lat));
    lat->ulut_ok = false;
    if (K == 1) {
      lat->ulut = uniform_lut(lat->D, algo, thr.data());
      CK(cudaMemcpyAsync(lat->thr + (size_t)K * kMaxClasses, &lat->ulut, sizeof(UniformLut), cudaMemcpyHostToDevice,
                         lat->stream));
      lat->ulut_ok = true;
    }
    lat->jit = nullptr;  // specialised lazily by the first launch that wants it
    lat->jit_algo = -1;
  } else if (lat->model == IANUS_POTTS4_PERM) {
    // compact table of the permutation model: counts n_k in 0..2D with
    // n0 + n1 + n2 + n3 = 2D, entry n0 + B (n1 + B n2), B = 2D + 1
    const int D = lat->D, B = 2 * D + 1;
    for (int k = 0; k < K; ++k)
      if (2.0 * D * beta[k] > 700.0) return IANUS_EINVAL;  // exp(2D beta) must stay finite
    const uint32_t NT = perm_table_entries(D);
    std::vector<uint4> tab((size_t)K * NT);
    std::memset(tab.data(), 0, tab.size() * sizeof(uint4));
    for (int k = 0; k < K; ++k)
      for (int n0 = 0; n0 <= 2 * D; ++n0)
        for (int n1 = 0; n0 + n1 <= 2 * D; ++n1)
          for (int n2 = 0; n0 + n1 + n2 <= 2 * D; ++n2) {
            const int n[4] = {n0, n1, n2, 2 * D - n0 - n1 - n2};
            uint64_t T[3];
            potts_thresholds(beta[k], n, T);
            uint4 e;
            e.x = (uint32_t)T[0];
            e.y = (uint32_t)T[1];
            e.z = (uint32_t)T[2];
            e.w = (T[0] >= kTwo32 ? 1u : 0u) | (T[1] >= kTwo32 ? 2u : 0u) | (T[2] >= kTwo32 ? 4u : 0u);
            tab[(size_t)k * NT + n0 + B * (n1 + B * n2)] = e;
          }
    CK(cudaMemcpyAsync(lat->ptab, tab.data(), tab.size() * sizeof(uint4), cudaMemcpyHostToDevice, lat->stream));
  } else {
    if (beta_ok(beta, K)) {
      for (int k = 0; k < K; ++k)
        if (beta[k] > 100.0) return IANUS_EINVAL;  // exp(6 beta) must stay finite
    }
    std::vector<uint64_t> flat(3u * 28561u);
    std::vector<uint4> tab((size_t)K * 65536);
    std::memset(tab.data(), 0, tab.size() * sizeof(uint4));
    for (int k = 0; k < K; ++k) {
      table_potts(beta[k], flat.data(), flat.size());
      size_t idx = 0;
      for (int n0 = 0; n0 < 13; ++n0)
        for (int n1 = 0; n1 < 13; ++n1)
          for (int n2 = 0; n2 < 13; ++n2)
            for (int n3 = 0; n3 < 13; ++n3, ++idx) {
              const uint32_t key = (uint32_t)n0 | ((uint32_t)n1 << 4) | ((uint32_t)n2 << 8) | ((uint32_t)n3 << 12);
              uint4 e;
              const uint64_t t0 = flat[3 * idx], t1 = flat[3 * idx + 1], t2 = flat[3 * idx + 2];
              e.x = (uint32_t)t0;
              e.y = (uint32_t)t1;
              e.z = (uint32_t)t2;
              e.w = (t0 >= kTwo32 ? 1u : 0u) | (t1 >= kTwo32 ? 2u : 0u) | (t2 >= kTwo32 ? 4u : 0u);
              tab[(size_t)k * 65536 + key] = e;
            }
    }
    CK(cudaMemcpyAsync(lat->ptab, tab.data(), tab.size() * sizeof(uint4), cudaMemcpyHostToDevice, lat->stream));
  }
  if (K > 1 && lat->model == IANUS_EA_PM_J && !lat->field) {
    // PT tables: T(m) for |d| = 4m until the first zero (or the largest
    // possible |d|/4 = D N / 2).
    std::vector<uint64_t> pt((size_t)(K - 1) * lat->pt_cap, 0);
    std::vector<int8_t> sign((size_t)K - 1);
    uint32_t len = 1;
    const uint64_t mmax = (uint64_t)lat->D * lat->N / 2;
    for (int k = 0; k + 1 < K; ++k) {
      const double db = beta[k] - beta[k + 1];
      sign[k] = db > 0 ? 1 : (db < 0 ? -1 : 0);
      if (sign[k] == 0) continue;
      std::vector<uint64_t> col(lat->pt_cap);
      table_pt(beta[k], beta[k + 1], col.data(), col.size());
      uint32_t m = 0;
      while (m < lat->pt_cap && m < mmax && col[m] != 0) ++m;
      if (m == lat->pt_cap && m < mmax) return IANUS_EUNSUPPORTED;  // temperatures too close for the table
      for (uint32_t q = 0; q < m; ++q) pt[(size_t)k * lat->pt_cap + q] = col[q];
      len = std::max(len, m);
    }
    lat->pt_len = lat->pt_cap;  // rows are stored with stride pt_cap; zeros end each row
    (void)len;
    CK(cudaMemcpyAsync(lat->pttab, pt.data(), pt.size() * 8, cudaMemcpyHostToDevice, lat->stream));
    CK(cudaMemcpyAsync(lat->pt_sign, sign.data(), sign.size(), cudaMemcpyHostToDevice, lat->stream));
  }
  lat->beta.assign(beta, beta + K);
  lat->algo = algo;
  lat->tables_ok = true;
  drop_graphs(lat);  // captured kernels depend on the tables and the algorithm
  return IANUS_OK;
}

void acc_fresh(Lattice* lat) {
  lat->acc_ok = true;
  lat->acc_sweeps = lat->sweeps;
  lat->acc_mut = lat->mut;
}

int measure_into(Lattice* lat, int64_t* E, int64_t* M, int64_t* Q, uint64_t* sweep_out, int want_q) {
  want_q = want_q && lat->R >= 2;
  if (lat->layout == IANUS_LAYOUT_I8)
    CK(launch_measure_i8(*lat, want_q));
  else if (lat->layout == IANUS_LAYOUT_BITS64)
    CK(launch_measure_bits(*lat, want_q));
  else
    CK(launch_measure_potts(*lat, want_q));
  acc_fresh(lat);
  CK(launch_finalize(*lat, E, M, Q, sweep_out, want_q));
  return IANUS_OK;
}

int record_row(Lattice* lat) {
  const size_t SKR = (size_t)lat->S * lat->K * lat->R;
  const size_t row = (size_t)(lat->ser_count % lat->cap);
  int st = measure_into(lat, lat->ser_E + row * SKR, lat->ser_M + row * SKR * lat->mq,
                        lat->ser_Q + row * (size_t)lat->S * lat->K, lat->ser_sweep + row, 1);
  if (st) return st;
  lat->ser_count += 1;
  return IANUS_OK;
}

int one_sweep(Lattice* lat, int inv) {
  const uint64_t t = lat->sweeps;
  for (int c = 0; c < 2; ++c) {
    if (lat->layout == IANUS_LAYOUT_I8)
      CK(launch_sweep_i8(*lat, c, t, inv));
    else if (lat->layout == IANUS_LAYOUT_BITS64)
      CK(launch_sweep_bits(*lat, c, t, inv));
    else
      CK(launch_sweep_potts(*lat, c, t));
  }
  lat->sweeps += 1;
  return IANUS_OK;
}

bool same_beta(const Lattice* lat, const double* beta) {
  if ((int)lat->beta.size() != lat->K) return false;
  for (int k = 0; k < lat->K; ++k)
    if (std::memcmp(&lat->beta[k], &beta[k], sizeof(double)) != 0) return false;
  return true;
}

int do_pt_swap(Lattice* lat) {
  // energies of every configuration: those of the last measurement when no
  // sweep or other change came after it, else measured (U only when
  // bit-sliced)
  if (!(lat->acc_ok && lat->acc_sweeps == lat->sweeps && lat->acc_mut == lat->mut)) {
    if (lat->layout == IANUS_LAYOUT_BITS64)
      CK(launch_measure_bits(*lat, 0, true));
    else
      CK(launch_measure_i8(*lat, 0));
    acc_fresh(lat);
  }
  CK(launch_pt_swap(*lat));
  lat->steps += 1;
  if (lat->layout == IANUS_LAYOUT_BITS64) CK(launch_build_planes(*lat));
  return IANUS_OK;
}

// ---- CUDA graphs of sweep blocks ----

void drop_graphs(Lattice* lat) {
  if (!lat->graphs) return;
  for (auto& kv : *lat->graphs) cudaGraphExecDestroy(kv.second);
  lat->graphs->clear();
}

// Captures B sweeps (2B colour kernels reading the device sweep counter at
// offsets 0..B-1) and the counter advance on a private stream.
int build_graph(Lattice* lat, int inv, uint32_t B, cudaGraphExec_t* out) {
  if (lat->layout == IANUS_LAYOUT_BITS64) prepare_sweep_bits(*lat, inv);  // compile before capturing
  if (!lat->cap_stream) CK(cudaStreamCreateWithFlags(&lat->cap_stream, cudaStreamNonBlocking));
  cudaStream_t user = lat->stream;
  lat->stream = lat->cap_stream;
  lat->capturing = true;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(lat->cap_stream, cudaStreamCaptureModeThreadLocal);
  for (uint32_t s = 0; e == cudaSuccess && s < B; ++s)
    for (int c = 0; e == cudaSuccess && c < 2; ++c) {
      if (lat->layout == IANUS_LAYOUT_I8)
        e = launch_sweep_i8(*lat, c, s, inv);
      else if (lat->layout == IANUS_LAYOUT_BITS64)
        e = launch_sweep_bits(*lat, c, s, inv);
      else
        e = launch_sweep_potts(*lat, c, s);
    }
  if (e == cudaSuccess) e = launch_advance_tick(*lat, B);
  cudaError_t e2 = cudaStreamEndCapture(lat->cap_stream, &g);
  lat->stream = user;
  lat->capturing = false;
  if (e != cudaSuccess || e2 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return IANUS_ECUDA;
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e == cudaSuccess ? IANUS_OK : fail(lat, IANUS_ECUDA);
}

// Runs n sweeps (no measurement inside) through cached graphs of blocks of
// up to 64 sweeps; short runs (< 4 sweeps) launch eagerly.
// Sweeps per launch of the resident bit-sliced sweep: long enough that the
// launch costs nothing, short enough that no launch runs for long.
constexpr uint32_t kResidentBlock = 4096;

int sweeps_graphed(Lattice* lat, int inv, uint64_t n) {
  // small bit-sliced lattices under the automatic variant: resident sweeps,
  // many per launch, the lattice in shared memory
  if (n >= 2 && lat->use_resident && lat->variant == 0 && resident_bits_fits(*lat)) {
    while (n > 0) {
      const uint32_t B = (uint32_t)std::min<uint64_t>(n, kResidentBlock);
      CK(launch_resident_bits(*lat, inv, lat->sweeps, B));
      lat->sweeps += B;
      lat->t_dev_valid = false;
      n -= B;
    }
    return IANUS_OK;
  }
  // the persistent one-temperature sweep: all n sweeps in launches of up to
  // 2^20 sweeps, no graphs needed (falls through when it cannot run)
  if (lat->layout == IANUS_LAYOUT_BITS64 && persistent_variant(*lat)) {
    bool ran = true;
    while (n > 0 && ran) {
      const uint32_t B = (uint32_t)std::min<uint64_t>(n, 1u << 20);
      cudaError_t e = launch_sweep_persistent(*lat, inv, lat->sweeps, B, &ran);
      if (e != cudaSuccess) return fail(lat, IANUS_ECUDA);
      if (!ran) break;
      lat->sweeps += B;
      lat->t_dev_valid = false;
      n -= B;
    }
    if (n == 0) return IANUS_OK;
  }
  while (n > 0) {
    const uint32_t B = (uint32_t)std::min<uint64_t>(n, 64);
    if (B < 4 || !lat->use_graphs || !lat->graphs) {
      for (uint32_t s = 0; s < B; ++s) {
        int st = one_sweep(lat, inv);
        if (st) return st;
      }
      lat->t_dev_valid = false;
      n -= B;
      continue;
    }
    auto it = lat->graphs->find(B);
    if (it == lat->graphs->end()) {
      cudaGraphExec_t ex = nullptr;
      int st = build_graph(lat, inv, B, &ex);
      if (st) return st;
      it = lat->graphs->emplace(B, ex).first;
    }
    if (!lat->t_dev_valid) CK(launch_set_tick(*lat, lat->sweeps));
    CK(cudaGraphLaunch(it->second, lat->stream));
    lat->sweeps += B;
    lat->t_dev_valid = true;  // the graph advanced the counter by B
    n -= B;
  }
  return IANUS_OK;
}

struct StateHeader {
  uint64_t magic;
  uint32_t version, model, dim, L, S, R, K, layout, disorder, pad;
  uint64_t seed, sweeps, steps, spins_bytes, J_bytes, sites_bytes, wheel_bytes;
  double field, occupation;
};

}  // namespace

extern "C" {

size_t ianus_required_bytes(const ianus_config* cfg) {
  Sizes z;
  if (plan(cfg, z) != IANUS_OK) return 0;
  return z.total;
}

ianus_status ianus_lattice_create(const ianus_config* cfg, ianus_lattice** out) {
  if (!out) return IANUS_EINVAL;
  *out = nullptr;
  Sizes z;
  int st = plan(cfg, z);
  if (st) return (ianus_status)st;
  Lattice* lat = new (std::nothrow) Lattice();
  if (!lat) return IANUS_ENOMEM;
  lat->cfg = *cfg;
  lat->model = z.model;
  lat->D = z.D;
  lat->L = z.L;
  lat->S = z.S;
  lat->R = z.R;
  lat->K = z.K;
  lat->slots = z.slots;
  lat->layout = z.layout;
  lat->G = z.G;
  lat->Q4 = z.Q4;
  lat->N = z.N;
  lat->mq = z.mq;
  lat->disorder = cfg->disorder;
  lat->field = z.field;
  lat->hmag = cfg->field;
  lat->rng = cfg->rng;
  lat->rows = z.rows;
  lat->cap = z.cap;
  lat->pt_cap = z.pt_cap;
  lat->pt_len = z.pt_cap;
  lat->geom.D = z.D;
  lat->geom.L = z.L;
  lat->geom.h = z.L / 2;
  lat->geom.lh = lat->geom.lL = 0;
  if ((z.L & (z.L - 1)) == 0) {  // power of two: shift-based index arithmetic
    while ((1 << lat->geom.lL) < z.L) ++lat->geom.lL;
    lat->geom.lh = lat->geom.lL - 1;
  }
  lat->geom.N = z.N;
  lat->geom.half = z.N / 2;
  lat->stream = (cudaStream_t)cfg->cuda_stream;
  lat->keys = make_keys(cfg->seed);
  if (cudaGetDevice(&lat->dev) != cudaSuccess) {
    cudaGetLastError();
    lat->dev = 0;
  }
  lat->algo = -1;
  lat->jit_algo = -1;
  lat->jit_variant = -1;
  lat->persist_timeout_ns = 2000000000ull;  // 2 s
  lat->persist_absent = -1;
  lat->jitf_algo = -1;
  lat->jitp[0] = lat->jitp[1] = nullptr;
  lat->jitp_tried[0] = lat->jitp_tried[1] = false;
  lat->mut = 0;
  lat->acc_ok = false;
  lat->bytes = z.total;
  if (cfg->device_buffer) {
    if (cfg->device_buffer_bytes < z.total || ((uintptr_t)cfg->device_buffer & 255u)) {
      delete lat;
      return IANUS_EINVAL;
    }
    lat->base = (uint8_t*)cfg->device_buffer;
    lat->owns_buffer = false;
  } else {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, z.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete lat;
      return e == cudaErrorMemoryAllocation ? IANUS_ENOMEM : IANUS_ECUDA;
    }
    lat->base = (uint8_t*)p;
    lat->owns_buffer = true;
  }
  uint8_t* b = lat->base;
  lat->spins = b + z.off_spins;
  lat->J = b + z.off_J;
  lat->thr = (uint64_t*)(b + z.off_thr);
  lat->tp = (uint64_t*)(b + z.off_tp);
  lat->fthr = (uint64_t*)(b + z.off_fthr);
  lat->ftp = (uint64_t*)(b + z.off_ftp);
  lat->hs = z.field && z.layout == IANUS_LAYOUT_I8 ? (int8_t*)(b + z.off_sites) : nullptr;
  lat->occ = z.field && z.layout == IANUS_LAYOUT_I8 ? (int8_t*)(b + z.off_sites) + (size_t)z.S * z.N : nullptr;
  lat->hbits = z.field && z.layout == IANUS_LAYOUT_BITS64 ? (uint64_t*)(b + z.off_sites) : nullptr;
  lat->xbits = lat->hbits ? lat->hbits + (size_t)z.G * z.N : nullptr;
  lat->dilute = z.field && z.layout == IANUS_LAYOUT_BITS64 && cfg->disorder == IANUS_DISORDER_DAFF;
  lat->fpc = z.fpc;
  lat->wheels = z.wheel_bytes ? (uint32_t*)(b + z.off_wheels) : nullptr;
  lat->segs = z.poolable ? (Segment*)(b + z.off_segs) : nullptr;
  lat->nseg = z.poolable ? (uint32_t*)(b + z.off_nseg) : nullptr;
  lat->ptab = (uint4*)(b + z.off_ptab);
  lat->pttab = (uint64_t*)(b + z.off_pttab);
  lat->pt_sign = (int8_t*)(b + z.off_ptsign);
  lat->slot_at = (int32_t*)(b + z.off_slot);
  lat->temp_of = (int32_t*)(b + z.off_temp);
  lat->accepted = (uint64_t*)(b + z.off_acc_pt);
  lat->acc = (int64_t*)(b + z.off_acc);
  lat->out_E = (int64_t*)(b + z.off_oE);
  lat->out_M = (int64_t*)(b + z.off_oM);
  lat->out_Q = (int64_t*)(b + z.off_oQ);
  lat->ser_sweep = (uint64_t*)(b + z.off_sw);
  lat->ser_E = (int64_t*)(b + z.off_sE);
  lat->ser_M = (int64_t*)(b + z.off_sM);
  lat->ser_Q = (int64_t*)(b + z.off_sQ);
  lat->err = (uint32_t*)(b + z.off_err);
  lat->flags = (z.layout == IANUS_LAYOUT_BITS64 && !z.field && z.K == 1) ? (uint32_t*)(b + z.off_flags) : nullptr;
  lat->t_dev = (uint64_t*)(b + z.off_tdev);
  lat->use_graphs = true;
  lat->use_resident = true;
  lat->resident_mode = 1;
  lat->graphs = new (std::nothrow) std::map<uint32_t, cudaGraphExec_t>();

  auto bail = [&](int code) {
    if (lat->owns_buffer) cudaFree(lat->base);
    delete lat->graphs;
    delete lat;
    return (ianus_status)code;
  };
  if (z.poolable) {
    lat->segs_host = new (std::nothrow) std::vector<Segment>((size_t)z.G * kMaxSegs);
    lat->nseg_host = new (std::nothrow) std::vector<uint32_t>((size_t)z.G, 0u);
    lat->tp_host = new (std::nothrow) std::vector<uint64_t>((size_t)z.G * kPlanes * kMaxClasses, 0ull);
    if (!lat->segs_host || !lat->nseg_host || !lat->tp_host) {
      delete lat->segs_host;
      delete lat->nseg_host;
      delete lat->tp_host;
      return bail(IANUS_ENOMEM);
    }
  }
  if (cudaMemsetAsync(lat->base, 0, z.total, lat->stream) != cudaSuccess) return bail(IANUS_ECUDA);
  {
    std::vector<int32_t> perm((size_t)z.S * z.R * z.K);
    for (size_t c = 0; c < perm.size(); ++c) perm[c] = (int32_t)(c % z.K);
    if (cudaMemcpyAsync(lat->slot_at, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice, lat->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(lat->temp_of, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice, lat->stream) !=
            cudaSuccess)
      return bail(IANUS_ECUDA);
  }
  // couplings: the J stream (EA), +1 (ferromagnet, RFIM) or -1 (DAFF)
  const int jmode = cfg->disorder == IANUS_DISORDER_PM_J ? 0 : (cfg->disorder == IANUS_DISORDER_DAFF ? 2 : 1);
  cudaError_t e;
  if (lat->layout == IANUS_LAYOUT_I8)
    e = launch_init_i8(*lat, jmode);
  else if (lat->layout == IANUS_LAYOUT_BITS64)
    e = launch_init_bits(*lat, jmode);
  else
    e = launch_init_potts(*lat, jmode);
  if (e == cudaSuccess && lat->field)
    e = lat->layout == IANUS_LAYOUT_I8 ? launch_init_sites_i8(*lat, cfg->occupation)
                                       : launch_init_sites_bits(*lat, cfg->occupation);
  if (e == cudaSuccess && lat->wheels) e = launch_init_wheels(*lat);
  if (e != cudaSuccess || cudaStreamSynchronize(lat->stream) != cudaSuccess) return bail(IANUS_ECUDA);
  *out = reinterpret_cast<ianus_lattice*>(lat);
  return IANUS_OK;
}

#define GET_LAT(h)                                          \
  Lattice* lat = reinterpret_cast<Lattice*>(h);             \
  if (!lat) return IANUS_EINVAL;                            \
  if (lat->sticky) return (ianus_status)lat->sticky;

ianus_status ianus_sweep(ianus_lattice* h, int32_t algo, const double* beta, uint64_t nsweeps,
                         uint32_t measure_every) {
  GET_LAT(h);
  if (lat->pool) return IANUS_EINVAL;  // a pool is driven by ianus_sweep_segments
  if (!beta || (algo != IANUS_METROPOLIS && algo != IANUS_HEATBATH)) return IANUS_EINVAL;
  if (!beta_ok(beta, lat->K)) return IANUS_EINVAL;
  if (lat->model != IANUS_EA_PM_J && algo == IANUS_METROPOLIS) return IANUS_EUNSUPPORTED;
  if (!lat->tables_ok || lat->algo != algo || !same_beta(lat, beta)) {
    int st = upload_tables(lat, algo, beta);
    if (st) return (ianus_status)st;
  }
  const int inv = algo == IANUS_HEATBATH;
  if (lat->use_resident && resident_i8_fits(*lat) && (lat->R == 1 || measure_every == 0) && nsweeps >= 2) {
    // small plain lattice: whole configurations in shared memory, many sweeps per launch
    uint64_t left = nsweeps;
    while (left > 0) {
      const uint32_t n = (uint32_t)std::min<uint64_t>(left, 65536);
      CK(launch_resident_i8(*lat, inv, n, measure_every));
      if (measure_every)  // measured sweeps t+1 in (sweeps, sweeps + n] with (t+1) % every == 0
        lat->ser_count += (lat->sweeps + n) / measure_every - lat->sweeps / measure_every;
      lat->sweeps += n;
      lat->t_dev_valid = false;
      left -= n;
    }
    return IANUS_OK;
  }
  uint64_t left = nsweeps;
  while (left > 0) {
    uint64_t chunk = left;  // sweeps up to the next measurement point
    if (measure_every) chunk = std::min<uint64_t>(chunk, measure_every - lat->sweeps % measure_every);
    int st = sweeps_graphed(lat, inv, chunk);
    if (st) return (ianus_status)st;
    left -= chunk;
    if (measure_every && lat->sweeps % measure_every == 0) {
      st = record_row(lat);
      if (st) return (ianus_status)st;
    }
  }
  return IANUS_OK;
}

ianus_status ianus_pt_swap(ianus_lattice* h) {
  GET_LAT(h);
  if (lat->pool) return IANUS_EINVAL;
  if (lat->K < 2 || !lat->tables_ok) return IANUS_EINVAL;
  if (lat->model != IANUS_EA_PM_J || lat->field) return IANUS_EUNSUPPORTED;
  return (ianus_status)do_pt_swap(lat);
}

ianus_status ianus_sweep_pt(ianus_lattice* h, int32_t algo, const double* beta, uint64_t nsweeps,
                            uint32_t swap_every, uint32_t measure_every) {
  GET_LAT(h);
  if (swap_every == 0 || nsweeps % swap_every != 0) return IANUS_EINVAL;
  if (lat->K < 2) return IANUS_EINVAL;
  if (lat->model != IANUS_EA_PM_J || lat->field) return IANUS_EUNSUPPORTED;
  for (uint64_t n = 0; n < nsweeps; n += swap_every) {
    ianus_status st = ianus_sweep(h, algo, beta, swap_every, measure_every);
    if (st) return st;
    st = ianus_pt_swap(h);
    if (st) return st;
  }
  return IANUS_OK;
}

ianus_status ianus_measure(ianus_lattice* h, int64_t* energy, int64_t* magnetisation, int64_t* overlap) {
  GET_LAT(h);
  if (overlap && lat->R < 2) return IANUS_EINVAL;
  int st = measure_into(lat, lat->out_E, lat->out_M, lat->out_Q, nullptr, overlap != nullptr);
  if (st) return (ianus_status)st;
  const size_t SKR = (size_t)lat->S * lat->K * lat->R;
  if (energy) CK(cudaMemcpyAsync(energy, lat->out_E, SKR * 8, cudaMemcpyDeviceToHost, lat->stream));
  if (magnetisation)
    CK(cudaMemcpyAsync(magnetisation, lat->out_M, SKR * lat->mq * 8, cudaMemcpyDeviceToHost, lat->stream));
  if (overlap)
    CK(cudaMemcpyAsync(overlap, lat->out_Q, (size_t)lat->S * lat->K * 8, cudaMemcpyDeviceToHost, lat->stream));
  CK(cudaStreamSynchronize(lat->stream));
  return IANUS_OK;
}

ianus_status ianus_read_series(ianus_lattice* h, uint64_t* sweep, int64_t* energy, int64_t* magnetisation,
                               int64_t* overlap, size_t cap_rows, size_t* n_rows, int32_t clear) {
  GET_LAT(h);
  const uint64_t first = std::max<uint64_t>(lat->ser_first, lat->ser_count > lat->cap ? lat->ser_count - lat->cap : 0);
  uint64_t n = lat->ser_count - first;
  if (n > cap_rows) n = cap_rows;
  const size_t SKR = (size_t)lat->S * lat->K * lat->R, SK = (size_t)lat->S * lat->K;
  // the rows are contiguous in the ring except where it wraps: at most two
  // copies per array
  for (uint64_t r = 0; r < n;) {
    const size_t pos = (size_t)((first + r) % lat->cap);
    const size_t m = (size_t)std::min<uint64_t>(n - r, lat->cap - pos);
    if (sweep) CK(cudaMemcpyAsync(sweep + r, lat->ser_sweep + pos, m * 8, cudaMemcpyDeviceToHost, lat->stream));
    if (energy)
      CK(cudaMemcpyAsync(energy + r * SKR, lat->ser_E + pos * SKR, m * SKR * 8, cudaMemcpyDeviceToHost, lat->stream));
    if (magnetisation)
      CK(cudaMemcpyAsync(magnetisation + r * SKR * lat->mq, lat->ser_M + pos * SKR * lat->mq,
                         m * SKR * lat->mq * 8, cudaMemcpyDeviceToHost, lat->stream));
    if (overlap && lat->R >= 2)
      CK(cudaMemcpyAsync(overlap + r * SK, lat->ser_Q + pos * SK, m * SK * 8, cudaMemcpyDeviceToHost, lat->stream));
    r += m;
  }
  CK(cudaStreamSynchronize(lat->stream));
  if (n_rows) *n_rows = (size_t)n;
  if (clear) lat->ser_first = lat->ser_count;
  return IANUS_OK;
}

static ianus_status staged_get(Lattice* lat, int8_t* host, size_t bytes,
                               cudaError_t (*fn)(Lattice&, int8_t*)) {
  int8_t* d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return IANUS_ENOMEM;
  }
  cudaError_t e = fn(*lat, d);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, d, bytes, cudaMemcpyDeviceToHost, lat->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
  cudaFree(d);
  return e == cudaSuccess ? IANUS_OK : (ianus_status)fail(lat, IANUS_ECUDA);
}

static ianus_status staged_set(Lattice* lat, const int8_t* host, size_t bytes,
                               cudaError_t (*fn)(Lattice&, const int8_t*)) {
  int8_t* d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return IANUS_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(d, host, bytes, cudaMemcpyHostToDevice, lat->stream);
  if (e == cudaSuccess) e = fn(*lat, d);
  if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
  cudaFree(d);
  return e == cudaSuccess ? IANUS_OK : (ianus_status)fail(lat, IANUS_ECUDA);
}

ianus_status ianus_get_spins_i8(ianus_lattice* h, int8_t* host) {
  GET_LAT(h);
  if (!host) return IANUS_EINVAL;
  const size_t bytes = (size_t)lat->S * lat->slots * lat->N;
  auto fn = lat->layout == IANUS_LAYOUT_I8 ? launch_get_spins_i8
            : lat->layout == IANUS_LAYOUT_BITS64 ? launch_get_spins_bits : launch_get_spins_potts;
  return staged_get(lat, host, bytes, fn);
}

ianus_status ianus_set_spins_i8(ianus_lattice* h, const int8_t* host) {
  GET_LAT(h);
  lat->mut += 1;  // the state changes other than by sweeps
  if (!host) return IANUS_EINVAL;
  const size_t bytes = (size_t)lat->S * lat->slots * lat->N;
  for (size_t i = 0; i < bytes; ++i) {
    const int v = host[i];
    if (lat->model == IANUS_EA_PM_J ? (v != 1 && v != -1) : (v < 0 || v > 3)) return IANUS_EINVAL;
  }
  auto fn = lat->layout == IANUS_LAYOUT_I8 ? launch_set_spins_i8
            : lat->layout == IANUS_LAYOUT_BITS64 ? launch_set_spins_bits : launch_set_spins_potts;
  return staged_set(lat, host, bytes, fn);
}

ianus_status ianus_get_couplings_i8(ianus_lattice* h, int8_t* host) {
  GET_LAT(h);
  if (!host) return IANUS_EINVAL;
  const size_t bytes = (size_t)lat->S * lat->D * lat->N;
  auto fn = lat->layout == IANUS_LAYOUT_I8 ? launch_get_couplings_i8
            : lat->layout == IANUS_LAYOUT_BITS64 ? launch_get_couplings_bits : launch_get_couplings_potts;
  return staged_get(lat, host, bytes, fn);
}

ianus_status ianus_set_couplings_i8(ianus_lattice* h, const int8_t* host) {
  GET_LAT(h);
  lat->mut += 1;  // the state changes other than by sweeps
  if (!host) return IANUS_EINVAL;
  const size_t bytes = (size_t)lat->S * lat->D * lat->N;
  for (size_t i = 0; i < bytes; ++i) {
    if (lat->model == IANUS_POTTS4_PERM) {  // the four 2-bit fields must be 0, 1, 2, 3 in some order
      const uint32_t c = (uint8_t)host[i];
      const uint32_t seen = (1u << (c & 3u)) | (1u << ((c >> 2) & 3u)) | (1u << ((c >> 4) & 3u)) | (1u << (c >> 6));
      if (seen != 0xFu) return IANUS_EINVAL;
    } else if (host[i] != 1 && host[i] != -1) {
      return IANUS_EINVAL;
    }
  }
  auto fn = lat->layout == IANUS_LAYOUT_I8 ? launch_set_couplings_i8
            : lat->layout == IANUS_LAYOUT_BITS64 ? launch_set_couplings_bits : launch_set_couplings_potts;
  return staged_set(lat, host, bytes, fn);
}

ianus_status ianus_get_sites_i8(ianus_lattice* h, int8_t* hsign, int8_t* occupied) {
  GET_LAT(h);
  if (lat->model != IANUS_EA_PM_J) return IANUS_EUNSUPPORTED;
  const size_t n = (size_t)lat->S * lat->N;
  if (!lat->field) {
    if (hsign) std::memset(hsign, 1, n);
    if (occupied) std::memset(occupied, 1, n);
    return IANUS_OK;
  }
  std::vector<int8_t> hs(n), occ(n, 1);
  ianus_status st;
  if (lat->layout == IANUS_LAYOUT_I8) {
    int8_t* d = nullptr;
    if (cudaMalloc(&d, 2 * n) != cudaSuccess) {
      cudaGetLastError();
      return IANUS_ENOMEM;
    }
    cudaError_t e = launch_get_sites_i8(*lat, d, d + n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), d, n, cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(occ.data(), d + n, n, cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    cudaFree(d);
    st = e == cudaSuccess ? IANUS_OK : (ianus_status)fail(lat, IANUS_ECUDA);
  } else {
    int8_t* d = nullptr;
    if (cudaMalloc(&d, 2 * n) != cudaSuccess) {
      cudaGetLastError();
      return IANUS_ENOMEM;
    }
    cudaError_t e = launch_get_sites_bits(*lat, d, d + n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), d, n, cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(occ.data(), d + n, n, cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    cudaFree(d);
    st = e == cudaSuccess ? IANUS_OK : (ianus_status)fail(lat, IANUS_ECUDA);
  }
  if (st) return st;
  if (hsign) std::memcpy(hsign, hs.data(), n);
  if (occupied) std::memcpy(occupied, occ.data(), n);
  return IANUS_OK;
}

ianus_status ianus_set_sites_i8(ianus_lattice* h, const int8_t* hsign, const int8_t* occupied) {
  GET_LAT(h);
  lat->mut += 1;  // the state changes other than by sweeps
  if (!lat->field) return IANUS_EUNSUPPORTED;
  const size_t n = (size_t)lat->S * lat->N;
  for (size_t i = 0; hsign && i < n; ++i)
    if (hsign[i] != 1 && hsign[i] != -1) return IANUS_EINVAL;
  for (size_t i = 0; occupied && i < n; ++i)
    if (occupied[i] != 0 && occupied[i] != 1) return IANUS_EINVAL;
  if (lat->layout == IANUS_LAYOUT_BITS64 && !lat->dilute) {  // the random-field model has no empty sites
    for (size_t i = 0; occupied && i < n; ++i)
      if (occupied[i] != 1) return IANUS_EUNSUPPORTED;
  }
  const bool bits = lat->layout == IANUS_LAYOUT_BITS64;
  int8_t* d = nullptr;
  if (cudaMalloc(&d, 2 * n) != cudaSuccess) {
    cudaGetLastError();
    return IANUS_ENOMEM;
  }
  cudaError_t e = bits ? launch_get_sites_bits(*lat, d, d + n) : launch_get_sites_i8(*lat, d, d + n);  // keep the rest
  if (e == cudaSuccess && hsign) e = cudaMemcpyAsync(d, hsign, n, cudaMemcpyHostToDevice, lat->stream);
  if (e == cudaSuccess && occupied) e = cudaMemcpyAsync(d + n, occupied, n, cudaMemcpyHostToDevice, lat->stream);
  if (e == cudaSuccess) e = bits ? launch_set_sites_bits(*lat, d, d + n) : launch_set_sites_i8(*lat, d, d + n);
  if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
  cudaFree(d);
  return e == cudaSuccess ? IANUS_OK : (ianus_status)fail(lat, IANUS_ECUDA);
}

// ---- fused serving: jobs in lanes of a pool lattice ----

static int segment_find(const Lattice* lat, int group, int lane0) {
  const uint32_t ns = (*lat->nseg_host)[group];
  for (uint32_t j = 0; j < ns; ++j)
    if ((int)(*lat->segs_host)[(size_t)group * kMaxSegs + j].lane0 == lane0) return (int)j;
  return -1;
}

static ianus_status upload_group(Lattice* lat, int group) {
  CK(cudaMemcpyAsync(lat->segs + (size_t)group * kMaxSegs, lat->segs_host->data() + (size_t)group * kMaxSegs,
                     kMaxSegs * sizeof(Segment), cudaMemcpyHostToDevice, lat->stream));
  CK(cudaMemcpyAsync(lat->nseg + group, lat->nseg_host->data() + group, 4, cudaMemcpyHostToDevice, lat->stream));
  CK(cudaMemcpyAsync(lat->tp + (size_t)group * kPlanes * kMaxClasses,
                     lat->tp_host->data() + (size_t)group * kPlanes * kMaxClasses,
                     kPlanes * kMaxClasses * sizeof(uint64_t), cudaMemcpyHostToDevice, lat->stream));
  // the host copies may change again before the copy runs: wait for it
  CK(cudaStreamSynchronize(lat->stream));
  return IANUS_OK;
}

ianus_status ianus_segment_load(ianus_lattice* h, int32_t group, int32_t lane0, int32_t n, uint64_t seed,
                                int32_t job_group, int32_t algo, double beta, uint64_t nsweeps) {
  GET_LAT(h);
  lat->mut += 1;  // the state changes other than by sweeps
  if (!lat->segs) return IANUS_EUNSUPPORTED;
  if (group < 0 || group >= lat->G || lane0 < 0 || n < 1 || lane0 + n > 64) return IANUS_EINVAL;
  if (job_group < 0 || job_group >= 4096) return IANUS_EINVAL;
  if ((algo != IANUS_METROPOLIS && algo != IANUS_HEATBATH) || !std::isfinite(beta) || beta < 0.0) return IANUS_EINVAL;
  const uint64_t mask = (n >= 64 ? ~0ull : ((1ull << n) - 1ull)) << lane0;
  uint32_t& ns = (*lat->nseg_host)[group];
  for (uint32_t j = 0; j < ns; ++j)
    if ((*lat->segs_host)[(size_t)group * kMaxSegs + j].mask & mask) return IANUS_EINVAL;  // lanes taken
  if (ns >= (uint32_t)kMaxSegs) return IANUS_EINVAL;
  if (!lat->pool) {
    lat->pool = true;
    drop_graphs(lat);
  }
  const PhiloxKeys keys = make_keys(seed);
  CK(launch_load_segment(*lat, group, (uint32_t)lane0, (uint32_t)n, (uint32_t)job_group, keys));
  // per-lane thresholds of the job's (algo, beta), as its own lattice would use
  uint64_t thr[kMaxClasses];
  class_thresholds(lat->D, algo, beta, thr);
  uint64_t* tp = lat->tp_host->data() + (size_t)group * kPlanes * kMaxClasses;
  for (int u = 0; u < kMaxClasses; ++u) {
    for (int q = 0; q < kPlanes; ++q) tp[q * kMaxClasses + u] &= ~mask;
    if (u > 2 * lat->D) continue;
    if (thr[u] >= kTwo32) {
      tp[32 * kMaxClasses + u] |= mask;
    } else {
      for (int q = 0; q < 32; ++q)
        if ((thr[u] >> (31 - q)) & 1ull) tp[q * kMaxClasses + u] |= mask;
    }
  }
  Segment sg{};
  sg.mask = mask;
  sg.t = 0;
  sg.t_end = nsweeps;
  sg.key_lo = (uint32_t)(seed & 0xffffffffu);
  sg.key_hi = (uint32_t)(seed >> 32);
  sg.lane0 = (uint32_t)lane0;
  sg.inv = algo == IANUS_HEATBATH ? 1u : 0u;
  sg.jgroup = (uint32_t)job_group;
  (*lat->segs_host)[(size_t)group * kMaxSegs + ns] = sg;
  ns += 1;
  return upload_group(lat, group);
}

ianus_status ianus_segment_release(ianus_lattice* h, int32_t group, int32_t lane0) {
  GET_LAT(h);
  lat->mut += 1;  // the state changes other than by sweeps
  if (!lat->segs || group < 0 || group >= lat->G) return IANUS_EINVAL;
  const int j = segment_find(lat, group, lane0);
  if (j < 0) return IANUS_EINVAL;
  uint32_t& ns = (*lat->nseg_host)[group];
  Segment* base = lat->segs_host->data() + (size_t)group * kMaxSegs;
  base[j] = base[ns - 1];  // keep the table compact; order is immaterial
  base[ns - 1] = Segment{};
  ns -= 1;
  return upload_group(lat, group);
}

ianus_status ianus_segment_state(ianus_lattice* h, int32_t group, int32_t lane0, uint64_t* sweeps_done,
                                 uint64_t* sweeps_requested) {
  GET_LAT(h);
  if (!lat->segs || group < 0 || group >= lat->G) return IANUS_EINVAL;
  const int j = segment_find(lat, group, lane0);
  if (j < 0) return IANUS_EINVAL;
  const Segment& sg = (*lat->segs_host)[(size_t)group * kMaxSegs + j];
  if (sweeps_done) *sweeps_done = sg.t;
  if (sweeps_requested) *sweeps_requested = sg.t_end;
  return IANUS_OK;
}

static int fused_sweep_once(Lattice* lat) {
  CK(launch_sweep_fused(*lat, 0));
  CK(launch_sweep_fused(*lat, 1));
  CK(launch_advance_segments(*lat));
  return IANUS_OK;
}

ianus_status ianus_sweep_segments(ianus_lattice* h, uint64_t nsweeps) {
  GET_LAT(h);
  lat->mut += 1;  // the state changes other than by sweeps
  if (!lat->segs) return IANUS_EUNSUPPORTED;
  uint64_t left = nsweeps;
  const bool resident = nsweeps >= 2 && lat->use_resident && resident_fused_fits(*lat);
  while (left > 0) {
    const uint32_t B = (uint32_t)std::min<uint64_t>(left, resident ? kResidentBlock : 64);
    if (resident) {
      CK(launch_resident_fused(*lat, B));
    } else if (B < 4 || !lat->use_graphs || !lat->graphs) {
      for (uint32_t k = 0; k < B; ++k) {
        int st = fused_sweep_once(lat);
        if (st) return (ianus_status)st;
      }
    } else {
      const uint32_t key = (1u << 31) | B;
      auto it = lat->graphs->find(key);
      if (it == lat->graphs->end()) {
        if (!lat->cap_stream) CK(cudaStreamCreateWithFlags(&lat->cap_stream, cudaStreamNonBlocking));
        cudaStream_t user = lat->stream;
        lat->stream = lat->cap_stream;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(lat->cap_stream, cudaStreamCaptureModeThreadLocal);
        int st = IANUS_OK;
        for (uint32_t k = 0; e == cudaSuccess && st == IANUS_OK && k < B; ++k) st = fused_sweep_once(lat);
        cudaError_t e2 = cudaStreamEndCapture(lat->cap_stream, &g);
        lat->stream = user;
        cudaGraphExec_t ex = nullptr;
        if (e != cudaSuccess || e2 != cudaSuccess || st != IANUS_OK || !g ||
            cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
          if (g) cudaGraphDestroy(g);
          cudaGetLastError();
          return IANUS_ECUDA;
        }
        cudaGraphDestroy(g);
        it = lat->graphs->emplace(key, ex).first;
      }
      CK(cudaGraphLaunch(it->second, lat->stream));
    }
    // the host copy follows the device counters: every live segment advances
    for (int g = 0; g < lat->G; ++g)
      for (uint32_t j = 0; j < (*lat->nseg_host)[g]; ++j) {
        Segment& sg = (*lat->segs_host)[(size_t)g * kMaxSegs + j];
        sg.t = std::min<uint64_t>(sg.t_end, sg.t + B);
      }
    left -= B;
  }
  return IANUS_OK;
}

ianus_status ianus_get_pt_state(ianus_lattice* h, int32_t* slot_at, uint64_t* accepted, uint64_t* swap_steps) {
  GET_LAT(h);
  const size_t n = (size_t)lat->S * lat->R * lat->K;
  if (slot_at) CK(cudaMemcpyAsync(slot_at, lat->slot_at, n * 4, cudaMemcpyDeviceToHost, lat->stream));
  if (accepted && lat->K > 1)
    CK(cudaMemcpyAsync(accepted, lat->accepted, (size_t)lat->S * lat->R * (lat->K - 1) * 8, cudaMemcpyDeviceToHost,
                       lat->stream));
  CK(cudaStreamSynchronize(lat->stream));
  if (swap_steps) *swap_steps = lat->steps;
  return IANUS_OK;
}

ianus_status ianus_get_sweeps(ianus_lattice* h, uint64_t* sweeps) {
  GET_LAT(h);
  if (!sweeps) return IANUS_EINVAL;
  *sweeps = lat->sweeps;
  return IANUS_OK;
}

ianus_status ianus_get_state(ianus_lattice* h, void* host_buf, size_t cap, size_t* n) {
  GET_LAT(h);
  if (lat->pool) return IANUS_EUNSUPPORTED;  // segment tables are not part of the blob
  Sizes z;
  plan(&lat->cfg, z);
  const size_t perm = (size_t)lat->S * lat->R * lat->K * 4;
  const size_t accb = (size_t)lat->S * lat->R * std::max(lat->K - 1, 1) * 8;
  const size_t need =
      sizeof(StateHeader) + 2 * perm + accb + z.J_bytes + z.spins_bytes + z.sites_bytes + z.wheel_bytes;
  if (n) *n = need;
  if (!host_buf) return IANUS_OK;
  if (cap < need) return IANUS_EINVAL;
  StateHeader hd{};
  hd.magic = kStateMagic;
  hd.version = IANUS_ABI_VERSION;
  hd.model = (uint32_t)lat->model;
  hd.dim = (uint32_t)lat->D;
  hd.L = (uint32_t)lat->L;
  hd.S = (uint32_t)lat->S;
  hd.R = (uint32_t)lat->R;
  hd.K = (uint32_t)lat->K;
  hd.layout = (uint32_t)lat->layout;
  hd.disorder = (uint32_t)lat->cfg.disorder;
  hd.seed = lat->cfg.seed;
  hd.sweeps = lat->sweeps;
  hd.steps = lat->steps;
  hd.spins_bytes = z.spins_bytes;
  hd.J_bytes = z.J_bytes;
  hd.sites_bytes = z.sites_bytes;
  hd.wheel_bytes = z.wheel_bytes;
  hd.field = lat->cfg.field;
  hd.occupation = lat->cfg.occupation;
  uint8_t* o = (uint8_t*)host_buf;
  std::memcpy(o, &hd, sizeof hd);
  o += sizeof hd;
  CK(cudaMemcpyAsync(o, lat->slot_at, perm, cudaMemcpyDeviceToHost, lat->stream));
  o += perm;
  CK(cudaMemcpyAsync(o, lat->temp_of, perm, cudaMemcpyDeviceToHost, lat->stream));
  o += perm;
  CK(cudaMemcpyAsync(o, lat->accepted, accb, cudaMemcpyDeviceToHost, lat->stream));
  o += accb;
  CK(cudaMemcpyAsync(o, lat->J, z.J_bytes, cudaMemcpyDeviceToHost, lat->stream));
  o += z.J_bytes;
  CK(cudaMemcpyAsync(o, lat->spins, z.spins_bytes, cudaMemcpyDeviceToHost, lat->stream));
  o += z.spins_bytes;
  if (z.sites_bytes) CK(cudaMemcpyAsync(o, lat->base + z.off_sites, z.sites_bytes, cudaMemcpyDeviceToHost, lat->stream));
  o += z.sites_bytes;
  if (z.wheel_bytes)
    CK(cudaMemcpyAsync(o, lat->base + z.off_wheels, z.wheel_bytes, cudaMemcpyDeviceToHost, lat->stream));
  CK(cudaStreamSynchronize(lat->stream));
  return IANUS_OK;
}

ianus_status ianus_set_state(ianus_lattice* h, const void* host_buf, size_t n) {
  Lattice* lat = reinterpret_cast<Lattice*>(h);
  if (!lat || !host_buf) return IANUS_EINVAL;
  Sizes z;
  plan(&lat->cfg, z);
  const size_t perm = (size_t)lat->S * lat->R * lat->K * 4;
  const size_t accb = (size_t)lat->S * lat->R * std::max(lat->K - 1, 1) * 8;
  const size_t need =
      sizeof(StateHeader) + 2 * perm + accb + z.J_bytes + z.spins_bytes + z.sites_bytes + z.wheel_bytes;
  if (n < need) return IANUS_ESTATE;
  StateHeader hd;
  std::memcpy(&hd, host_buf, sizeof hd);
  if (hd.magic != kStateMagic || hd.version != IANUS_ABI_VERSION || hd.model != (uint32_t)lat->model ||
      hd.dim != (uint32_t)lat->D || hd.L != (uint32_t)lat->L || hd.S != (uint32_t)lat->S ||
      hd.R != (uint32_t)lat->R || hd.K != (uint32_t)lat->K || hd.layout != (uint32_t)lat->layout ||
      hd.seed != lat->cfg.seed || hd.spins_bytes != z.spins_bytes || hd.J_bytes != z.J_bytes ||
      hd.disorder != (uint32_t)lat->cfg.disorder || hd.sites_bytes != z.sites_bytes ||
      hd.wheel_bytes != z.wheel_bytes ||
      std::memcmp(&hd.field, &lat->cfg.field, sizeof(double)) != 0)
    return IANUS_ESTATE;
  const uint8_t* in = (const uint8_t*)host_buf + sizeof hd;
  lat->sticky = 0;
  lat->mut += 1;  // the state changes other than by sweeps
  CK(cudaMemcpyAsync(lat->slot_at, in, perm, cudaMemcpyHostToDevice, lat->stream));
  in += perm;
  CK(cudaMemcpyAsync(lat->temp_of, in, perm, cudaMemcpyHostToDevice, lat->stream));
  in += perm;
  CK(cudaMemcpyAsync(lat->accepted, in, accb, cudaMemcpyHostToDevice, lat->stream));
  in += accb;
  CK(cudaMemcpyAsync(lat->J, in, z.J_bytes, cudaMemcpyHostToDevice, lat->stream));
  in += z.J_bytes;
  CK(cudaMemcpyAsync(lat->spins, in, z.spins_bytes, cudaMemcpyHostToDevice, lat->stream));
  in += z.spins_bytes;
  if (z.sites_bytes) CK(cudaMemcpyAsync(lat->base + z.off_sites, in, z.sites_bytes, cudaMemcpyHostToDevice, lat->stream));
  in += z.sites_bytes;
  if (z.wheel_bytes)
    CK(cudaMemcpyAsync(lat->base + z.off_wheels, in, z.wheel_bytes, cudaMemcpyHostToDevice, lat->stream));
  CK(cudaMemsetAsync(lat->err, 0, 4, lat->stream));
  // The tables depend on beta and the algorithm only, the per-lane planes
  // also on the restored temperature permutation: those are rebuilt in
  // place, so that the tables, the specialised kernels and the captured
  // sweep graphs stay valid.
  if (lat->tables_ok && lat->layout == IANUS_LAYOUT_BITS64)
    CK(lat->field ? launch_build_field_planes(*lat) : launch_build_planes(*lat));
  CK(cudaStreamSynchronize(lat->stream));
  lat->sweeps = hd.sweeps;
  lat->steps = hd.steps;
  lat->t_dev_valid = false;
  return IANUS_OK;
}

ianus_status ianus_synchronize(ianus_lattice* h) {
  GET_LAT(h);
  CK(cudaStreamSynchronize(lat->stream));
  uint32_t err = 0;
  CK(cudaMemcpy(&err, lat->err, 4, cudaMemcpyDeviceToHost));
  if (err & ERR_TIMEOUT) {
    lat->sticky = IANUS_ESTATE;
    return IANUS_ETIMEOUT;
  }
  if (err) {
    lat->sticky = IANUS_ESTATE;
    return IANUS_ESTATE;
  }
  return IANUS_OK;
}

ianus_status ianus_set_variant(ianus_lattice* h, int32_t variant) {
  GET_LAT(h);
  if (variant < 0 || variant > kMaxVariant) return IANUS_EINVAL;
  if (lat->variant != variant) drop_graphs(lat);
  lat->variant = variant;
  return IANUS_OK;
}

ianus_status ianus_prepare_sweep(ianus_lattice* h, int32_t algo, const double* beta, int32_t variant,
                                 int32_t* ready) {
  Lattice* lat = reinterpret_cast<Lattice*>(h);
  if (!lat || !beta || !ready) return IANUS_EINVAL;
  *ready = 0;
  if ((algo != IANUS_METROPOLIS && algo != IANUS_HEATBATH) || variant < 0 || variant > kMaxVariant) return IANUS_EINVAL;
  if (!beta_ok(beta, lat->K)) return IANUS_EINVAL;
  // only the bit-sliced +-J sweep at one temperature has specialised kernels
  if (lat->model != IANUS_EA_PM_J || lat->layout != IANUS_LAYOUT_BITS64 || lat->field || lat->pool || lat->K != 1)
    return IANUS_OK;
  const int v = specialised_variant(*lat, variant);
  if (v < 2) return IANUS_OK;
  uint64_t thr[kMaxClasses];
  class_thresholds(lat->D, algo, beta[0], thr);
  const UniformLut u = uniform_lut(lat->D, algo, thr);
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    prev = -1;
  }
  if (prev != lat->dev && cudaSetDevice(lat->dev) != cudaSuccess) {
    cudaGetLastError();
    return IANUS_ECUDA;
  }
  *ready = specialised_sweep_kernel(*lat, u, algo, v) ? 1 : 0;
  if (prev >= 0 && prev != lat->dev) cudaSetDevice(prev);
  cudaGetLastError();
  return IANUS_OK;
}

ianus_status ianus_set_persistent_wait(ianus_lattice* h, uint64_t timeout_ns, int32_t absent_block) {
  GET_LAT(h);
  if (timeout_ns == 0 || absent_block < -1) return IANUS_EINVAL;
  lat->persist_timeout_ns = timeout_ns;
  lat->persist_absent = absent_block;
  return IANUS_OK;
}

ianus_status ianus_set_block_words(ianus_lattice* h, uint32_t words_per_block) {
  GET_LAT(h);
  if (words_per_block > (1u << 24)) return IANUS_EINVAL;
  if (lat->block_words != words_per_block) drop_graphs(lat);
  lat->block_words = words_per_block;
  return IANUS_OK;
}

ianus_status ianus_set_graphs(ianus_lattice* h, int32_t enable) {
  GET_LAT(h);
  lat->use_graphs = enable != 0;
  return IANUS_OK;
}

ianus_status ianus_set_resident(ianus_lattice* h, int32_t enable) {
  GET_LAT(h);
  if (enable < 0 || enable > 3) return IANUS_EINVAL;
  lat->use_resident = enable != 0;
  if (enable) lat->resident_mode = enable;
  return IANUS_OK;
}

ianus_status ianus_destroy(ianus_lattice* h) {
  Lattice* lat = reinterpret_cast<Lattice*>(h);
  if (!lat) return IANUS_OK;
  cudaStreamSynchronize(lat->stream);
  drop_graphs(lat);
  delete lat->graphs;
  delete lat->segs_host;
  delete lat->nseg_host;
  delete lat->tp_host;
  if (lat->cap_stream) cudaStreamDestroy(lat->cap_stream);
  if (lat->owns_buffer) cudaFree(lat->base);
  delete lat;
  return IANUS_OK;
}

const char* ianus_status_string(int32_t status) {
  switch (status) {
    case IANUS_OK: return "ok";
    case IANUS_EINVAL: return "invalid argument";
    case IANUS_ENOMEM: return "out of memory";
    case IANUS_ECUDA: return "CUDA runtime error";
    case IANUS_ETIMEOUT: return "bounded device wait expired";
    case IANUS_EUNSUPPORTED: return "unsupported configuration";
    case IANUS_ESTATE: return "lattice in error state or bad state blob";
    default: return "unknown status";
  }
}

}  // extern "C"
