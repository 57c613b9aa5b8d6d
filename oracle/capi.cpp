/*
 * capi.cpp -- extern "C" entry points of the oracle for ctypes.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Built into liboracle.so, which
 * only the tests, the smoke check and the CPU-baseline leg of bench.py load.
 */
#include <cstring>
#include <vector>

#include "oracle.h"

using namespace oracle;

extern "C" {

void* oracle_create(int model, int q, int dim, int L, const int32_t* sample_ids, int n_ids, int R,
                    int K, uint64_t seed, int disorder, double field, double occupation, int rng) {
  if (dim < 1 || dim > 4 || L < 2 || (L & 1) || n_ids < 1 || R < 1 || K < 1 || q < 2) return nullptr;
  if (model < 0 || model > 2 || (model == MODEL_PERM && q != 4)) return nullptr;
  if (disorder < 0 || disorder > 3 || !(field >= 0.0) || !(occupation >= 0.0 && occupation <= 1.0)) return nullptr;
  State* st = new State();
  std::vector<int> ids(sample_ids, sample_ids + n_ids);
  if (rng < 0 || rng > 1 || (rng == RNG_WHEEL && model != MODEL_ISING)) {
    delete st;
    return nullptr;
  }
  init_state(*st, model, q, dim, L, ids, R, K, seed, disorder, field, occupation, rng);
  return st;
}

void oracle_destroy(void* h) { delete static_cast<State*>(h); }

void oracle_sweep(void* h, int algo, const double* beta, uint64_t nsweeps, uint32_t measure_every,
                  int nthreads) {
  run_sweeps(*static_cast<State*>(h), algo, beta, nsweeps, measure_every, nthreads);
}

void oracle_pt_swap(void* h, const double* beta) { pt_swap(*static_cast<State*>(h), beta); }

void oracle_measure(void* h, int64_t* E, int64_t* M, int64_t* Q) {
  measure_all(*static_cast<State*>(h), E, M, Q);
}

uint64_t oracle_sweeps(void* h) { return static_cast<State*>(h)->sweeps; }

size_t oracle_series_rows(void* h) { return static_cast<State*>(h)->ser_sweep.size(); }

/* Copies all rows; caller sizes arrays from oracle_series_rows. */
void oracle_series(void* h, uint64_t* sweep, int64_t* E, int64_t* M, int64_t* Q) {
  State* st = static_cast<State*>(h);
  if (sweep) std::memcpy(sweep, st->ser_sweep.data(), st->ser_sweep.size() * 8);
  if (E) std::memcpy(E, st->ser_E.data(), st->ser_E.size() * 8);
  if (M) std::memcpy(M, st->ser_M.data(), st->ser_M.size() * 8);
  if (Q) std::memcpy(Q, st->ser_Q.data(), st->ser_Q.size() * 8);
}

void oracle_series_clear(void* h) {
  State* st = static_cast<State*>(h);
  st->ser_sweep.clear();
  st->ser_E.clear();
  st->ser_M.clear();
  st->ser_Q.clear();
}

/* spins int8 [n_ids][slots][N] */
void oracle_get_spins(void* h, int8_t* out) {
  State* st = static_cast<State*>(h);
  size_t o = 0;
  for (auto& smp : st->samples)
    for (auto& v : smp.spin) {
      std::memcpy(out + o, v.data(), v.size());
      o += v.size();
    }
}

static void rebook(State* st) {
  for (auto& smp : st->samples)
    for (size_t sl = 0; sl < smp.spin.size(); ++sl) {
      smp.E_run[sl] = energy(*st, smp, (int)sl);
      smp.F_run[sl] = st->model == MODEL_ISING ? field_sum(*st, smp, (int)sl) : 0;
    }
}

void oracle_set_spins(void* h, const int8_t* in) {
  State* st = static_cast<State*>(h);
  size_t o = 0;
  for (auto& smp : st->samples)
    for (auto& v : smp.spin) {
      std::memcpy(v.data(), in + o, v.size());
      o += v.size();
    }
  rebook(st);
}

/* field signs / occupations int8 [n_ids][N] */
void oracle_get_sites(void* h, int8_t* hs, int8_t* x) {
  State* st = static_cast<State*>(h);
  size_t o = 0;
  for (auto& smp : st->samples) {
    if (hs) std::memcpy(hs + o, smp.hs.data(), smp.hs.size());
    if (x) std::memcpy(x + o, smp.x.data(), smp.x.size());
    o += smp.hs.size();
  }
}

void oracle_set_sites(void* h, const int8_t* hs, const int8_t* x) {
  State* st = static_cast<State*>(h);
  size_t o = 0;
  for (auto& smp : st->samples) {
    if (hs) std::memcpy(smp.hs.data(), hs + o, smp.hs.size());
    if (x) std::memcpy(smp.x.data(), x + o, smp.x.size());
    o += smp.hs.size();
  }
  rebook(st);
}

/* couplings int8 [n_ids][D][N]: J = +-1, or for model 2 the 8-bit code
 * pi(0) | pi(1) << 2 | pi(2) << 4 | pi(3) << 6 stored as int8 */
void oracle_get_couplings(void* h, int8_t* out) {
  State* st = static_cast<State*>(h);
  size_t o = 0;
  for (auto& smp : st->samples)
    for (size_t k = 0; k < smp.J.size(); ++k)
      out[o++] = st->model == MODEL_PERM ? (int8_t)(uint8_t)perm_code(smp.J[k]) : smp.J[k];
}

/* Returns 0, or -1 (nothing changed) when a model-2 code is not a permutation. */
int oracle_set_couplings(void* h, const int8_t* in) {
  State* st = static_cast<State*>(h);
  size_t n = 0;
  for (auto& smp : st->samples) n += smp.J.size();
  if (st->model == MODEL_PERM)
    for (size_t k = 0; k < n; ++k)
      if (perm_index_of_code((uint8_t)in[k]) < 0) return -1;
  size_t o = 0;
  for (auto& smp : st->samples)
    for (size_t k = 0; k < smp.J.size(); ++k, ++o)
      smp.J[k] = st->model == MODEL_PERM ? (int8_t)perm_index_of_code((uint8_t)in[o]) : in[o];
  rebook(st);
  return 0;
}

/* slot_at int32 [n_ids][R][K], accepted uint64 [n_ids][R][K-1] */
void oracle_get_pt(void* h, int32_t* slot_at, uint64_t* accepted, uint64_t* steps) {
  State* st = static_cast<State*>(h);
  size_t o = 0, p = 0;
  for (auto& smp : st->samples)
    for (int a = 0; a < st->R; ++a) {
      for (int k = 0; k < st->K; ++k)
        if (slot_at) slot_at[o++] = smp.slot_at[a][k];
      for (int k = 0; k + 1 < st->K; ++k)
        if (accepted) accepted[p++] = smp.accepted[a][k];
    }
  if (steps) *steps = st->steps;
}

/* max over configurations of |E_run - E recomputed| and |F_run - F recomputed| */
int64_t oracle_bookkeeping_error(void* h) {
  State* st = static_cast<State*>(h);
  int64_t worst = 0;
  for (auto& smp : st->samples)
    for (size_t sl = 0; sl < smp.spin.size(); ++sl) {
      int64_t diff = smp.E_run[sl] - energy(*st, smp, (int)sl);
      if (diff < 0) diff = -diff;
      if (diff > worst) worst = diff;
      if (st->model == 0) {
        int64_t df = smp.F_run[sl] - field_sum(*st, smp, (int)sl);
        if (df < 0) df = -df;
        if (df > worst) worst = df;
      }
    }
  return worst;
}

void oracle_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

uint32_t oracle_ising_random(uint64_t seed, int sample, int slot, uint32_t site, uint64_t sweep) {
  return ising_random(seed, sample, slot, site, sweep);
}
uint32_t oracle_potts_random(uint64_t seed, int sample, int slot, uint32_t site, uint64_t sweep) {
  return potts_random(seed, sample, slot, site, sweep);
}
uint32_t oracle_pt_random(uint64_t seed, int sample, int replica, int pair, uint64_t step) {
  return pt_random(seed, sample, replica, pair, step);
}
uint64_t oracle_table_metropolis(double beta, int dE) { return table_metropolis(beta, dE); }
uint64_t oracle_table_heatbath(double beta, int x) { return table_heatbath(beta, x); }
void oracle_table_potts(double beta, int q, const int32_t* n, uint64_t* T) {
  std::vector<int> nn(n, n + q);
  table_potts(beta, q, nn.data(), T);
}
uint64_t oracle_table_pt(double dbeta_abs, int64_t dabs) { return table_pt(dbeta_abs, dabs); }
uint64_t oracle_table_metropolis_x(double beta, double x) { return table_metropolis_x(beta, x); }
uint64_t oracle_table_heatbath_x(double beta, double x) { return table_heatbath_x(beta, x); }
int oracle_field_sign_bit(uint64_t seed, int sample, uint32_t site) { return field_sign_bit(seed, sample, site); }
uint32_t oracle_occupation_random(uint64_t seed, int sample, uint32_t site) {
  return occupation_random(seed, sample, site);
}
int oracle_perm_coupling_index(uint64_t seed, int sample, int d, uint32_t site) {
  return perm_coupling_index(seed, sample, d, site);
}
int oracle_perm_code(int index) { return perm_code(index); }

/* A freshly seeded wheel: its 61 starting values and its first n outputs. */
void oracle_wheel(uint64_t seed, int sample, int slot, uint32_t row, int colour, uint32_t* start61, uint32_t n,
                  uint32_t* out) {
  Wheel w = wheel_seeded(seed, sample, slot, row, colour);
  if (start61)
    for (int k = 0; k < 61; ++k) start61[k] = w.hist[k];
  for (uint32_t k = 0; k < n; ++k) out[k] = w.next();
}

/* n outputs of Eq. (5) from caller-given starting values I(-61) .. I(-1). */
void oracle_wheel_from(const uint32_t* start61, uint32_t n, uint32_t* out) {
  Wheel w;
  w.hist.assign(start61, start61 + 61);
  for (uint32_t k = 0; k < n; ++k) out[k] = w.next();
}

}  // extern "C"
