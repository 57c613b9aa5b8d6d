// tables.cpp -- host construction of the integer acceptance tables: the
// look-up table the update cell indexes with its local energy (Sec. 3.2),
// compared against a 32-bit random number (Sec. 3.3).  Probabilities are
// those of Sec. 2.2: Metropolis exp(-beta dE), heat bath Eq. (4), evaluated
// in IEEE double precision exactly as stated in include/ianus.h and stored
// as floor(2^32 p) in [0, 2^32].
#include <cmath>
#include <cstdint>

#include "lattice.h"

namespace ianus {

static uint64_t to_threshold(double p) { return (uint64_t)std::floor(std::ldexp(p, 32)); }

size_t table_ising(int dim, int algo, double beta, uint64_t* out, size_t n) {
  if ((dim != 2 && dim != 3) || !out || !(beta >= 0.0) || !std::isfinite(beta)) return 0;
  if (algo == IANUS_METROPOLIS) {
    if (n < (size_t)dim) return 0;
    for (int j = 0; j < dim; ++j) out[j] = to_threshold(std::exp(-beta * (double)(4 * (j + 1))));
    return (size_t)dim;
  }
  if (algo == IANUS_HEATBATH) {
    if (n < (size_t)(2 * dim + 1)) return 0;
    for (int j = 0; j <= 2 * dim; ++j) {
      const int x = -2 * dim + 2 * j;
      out[j] = to_threshold(1.0 / (1.0 + std::exp(-2.0 * beta * (double)x)));
    }
    return (size_t)(2 * dim + 1);
  }
  return 0;
}

void class_thresholds(int dim, int algo, double beta, uint64_t* thr) {
  for (int u = 0; u < kMaxClasses; ++u) thr[u] = 0;
  if (algo == IANUS_METROPOLIS) {
    for (int u = 0; u <= 2 * dim; ++u) {
      const int dE = 4 * dim - 4 * u;
      thr[u] = dE <= 0 ? kTwo32 : to_threshold(std::exp(-beta * (double)dE));
    }
  } else {
    for (int u = 0; u <= 2 * dim; ++u) {
      const int x = 2 * dim - 2 * u;
      thr[u] = to_threshold(1.0 / (1.0 + std::exp(-2.0 * beta * (double)x)));
    }
  }
}

// x = (double)v + w, w = +|h| (f = 1, s_i h_i > 0) or -|h| (f = 0), w = +0.0
// when |h| = 0; dE = 2.0 * x.  The expressions follow include/ianus.h.
static double field_x(int v, int f, double hmag) {
  const double w = hmag == 0.0 ? 0.0 : (f ? hmag : -hmag);
  return (double)v + w;
}

void field_thresholds(int dim, int algo, double beta, double hmag, uint64_t* thr) {
  for (int c = 0; c < kFieldClasses; ++c) thr[c] = 0;
  for (int v = -2 * dim; v <= 2 * dim; ++v)
    for (int f = 0; f < 2; ++f) {
      const double x = field_x(v, f, hmag);
      uint64_t T;
      if (algo == IANUS_METROPOLIS) {
        const double dE = 2.0 * x;
        T = dE <= 0.0 ? kTwo32 : to_threshold(std::exp(-beta * dE));
      } else {
        T = to_threshold(1.0 / (1.0 + std::exp(-2.0 * beta * x)));
      }
      thr[(v + 2 * dim) * 2 + f] = T;
    }
}

// w_k = exp(beta n_k); S0 = w0, S1 = S0 + w1, S2 = S1 + w2, Z = S2 + w3;
// T_k = floor(2^32 S_k / Z): the cumulative heat-bath thresholds.
void potts_thresholds(double beta, const int* n, uint64_t* T) {
  const double w0 = std::exp(beta * (double)n[0]), w1 = std::exp(beta * (double)n[1]);
  const double w2 = std::exp(beta * (double)n[2]), w3 = std::exp(beta * (double)n[3]);
  const double S0 = w0, S1 = S0 + w1, S2 = S1 + w2, Z = S2 + w3;
  T[0] = to_threshold(S0 / Z);
  T[1] = to_threshold(S1 / Z);
  T[2] = to_threshold(S2 / Z);
}

size_t table_potts(double beta, uint64_t* out, size_t n) {
  const size_t need = 3u * 13u * 13u * 13u * 13u;
  if (!out || n < need || !(beta >= 0.0) || !std::isfinite(beta)) return 0;
  size_t idx = 0;
  int c[4];
  for (c[0] = -6; c[0] <= 6; ++c[0])
    for (c[1] = -6; c[1] <= 6; ++c[1])
      for (c[2] = -6; c[2] <= 6; ++c[2])
        for (c[3] = -6; c[3] <= 6; ++c[3], idx += 3) potts_thresholds(beta, c, out + idx);
  return need;
}

size_t table_pt(double beta_k, double beta_k1, uint64_t* out, size_t n) {
  if (!out || !std::isfinite(beta_k) || !std::isfinite(beta_k1)) return 0;
  double db = beta_k - beta_k1;
  if (db < 0) db = -db;
  for (size_t m = 1; m <= n; ++m) out[m - 1] = to_threshold(std::exp(-db * (double)(4 * m)));
  return n;
}

}  // namespace ianus

extern "C" {
size_t ianus_table_ising(int32_t dim, int32_t algo, double beta, uint64_t* out, size_t n) {
  return ianus::table_ising(dim, algo, beta, out, n);
}
size_t ianus_table_potts(double beta, uint64_t* out, size_t n) { return ianus::table_potts(beta, out, n); }
size_t ianus_table_pt(double beta_k, double beta_k1, uint64_t* out, size_t n) {
  return ianus::table_pt(beta_k, beta_k1, out, n);
}
size_t ianus_table_potts_counts(double beta, const int32_t* n, uint64_t* T) {
  if (!n || !T || !(beta >= 0.0) || !std::isfinite(beta)) return 0;
  const int c[4] = {n[0], n[1], n[2], n[3]};
  ianus::potts_thresholds(beta, c, T);
  return 3;
}
size_t ianus_table_field(int32_t dim, int32_t algo, double beta, double field, uint64_t* out, size_t n) {
  const size_t need = (size_t)(2 * (4 * dim + 1));
  if ((dim != 2 && dim != 3) || !out || n < need || !(beta >= 0.0) || !std::isfinite(beta) || !(field >= 0.0) ||
      !std::isfinite(field) || (algo != IANUS_METROPOLIS && algo != IANUS_HEATBATH))
    return 0;
  uint64_t t[ianus::kFieldClasses];
  ianus::field_thresholds(dim, algo, beta, field, t);
  for (size_t c = 0; c < need; ++c) out[c] = t[c];
  return need;
}
}
