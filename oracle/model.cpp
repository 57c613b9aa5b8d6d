/*
 * model.cpp -- the oracle's lattice, Hamiltonians, sweeps, measurements and
 * parallel tempering.  Plain site loops, no blocking, no bit tricks.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <thread>

namespace oracle {

/* ---- geometry: periodic D-dimensional cubic lattice (Sec. 2.1) ---- */

void site_coords(const State& st, uint32_t i, int* x) {
  for (int d = 0; d < st.D; ++d) {
    x[d] = (int)(i % (uint32_t)st.L);
    i /= (uint32_t)st.L;
  }
}

static uint32_t site_index(const State& st, const int* x) {
  uint32_t i = 0;
  for (int d = st.D - 1; d >= 0; --d) i = i * (uint32_t)st.L + (uint32_t)x[d];
  return i;
}

uint32_t neighbour(const State& st, uint32_t i, int d, int dir) {
  int x[4];
  site_coords(st, i, x);
  x[d] = (x[d] + dir + st.L) % st.L;
  return site_index(st, x);
}

/* Sec. 3.1: the lattice is bipartite; colour = parity of the coordinate sum. */
int colour(const State& st, uint32_t i) {
  int x[4];
  site_coords(st, i, x);
  int sum = 0;
  for (int d = 0; d < st.D; ++d) sum += x[d];
  return sum % 2;
}

/* ---- set-up: quenched couplings and initial configurations ---- */

void init_state(State& st, int model, int q, int D, int L, const std::vector<int>& sample_ids,
                int R, int K, uint64_t seed, int disorder, double field, double occupation, int rng) {
  st.model = model;
  st.rng = model == MODEL_ISING ? rng : RNG_PHILOX;
  st.disorder = model == 0 ? disorder : (disorder == DIS_FERRO ? DIS_FERRO : DIS_EA);
  st.hmag = field;
  st.q = q;
  st.D = D;
  st.L = L;
  st.N = 1;
  for (int d = 0; d < D; ++d) st.N *= L;
  st.R = R;
  st.K = K;
  st.seed = seed;
  st.sweeps = 0;
  st.steps = 0;
  st.samples.clear();
  const int slots = K * R;
  /* site occupied iff its dilution random is below floor(2^32 occupation) */
  const uint64_t T_occ = (uint64_t)std::floor(std::ldexp(occupation, 32));
  for (int s : sample_ids) {
    Sample smp;
    smp.s = s;
    smp.J.assign((size_t)D * st.N, 1);
    for (int d = 0; d < D; ++d)
      for (uint32_t i = 0; i < (uint32_t)st.N; ++i) {
        int J;
        if (model == MODEL_PERM) J = perm_coupling_index(seed, s, d, i);
        else if (st.disorder == DIS_EA) J = coupling_bit(seed, s, d, i) ? -1 : 1;
        else if (st.disorder == DIS_DAFF) J = -1;  /* antiferromagnet */
        else J = 1;                                /* ferromagnet, RFIM */
        smp.J[(size_t)d * st.N + i] = (int8_t)J;
      }
    smp.x.assign(st.N, 1);
    smp.hs.assign(st.N, 1);
    for (uint32_t i = 0; i < (uint32_t)st.N; ++i) {
      if (st.disorder == DIS_RFIM) smp.hs[i] = field_sign_bit(seed, s, i) ? -1 : 1;
      if (st.disorder == DIS_DAFF) smp.x[i] = ((uint64_t)occupation_random(seed, s, i) < T_occ) ? 1 : 0;
    }
    smp.spin.assign(slots, std::vector<int8_t>(st.N));
    for (int sl = 0; sl < slots; ++sl)
      for (uint32_t i = 0; i < (uint32_t)st.N; ++i)
        smp.spin[sl][i] = model == 0 ? (ising_init_bit(seed, s, sl, i) ? -1 : 1)
                                     : (int8_t)(potts_init_state(seed, s, sl, i) % q);
    smp.slot_at.assign(R, std::vector<int>(K));
    for (int a = 0; a < R; ++a)
      for (int k = 0; k < K; ++k) smp.slot_at[a][k] = k;
    smp.accepted.assign(R, std::vector<uint64_t>(K > 1 ? K - 1 : 0, 0));
    if (st.rng == RNG_WHEEL) {
      const uint32_t rows = (uint32_t)st.N / (uint32_t)L;
      smp.wheels.assign(slots, std::vector<Wheel>());
      for (int sl = 0; sl < slots; ++sl)
        for (uint32_t row = 0; row < rows; ++row)
          for (int c = 0; c < 2; ++c) smp.wheels[sl].push_back(wheel_seeded(seed, s, sl, row, c));
    }
    st.samples.push_back(smp);
  }
  for (auto& smp : st.samples) {
    smp.E_run.assign(slots, 0);
    smp.F_run.assign(slots, 0);
    for (int sl = 0; sl < slots; ++sl) {
      smp.E_run[sl] = energy(st, smp, sl);
      if (model == 0) smp.F_run[sl] = field_sum(st, smp, sl);
    }
  }
}

/* ---- observables (Sec. 4.1) ---- */

/* Bond part of Eq. (2): E_J = -sum over bonds of J_ij x_i x_j s_i s_j (EA:
 * x = 1).  Potts: E = -sum over bonds of J_ij delta(s_i, s_j).  Every bond is
 * counted once, as the forward bond of its lower end along d. */
int64_t energy(const State& st, const Sample& smp, int slot) {
  const std::vector<int8_t>& s = smp.spin[slot];
  int64_t E = 0;
  for (uint32_t i = 0; i < (uint32_t)st.N; ++i)
    for (int d = 0; d < st.D; ++d) {
      uint32_t j = neighbour(st, i, d, +1);
      int J = smp.J[(size_t)d * st.N + i];
      if (st.model == MODEL_ISING) {
        E -= (int64_t)J * smp.x[i] * smp.x[j] * s[i] * s[j];
      } else if (st.model == MODEL_POTTS) {
        E -= (s[i] == s[j]) ? J : 0;
      } else {
        /* Eq. (3): the bond is satisfied iff s_i = pi_ij(s_j) */
        int pi[4];
        perm_unrank(J, pi);
        E -= (s[i] == pi[s[j]]) ? 1 : 0;
      }
    }
  return E;
}

/* M = sum_i x_i s_i */
int64_t magnetisation(const State& st, const Sample& smp, int slot) {
  int64_t M = 0;
  for (uint32_t i = 0; i < (uint32_t)st.N; ++i) M += (int64_t)smp.x[i] * smp.spin[slot][i];
  return M;
}

/* Field part of Eq. (2) in units of |h|: F = sum_i sign(h_i) x_i s_i, so the
 * energy is E_J - |h| F. */
int64_t field_sum(const State& st, const Sample& smp, int slot) {
  int64_t F = 0;
  for (uint32_t i = 0; i < (uint32_t)st.N; ++i) F += (int64_t)smp.hs[i] * smp.x[i] * smp.spin[slot][i];
  return F;
}

void potts_counts(const State& st, const Sample& smp, int slot, int64_t* counts) {
  for (int k = 0; k < st.q; ++k) counts[k] = 0;
  for (uint32_t i = 0; i < (uint32_t)st.N; ++i) counts[smp.spin[slot][i]] += 1;
}

/* Sec. 4.1 overlap between two real replicas of one sample (times N). */
int64_t overlap(const State& st, const Sample& smp, int slot_a, int slot_b) {
  int64_t Q = 0;
  for (uint32_t i = 0; i < (uint32_t)st.N; ++i) {
    if (st.model == 0)
      Q += (int64_t)smp.x[i] * smp.spin[slot_a][i] * smp.spin[slot_b][i];
    else
      Q += (smp.spin[slot_a][i] == smp.spin[slot_b][i]) ? 1 : 0;
  }
  return Q;
}

/* ---- one sweep (Sec. 2.2), colour 0 then colour 1 (Sec. 3.1) ---- */

void sweep_ising(const State& st, Sample& smp, int slot, int algo, double beta, uint64_t t) {
  std::vector<int8_t>& s = smp.spin[slot];
  const int D = st.D;
  for (int c = 0; c < 2; ++c) {
    for (uint32_t i = 0; i < (uint32_t)st.N; ++i) {
      if (colour(st, i) != c) continue;
      /* the wheel of the site's row and colour gives one number per site and
       * sweep, empty sites included, in increasing x */
      uint32_t r_wheel = 0;
      if (st.rng == RNG_WHEEL) r_wheel = smp.wheels[slot][(i / (uint32_t)st.L) * 2 + c].next();
      if (!smp.x[i]) continue; /* an empty site carries no spin */
      /* local field of the bonds: phi = sum_j J_ij x_j s_j; v = s_i phi */
      int phi = 0;
      for (int d = 0; d < D; ++d) {
        uint32_t jf = neighbour(st, i, d, +1);
        uint32_t jb = neighbour(st, i, d, -1);
        phi += smp.J[(size_t)d * st.N + i] * smp.x[jf] * s[jf];
        phi += smp.J[(size_t)d * st.N + jb] * smp.x[jb] * s[jb];
      }
      const int v = s[i] * phi;
      /* x = s_i (phi + h_i): the field adds +|h| if s_i h_i > 0, else -|h| */
      double w = 0.0;
      if (st.hmag != 0.0) w = (s[i] * smp.hs[i] > 0) ? st.hmag : -st.hmag;
      const double x = (double)v + w;
      const double dE = 2.0 * x; /* energy change if s_i flips */
      const uint32_t r = st.rng == RNG_WHEEL ? r_wheel : ising_random(st.seed, smp.s, slot, i, t);
      bool flip;
      if (algo == 0) {
        /* Metropolis: dE <= 0 is always taken; else with prob exp(-beta dE) */
        flip = (dE <= 0.0) || ((uint64_t)r < table_metropolis_x(beta, x));
      } else {
        /* heat bath, Eq. (4) for the current value: keep with prob
         * 1/(1+exp(-2 beta x)) */
        flip = !((uint64_t)r < table_heatbath_x(beta, x));
      }
      if (flip) {
        smp.E_run[slot] += 2 * v;
        smp.F_run[slot] -= 2 * smp.hs[i] * s[i];
        s[i] = (int8_t)-s[i];
      }
    }
  }
}

void sweep_potts(const State& st, Sample& smp, int slot, double beta, uint64_t t) {
  std::vector<int8_t>& s = smp.spin[slot];
  const int q = st.q;
  std::vector<int> n(q);
  std::vector<uint64_t> T(q - 1);
  for (int c = 0; c < 2; ++c) {
    for (uint32_t i = 0; i < (uint32_t)st.N; ++i) {
      if (colour(st, i) != c) continue;
      /* n_k = sum_j J_ij [s_j == k]: minus the local energy of state k */
      std::fill(n.begin(), n.end(), 0);
      for (int d = 0; d < st.D; ++d) {
        uint32_t jf = neighbour(st, i, d, +1);
        uint32_t jb = neighbour(st, i, d, -1);
        n[s[jf]] += smp.J[(size_t)d * st.N + i];
        n[s[jb]] += smp.J[(size_t)d * st.N + jb];
      }
      table_potts(beta, q, n.data(), T.data());
      const uint32_t r = potts_random(st.seed, smp.s, slot, i, t);
      int knew = q - 1;
      for (int k = 0; k < q - 1; ++k)
        if ((uint64_t)r < T[k]) {
          knew = k;
          break;
        }
      smp.E_run[slot] += n[s[i]] - n[knew];
      s[i] = (int8_t)knew;
    }
  }
}

/* Eq. (3) heat bath: n_c counts the bonds of site i satisfied when s_i = c.
 * A forward bond (i, i + e_d) carries pi = pi_d(i) and is satisfied iff
 * c = pi(s_j); a backward bond (i - e_d, i) carries pi = pi_d(i - e_d) and is
 * satisfied iff s_{i - e_d} = pi(c).  The new state follows the cumulative
 * thresholds of exp(beta n_c), as for model 1. */
void sweep_perm(const State& st, Sample& smp, int slot, double beta, uint64_t t) {
  std::vector<int8_t>& s = smp.spin[slot];
  int n[4];
  uint64_t T[3];
  for (int c = 0; c < 2; ++c) {
    for (uint32_t i = 0; i < (uint32_t)st.N; ++i) {
      if (colour(st, i) != c) continue;
      for (int k = 0; k < 4; ++k) n[k] = 0;
      for (int d = 0; d < st.D; ++d) {
        const uint32_t jf = neighbour(st, i, d, +1);
        const uint32_t jb = neighbour(st, i, d, -1);
        int pf[4], pb[4];
        perm_unrank(smp.J[(size_t)d * st.N + i], pf);
        perm_unrank(smp.J[(size_t)d * st.N + jb], pb);
        for (int cand = 0; cand < 4; ++cand) {
          if (cand == pf[s[jf]]) n[cand] += 1;
          if (s[jb] == pb[cand]) n[cand] += 1;
        }
      }
      table_potts(beta, 4, n, T);
      const uint32_t r = potts_random(st.seed, smp.s, slot, i, t);
      int knew = 3;
      for (int k = 0; k < 3; ++k)
        if ((uint64_t)r < T[k]) {
          knew = k;
          break;
        }
      smp.E_run[slot] += n[s[i]] - n[knew];
      s[i] = (int8_t)knew;
    }
  }
}

/* ---- measurement rows, indexed by temperature k (not slot) ---- */

static int mag_entries(const State& st) {
  if (st.model != 0) return st.q;
  return (st.disorder == DIS_RFIM || st.disorder == DIS_DAFF) ? 2 : 1;
}

void measure_all(const State& st, int64_t* E, int64_t* M, int64_t* Q) {
  const int K = st.K, R = st.R, q = st.q, mq = mag_entries(st);
  for (size_t si = 0; si < st.samples.size(); ++si) {
    const Sample& smp = st.samples[si];
    for (int k = 0; k < K; ++k) {
      for (int a = 0; a < R; ++a) {
        const int slot = smp.slot_at[a][k] * R + a;
        const size_t row = (si * K + k) * R + a;
        if (E) E[row] = energy(st, smp, slot);
        if (M) {
          if (st.model != 0) {
            potts_counts(st, smp, slot, M + row * q);
          } else if (mq == 2) {
            M[row * 2] = magnetisation(st, smp, slot);
            M[row * 2 + 1] = field_sum(st, smp, slot);
          } else {
            M[row] = magnetisation(st, smp, slot);
          }
        }
      }
      if (Q && R >= 2) {
        const int sa = smp.slot_at[0][k] * R + 0;
        const int sb = smp.slot_at[1][k] * R + 1;
        Q[si * K + k] = overlap(st, smp, sa, sb);
      }
    }
  }
}

static void append_row(State& st) {
  const size_t S = st.samples.size();
  const size_t nEM = S * st.K * st.R;
  const size_t nM = nEM * (size_t)mag_entries(st);
  const size_t nQ = S * st.K;
  size_t e0 = st.ser_E.size(), m0 = st.ser_M.size(), q0 = st.ser_Q.size();
  st.ser_E.resize(e0 + nEM);
  st.ser_M.resize(m0 + nM);
  st.ser_Q.resize(q0 + nQ, 0);
  st.ser_sweep.push_back(st.sweeps);
  measure_all(st, &st.ser_E[e0], &st.ser_M[m0], st.R >= 2 ? &st.ser_Q[q0] : nullptr);
}

/* nsweeps sweeps of every configuration; each configuration uses the beta
 * of the temperature its slot currently holds.  Configurations are
 * independent between swap steps, so samples are spread over threads; every
 * sweep of every configuration is the plain serial loop above. */
void run_sweeps(State& st, int algo, const double* beta, uint64_t nsweeps, uint32_t measure_every,
                int nthreads) {
  const int R = st.R, K = st.K;
  uint64_t done = 0;
  while (done < nsweeps) {
    /* advance to the next measurement point (or the end) */
    uint64_t chunk = nsweeps - done;
    if (measure_every) {
      uint64_t to_next = measure_every - (st.sweeps % measure_every);
      chunk = std::min(chunk, to_next);
    }
    const uint64_t t0 = st.sweeps;
    auto work = [&](size_t first, size_t stride) {
      for (size_t si = first; si < st.samples.size(); si += stride) {
        Sample& smp = st.samples[si];
        for (int a = 0; a < R; ++a)
          for (int k = 0; k < K; ++k) {
            const int tslot = smp.slot_at[a][k];
            const int slot = tslot * R + a;
            for (uint64_t t = t0; t < t0 + chunk; ++t) {
              if (st.model == MODEL_ISING)
                sweep_ising(st, smp, slot, algo, beta[k], t);
              else if (st.model == MODEL_POTTS)
                sweep_potts(st, smp, slot, beta[k], t);
              else
                sweep_perm(st, smp, slot, beta[k], t);
            }
          }
      }
    };
    int nt = std::max(1, std::min<int>(nthreads, (int)st.samples.size()));
    if (nt == 1) {
      work(0, 1);
    } else {
      std::vector<std::thread> th;
      for (int w = 0; w < nt; ++w) th.emplace_back(work, (size_t)w, (size_t)nt);
      for (auto& x : th) x.join();
    }
    st.sweeps += chunk;
    done += chunk;
    if (measure_every && st.sweeps % measure_every == 0) append_row(st);
  }
}

/* Parallel tempering swap step: for every chain (sample, replica) and for
 * k = 0..K-2 in order, exchange the temperatures of the configurations at k
 * and k+1 with probability min(1, exp((beta_k - beta_k+1)(E_k - E_k+1))). */
void pt_swap(State& st, const double* beta) {
  const int R = st.R, K = st.K;
  for (auto& smp : st.samples) {
    for (int a = 0; a < R; ++a) {
      for (int k = 0; k + 1 < K; ++k) {
        const int A = smp.slot_at[a][k], B = smp.slot_at[a][k + 1];
        const int64_t EA = energy(st, smp, A * R + a);
        const int64_t EB = energy(st, smp, B * R + a);
        const int64_t d = EB - EA;
        const double db = beta[k] - beta[k + 1];
        bool swap;
        if (d == 0 || db == 0.0 || ((d > 0) != (db > 0.0))) {
          swap = true; /* db * d <= 0: the exchange does not lower the weight */
        } else {
          const uint32_t r = pt_random(st.seed, smp.s, a, k, st.steps);
          const double dba = db > 0 ? db : -db;
          const int64_t dabs = d > 0 ? d : -d;
          swap = (uint64_t)r < table_pt(dba, dabs);
        }
        if (swap) {
          smp.slot_at[a][k] = B;
          smp.slot_at[a][k + 1] = A;
          smp.accepted[a][k] += 1;
        }
      }
    }
  }
  st.steps += 1;
}

}  // namespace oracle
