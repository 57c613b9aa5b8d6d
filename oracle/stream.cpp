/*
 * stream.cpp -- the oracle's own random stream and acceptance tables.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper drives every update with a 32-bit random number compared with a
 * look-up-table value (Sec. 3.2, Sec. 3.3).  Its Parisi-Rapuano wheel
 * (Eq. (5)) is serial per wheel; the stream here is counter based instead,
 * so that every random number is a function of (seed, sample, slot, site,
 * sweep) alone.  The generator is Philox4x32-10 as published by Salmon,
 * Moraes, Dror and Shaw (SC'11): a 4-word counter goes through 10 rounds of
 * two 32x32->64 multiplications whose halves are XORed with the other
 * counter words and a round key; the key is advanced by two Weyl constants
 * between rounds.
 */
#include "oracle.h"

#include <cmath>

namespace oracle {

void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* round multipliers */
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* key increments    */
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void call(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t x[4]) {
  const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  const uint32_t ctr[4] = {c0, c1, c2, c3};
  philox4x32_10(ctr, key, x);
}

/* The 32-bit random of one Ising update, assembled in full from its 32
 * bit-planes (plane 0 is the most significant bit). */
uint32_t ising_random(uint64_t seed, int sample, int slot, uint32_t site, uint64_t sweep) {
  const uint32_t g = (uint32_t)sample >> 6;
  const int lane = sample & 63;
  uint64_t W[32];
  for (uint32_t m = 0; m < 16; ++m) {
    uint32_t x[4];
    uint32_t c2 = ((uint32_t)TAG_SPIN << 28) | (m << 24) | ((uint32_t)slot << 12) | g;
    call(seed, site, (uint32_t)(sweep & 0xffffffffu), c2, (uint32_t)(sweep >> 32), x);
    W[2 * m] = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
    W[2 * m + 1] = (uint64_t)x[2] | ((uint64_t)x[3] << 32);
  }
  uint32_t r = 0;
  for (int p = 0; p < 32; ++p) {
    uint32_t bit = (uint32_t)((W[p] >> lane) & 1u);
    r |= bit << (31 - p);
  }
  return r;
}

uint32_t potts_random(uint64_t seed, int sample, int slot, uint32_t site, uint64_t sweep) {
  uint32_t x[4];
  uint32_t c2 = ((uint32_t)TAG_POTTS << 28) | ((uint32_t)slot << 16) | ((uint32_t)sample >> 2);
  call(seed, site, (uint32_t)(sweep & 0xffffffffu), c2, (uint32_t)(sweep >> 32), x);
  return x[sample & 3];
}

uint32_t pt_random(uint64_t seed, int sample, int replica, int pair, uint64_t step) {
  uint32_t x[4];
  uint32_t c2 = ((uint32_t)TAG_PT << 28) | ((uint32_t)replica << 16) | ((uint32_t)sample >> 2);
  call(seed, (uint32_t)pair, (uint32_t)(step & 0xffffffffu), c2, (uint32_t)(step >> 32), x);
  return x[sample & 3];
}

int coupling_bit(uint64_t seed, int sample, int d, uint32_t site) {
  uint32_t x[4];
  uint32_t c2 = ((uint32_t)TAG_J << 28) | ((uint32_t)sample >> 6);
  call(seed, site, (uint32_t)d, c2, 0u, x);
  uint64_t w = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
  return (int)((w >> (sample & 63)) & 1u);
}

int ising_init_bit(uint64_t seed, int sample, int slot, uint32_t site) {
  uint32_t x[4];
  uint32_t c2 = ((uint32_t)TAG_INIT << 28) | ((uint32_t)slot << 12) | ((uint32_t)sample >> 6);
  call(seed, site, 0u, c2, 0u, x);
  uint64_t w = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
  return (int)((w >> (sample & 63)) & 1u);
}

int potts_init_state(uint64_t seed, int sample, int slot, uint32_t site) {
  uint32_t x[4];
  uint32_t c2 = ((uint32_t)TAG_PINIT << 28) | ((uint32_t)slot << 16) | ((uint32_t)sample >> 2);
  call(seed, site, 0u, c2, 0u, x);
  return (int)(x[sample & 3] >> 30);
}

int field_sign_bit(uint64_t seed, int sample, uint32_t site) {
  uint32_t x[4];
  call(seed, site, 0u, ((uint32_t)TAG_H << 28) | ((uint32_t)sample >> 6), 0u, x);
  uint64_t w = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
  return (int)((w >> (sample & 63)) & 1u);
}

/* Eq. (3) couplings: one of the 4! permutations, chosen by the 32-bit random
 * x of the bond as floor(24 x / 2^32). */
int perm_coupling_index(uint64_t seed, int sample, int d, uint32_t site) {
  uint32_t x[4];
  call(seed, site, (uint32_t)d, ((uint32_t)TAG_PERM << 28) | ((uint32_t)sample >> 2), 0u, x);
  return (int)(((uint64_t)x[sample & 3] * 24u) >> 32);
}

/* Lexicographic unranking: digit pos of the factorial number system picks
 * among the values not used yet, in increasing order. */
void perm_unrank(int index, int out[4]) {
  int pool[4] = {0, 1, 2, 3};
  int left = 4;
  const int weight[4] = {6, 2, 1, 1};
  for (int pos = 0; pos < 4; ++pos) {
    const int pick = index / weight[pos];
    index %= weight[pos];
    out[pos] = pool[pick];
    for (int m = pick; m + 1 < left; ++m) pool[m] = pool[m + 1];
    --left;
  }
}

int perm_code(int index) {
  int p[4];
  perm_unrank(index, p);
  return p[0] | (p[1] << 2) | (p[2] << 4) | (p[3] << 6);
}

int perm_index_of_code(int code) {
  for (int k = 0; k < 24; ++k)
    if (perm_code(k) == (code & 0xff)) return k;
  return -1;
}

uint32_t Wheel::next() {
  const size_t n = hist.size(); /* 61 */
  const uint32_t Ik = hist[n - 24] + hist[n - 55];
  const uint32_t R = Ik ^ hist[n - 61];
  hist.erase(hist.begin());
  hist.push_back(Ik);
  return R;
}

Wheel wheel_seeded(uint64_t seed, int sample, int slot, uint32_t row, int colour) {
  Wheel w;
  for (uint32_t n = 0; n < 61; ++n) {
    uint32_t x[4];
    const uint32_t c2 = ((uint32_t)TAG_WHEEL << 28) | ((n >> 2) << 24) | ((uint32_t)slot << 12) | (uint32_t)colour;
    call(seed, row, (uint32_t)sample, c2, 0u, x);
    w.hist.push_back(x[n & 3]);
  }
  w.hist[0] |= 1u; /* an odd value gives the additive generator its full period */
  return w;
}

/* 32-bit random of the dilution stream, assembled from its bit-planes. */
uint32_t occupation_random(uint64_t seed, int sample, uint32_t site) {
  const uint32_t g = (uint32_t)sample >> 6;
  const int lane = sample & 63;
  uint64_t W[32];
  for (uint32_t m = 0; m < 16; ++m) {
    uint32_t x[4];
    call(seed, site, 0u, ((uint32_t)TAG_X << 28) | (m << 24) | g, 0u, x);
    W[2 * m] = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
    W[2 * m + 1] = (uint64_t)x[2] | ((uint64_t)x[3] << 32);
  }
  uint32_t r = 0;
  for (int p = 0; p < 32; ++p) r |= (uint32_t)((W[p] >> lane) & 1u) << (31 - p);
  return r;
}

/* Sec. 2.2 Metropolis: a move that raises the energy by dE > 0 is taken with
 * probability exp(-beta dE); here as an integer threshold against 32-bit r. */
uint64_t table_metropolis(double beta, int dE) {
  double p = std::exp(-beta * (double)dE);
  return (uint64_t)std::floor(std::ldexp(p, 32));
}

/* Sec. 2.2 heat bath, Eq. (4): probability that spin i keeps its value,
 * x = s_i h_i, is exp(beta x) / (exp(beta x) + exp(-beta x)). */
uint64_t table_heatbath(double beta, int x) {
  double p = 1.0 / (1.0 + std::exp(-2.0 * beta * (double)x));
  return (uint64_t)std::floor(std::ldexp(p, 32));
}

/* Potts heat bath: state k has weight exp(beta n_k); cumulative sums in state
 * order 0, 1, ..., q-1 give q-1 thresholds. */
void table_potts(double beta, int q, const int* n, uint64_t* T) {
  std::vector<double> w(q);
  for (int k = 0; k < q; ++k) w[k] = std::exp(beta * (double)n[k]);
  std::vector<double> S(q);
  S[0] = w[0];
  for (int k = 1; k < q; ++k) S[k] = S[k - 1] + w[k];
  double Z = S[q - 1];
  for (int k = 0; k < q - 1; ++k) T[k] = (uint64_t)std::floor(std::ldexp(S[k] / Z, 32));
}

/* Eq. (2) with a field: dE = 2x for x = v + w (v integer, w = +-|h|). */
uint64_t table_metropolis_x(double beta, double x) {
  const double dE = 2.0 * x;
  double p = std::exp(-beta * dE);
  return (uint64_t)std::floor(std::ldexp(p, 32));
}

uint64_t table_heatbath_x(double beta, double x) {
  double p = 1.0 / (1.0 + std::exp(-2.0 * beta * x));
  return (uint64_t)std::floor(std::ldexp(p, 32));
}

/* Parallel-tempering rejection branch: probability exp(-|dbeta| |d|). */
uint64_t table_pt(double dbeta_abs, int64_t dabs) {
  double p = std::exp(-dbeta_abs * (double)dabs);
  return (uint64_t)std::floor(std::ldexp(p, 32));
}

}  // namespace oracle
