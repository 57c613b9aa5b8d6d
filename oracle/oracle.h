/*
 * oracle.h -- plain, slow CPU oracle for the checkerboard Metropolis /
 * heat-bath sweep of the EA +-J Ising glass and the q-state Potts glass.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library imports, links or calls
 * this code; only the tests, __graft_entry__.smoke() and the CPU-baseline leg
 * of bench.py use it.  It shares no code, header, table builder or constant
 * with the CUDA path: the random stream, the acceptance tables, the energy
 * code and the update rules are all re-implemented here from the paper and
 * from the published definition of Philox4x32-10.
 *
 * Every function follows the paper's steps in plain loops:
 *   Hamiltonians          Sec. 2.1, Eq. (2) (EA: x_i = 1, h_i = 0, J = +-1;
 *                         RFIM, DAFF), a J-weighted form of Eq. (3) for
 *                         Potts (model 1) and the permutation form of
 *                         Eq. (3) itself (model 2, 2 to 4 dimensions)
 *   Metropolis, heat bath Sec. 2.2 (acceptance exp(-beta dE); Eq. (4))
 *   sweep                 Sec. 2.2 (every site once per sweep)
 *   checkerboard          Sec. 3.1 (all of one colour, then the other)
 *   32-bit LUT compare    Sec. 3.2, Sec. 3.3
 *   parallel tempering    Sec. 2.2 names it; the rule is the standard one
 *   E, M, Q measurements  Sec. 4.1
 *   Parisi-Rapuano wheel  Sec. 3.3, Eq. (5) (the alternative random stream)
 */
#pragma once
#include <cstdint>
#include <vector>

namespace oracle {

/* Philox4x32 with 10 rounds (Salmon et al., SC'11). */
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

enum { TAG_SPIN = 1, TAG_J = 2, TAG_INIT = 3, TAG_POTTS = 4, TAG_PINIT = 5, TAG_PT = 6, TAG_H = 7, TAG_X = 8,
       TAG_PERM = 9, TAG_WHEEL = 10 };

/* Random streams of the Ising-like sweep: the counter-based plane stream, or
 * one Parisi-Rapuano wheel per (sample, slot, row, colour). */
enum { RNG_PHILOX = 0, RNG_WHEEL = 1 };

/* Parisi-Rapuano shift register, Eq. (5): I(k) = I(k-24) + I(k-55) mod 2^32,
 * R(k) = I(k) xor I(k-61).  hist holds I(k-61) .. I(k-1), oldest first. */
struct Wheel {
  std::vector<uint32_t> hist;
  uint32_t next();
};
/* The 61 starting values I(-61) .. I(-1) of the wheel of (sample, slot, row,
 * colour): words of the WHEEL stream; I(-61) is made odd. */
Wheel wheel_seeded(uint64_t seed, int sample, int slot, uint32_t row, int colour);

/* Models: 0 = Ising-like (Eq. 2), 1 = Potts with J = +-1 weights, 2 = the
 * glassy Potts model of Eq. (3) with permutation couplings. */
enum { MODEL_ISING = 0, MODEL_POTTS = 1, MODEL_PERM = 2 };

/* Disorder kinds of the Ising-like Hamiltonian, Eq. (2) (Sec. 2.1). */
enum { DIS_EA = 0, DIS_FERRO = 1, DIS_RFIM = 2, DIS_DAFF = 3 };

uint32_t ising_random(uint64_t seed, int sample, int slot, uint32_t site, uint64_t sweep);
uint32_t potts_random(uint64_t seed, int sample, int slot, uint32_t site, uint64_t sweep);
uint32_t pt_random(uint64_t seed, int sample, int replica, int pair, uint64_t step);
int coupling_bit(uint64_t seed, int sample, int d, uint32_t site);        /* 1 means J = -1 */
int ising_init_bit(uint64_t seed, int sample, int slot, uint32_t site);   /* 1 means s = -1 */
int potts_init_state(uint64_t seed, int sample, int slot, uint32_t site); /* 0..3           */
int field_sign_bit(uint64_t seed, int sample, uint32_t site);             /* 1 means h_i < 0 */
uint32_t occupation_random(uint64_t seed, int sample, uint32_t site);     /* plane-assembled  */
/* Permutation coupling of bond (d, site) of sample s: an index 0..23 into the
 * permutations of (0,1,2,3) in lexicographic order. */
int perm_coupling_index(uint64_t seed, int sample, int d, uint32_t site);
void perm_unrank(int index, int out[4]);   /* the index-th permutation, lexicographic */
int perm_code(int index);                  /* pi(0) | pi(1) << 2 | pi(2) << 4 | pi(3) << 6 */
int perm_index_of_code(int code);          /* inverse of perm_code; -1 if not a permutation */

/* Acceptance thresholds, values in [0, 2^32]; decision is r < T. */
uint64_t table_metropolis(double beta, int dE);
uint64_t table_heatbath(double beta, int x);
/* q-state Potts heat bath; n has q entries; T receives q-1 cumulative values. */
void table_potts(double beta, int q, const int* n, uint64_t* T);
uint64_t table_pt(double dbeta_abs, int64_t dabs);
/* Ising-like model with a field: x = v + w (see sweep_ising). */
uint64_t table_metropolis_x(double beta, double x); /* flip prob for dE = 2x > 0 */
uint64_t table_heatbath_x(double beta, double x);   /* keep prob                */

struct Sample {
  int s;                                    /* true sample index (drives the streams) */
  std::vector<int8_t> J;                    /* [D][N] forward bonds J_d(i): +-1, or the
                                               permutation index (model 2)             */
  std::vector<int8_t> x;                    /* [N] dilution, 1 = occupied              */
  std::vector<int8_t> hs;                   /* [N] sign of the field h_i (+-1)         */
  std::vector<std::vector<int8_t>> spin;    /* [slots][N]; Ising +-1, Potts 0..q-1     */
  std::vector<int64_t> E_run;               /* [slots] incremental (bond) energy      */
  std::vector<int64_t> F_run;               /* [slots] incremental field sum          */
  std::vector<std::vector<int>> slot_at;    /* [R][K] temperature slot at temperature k */
  std::vector<std::vector<uint64_t>> accepted; /* [R][K-1] */
  std::vector<std::vector<Wheel>> wheels;   /* [slots][row * 2 + colour], RNG_WHEEL only */
};

struct State {
  int model;        /* MODEL_* */
  int disorder;     /* DIS_* for the Ising-like model */
  double hmag;      /* |h| */
  int rng;          /* RNG_* (Ising-like model) */
  int q;            /* Potts states (4 in the library; any >= 2 here) */
  int D, L, N, R, K;
  uint64_t seed;
  uint64_t sweeps;  /* absolute sweep counter t */
  uint64_t steps;   /* parallel-tempering swap steps tau */
  std::vector<Sample> samples;
  /* measurement series: rows of (sweep, E[S][K][R], M[S][K][R](*q for Potts), Q[S][K]) */
  std::vector<uint64_t> ser_sweep;
  std::vector<int64_t> ser_E, ser_M, ser_Q;
};

/* geometry */
void site_coords(const State& st, uint32_t i, int* x);
uint32_t neighbour(const State& st, uint32_t i, int d, int dir); /* dir +1 / -1 */
int colour(const State& st, uint32_t i);

void init_state(State& st, int model, int q, int D, int L, const std::vector<int>& sample_ids,
                int R, int K, uint64_t seed, int disorder, double field, double occupation, int rng = RNG_PHILOX);
int64_t energy(const State& st, const Sample& smp, int slot);
int64_t magnetisation(const State& st, const Sample& smp, int slot);
int64_t field_sum(const State& st, const Sample& smp, int slot);
void potts_counts(const State& st, const Sample& smp, int slot, int64_t* counts);
int64_t overlap(const State& st, const Sample& smp, int slot_a, int slot_b);

/* One sweep of one configuration at inverse temperature beta (sweep index t). */
void sweep_ising(const State& st, Sample& smp, int slot, int algo, double beta, uint64_t t);
void sweep_potts(const State& st, Sample& smp, int slot, double beta, uint64_t t);
void sweep_perm(const State& st, Sample& smp, int slot, double beta, uint64_t t);

/* nsweeps sweeps of every configuration; beta indexed by temperature. */
void run_sweeps(State& st, int algo, const double* beta, uint64_t nsweeps, uint32_t measure_every,
                int nthreads);
void measure_all(const State& st, int64_t* E, int64_t* M, int64_t* Q);
void pt_swap(State& st, const double* beta);

}  // namespace oracle
