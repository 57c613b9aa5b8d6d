/*
 * ianus.h -- C ABI of the GB300 spin-glass Monte Carlo library (libianus.so).
 *
 * The library runs the checkerboard Metropolis / heat-bath sweep of the
 * lattice spin models of "Simulating spin systems on IANUS, an FPGA-based
 * computer" (Sec. 2 and Sec. 3.1 of the paper):
 *
 *   - the 3D (and 2D) Edwards-Anderson +-J Ising spin glass, Eq. (2) with
 *     x_i = 1, h_i = 0, J_ij = +-1 i.i.d. (Sec. 2.1);
 *   - a q = 4 Potts glass H = -sum_<ij> J_ij delta(s_i, s_j), J_ij = +-1,
 *     a J-weighted variant of the glassy Potts model of Eq. (3);
 *
 * with single-spin Metropolis and heat-bath updates (Sec. 2.2), the
 * two-colour (bipartite) parallel update (Sec. 3.1), integer look-up-table
 * acceptance against 32-bit random numbers (Sec. 3.2, Sec. 3.3), energy,
 * magnetisation and replica-overlap measurements (Sec. 4.1) and parallel
 * tempering, which Sec. 2.2 names as a required add-on without giving rules.
 *
 * All signatures use plain C types and pointers.  Host pointers are owned by
 * the caller.  Every entry point returns an ianus_status and never aborts,
 * exits or prints.  Every device operation is enqueued on the lattice's CUDA
 * stream; the calls documented as synchronous synchronise that stream only.
 * The run-time specialised bit-sliced sweeps and the Potts sweeps are
 * launched as programmatic dependents: they wait for the previous kernel on
 * the stream to complete before touching memory, and let the next kernel's
 * blocks start early.  A caller kernel enqueued after a
 * sweep with the programmatic-serialisation attribute must itself wait
 * (griddepcontrol.wait / cudaGridDependencySynchronize) before reading the
 * lattice; plain launches are ordered as usual.
 *
 * ------------------------------------------------------------------------
 * Lattice, colours, bonds (Sec. 2.1; Sec. 3.1)
 * ------------------------------------------------------------------------
 *   D in {2,3} (the permutation Potts model: D in {2,3,4}), side L even and
 *   >= 2, N = L^D sites, periodic boundaries.
 *   Site index i = x + L*(y + L*(z + L*w))  (missing coordinates are 0).
 *   Colour c(i) = (x + y + z + w) mod 2.  A sweep updates every colour-0 site,
 *   then every colour-1 site; no bond joins two sites of the same colour.
 *   Bonds are stored as forward bonds J_d(i) joining i and i + e_d
 *   (d = 0..D-1, periodic); the backward bond of i along d is J_d(i - e_d).
 *   For L = 2 the forward and backward neighbour coincide but the two bonds
 *   are distinct.
 *
 * Configurations.  A lattice object holds n_samples disorder samples; each
 * sample has n_temps * n_replicas spin configurations ("slots") that share
 * the sample's couplings.  Slot sigma = tslot * n_replicas + a, where a is the
 * replica index and tslot the temperature index the slot started at.  With
 * n_temps > 1 the slots of one chain (sample s, replica a) exchange
 * temperatures by parallel tempering; a configuration keeps its slot (and
 * its random stream) and only its temperature label moves.
 *
 * Ising encoding.  Spin bit b = (1 - s)/2 (1 means s = -1); coupling bit
 * c = (1 - J)/2.  Bond (i,j) is unsatisfied (J s_i s_j = -1) iff
 * b_i ^ b_j ^ c_ij = 1.  u_i = number of unsatisfied bonds at i (0..2D).
 *   Metropolis flip cost  dE_i = 4D - 4 u_i.
 *   Heat-bath local field x_i = s_i h_i = 2D - 2 u_i.
 *   Total energy E = -sum_bonds J s s = 2U - D N, U = unsatisfied bonds.
 *
 * ------------------------------------------------------------------------
 * Random stream (replaces the Parisi-Rapuano wheel of Sec. 3.3, Eq. (5))
 * ------------------------------------------------------------------------
 *   Generator: Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw,
 *   "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Key
 *   (k0,k1) = (seed & 0xffffffff, seed >> 32); counter (c0,c1,c2,c3);
 *   output (x0,x1,x2,x3).  Every random number is a function of the seed and
 *   of its coordinates only, so results do not depend on memory layout,
 *   kernel choice, launch shape or on how sweeps are split across calls.
 *   Tags: SPIN = 1, J = 2, INIT = 3, POTTS = 4, PINIT = 5, PT = 6, H = 7,
 *   X = 8, PERM = 9, WHEEL = 10.
 *   Sample s lives in group g = s >> 6 at lane l = s & 63.
 *
 *   Ising update random r(s, sigma, i, t), t = absolute sweep index:
 *     for plane pair m = 0..15:
 *       (x0..x3) = Philox(key, c0 = i, c1 = t & 0xffffffff,
 *                         c2 = (SPIN << 28) | (m << 24) | (sigma << 12) | g,
 *                         c3 = t >> 32)
 *       W[2m] = x0 | x1 << 32,  W[2m+1] = x2 | x3 << 32
 *     r = sum_{p=0..31} bit_l(W[p]) << (31 - p)      (plane 0 is the MSB)
 *   Deciding r < T from the most significant plane down and stopping at the
 *   first plane where r and T differ gives the same decision.
 *
 *   Couplings: J_d(i) of sample s is -1 iff bit l of (x0 | x1 << 32) of
 *     Philox(key, c0 = i, c1 = d, c2 = (J << 28) | g, c3 = 0) is set.
 *     (IANUS_DISORDER_FERRO and RFIM: every J = +1; DAFF: every J = -1.)
 *     Both models use this stream.
 *   Random-field signs (RFIM): h_i of sample s is -|h| iff bit l of
 *     (x0 | x1 << 32) of Philox(key, c0 = i, c1 = 0, c2 = (H << 28) | g,
 *     c3 = 0) is set, else +|h|.  (DAFF: h_i = +|h| everywhere.)
 *   Dilution (DAFF): site i of sample s is occupied (x_i = 1) iff
 *     r_x < floor(ldexp(occupation, 32)), r_x assembled from bit-planes as the
 *     update random, with c1 = 0 and c2 = (X << 28) | (m << 24) | g,
 *     c3 = 0.  (Other disorder kinds: x_i = 1.)
 *   Parisi-Rapuano wheels (IANUS_RNG_WHEEL, Sec. 3.3, Eq. (5)): the Ising
 *     update random of a site is drawn instead from the wheel of its
 *     (sample s, slot sigma, row, colour c), row = i / L:
 *       I(k) = I(k-24) + I(k-55) mod 2^32,  R(k) = I(k) xor I(k-61),
 *     with starting values I(-61 + n), n = 0..60, = x_{n & 3} of
 *     Philox(key, c0 = row, c1 = s, c2 = (WHEEL << 28) | ((n >> 2) << 24) |
 *     (sigma << 12) | c, c3 = 0), and I(-61) made odd (full period).  In sweep
 *     t the colour-c site of the row with x = 2 j + ((c + row parity) mod 2)
 *     takes r = R(t L/2 + j), empty sites included; the decision and tables
 *     are those of the plane stream.
 *   Initial Ising spin of (s, sigma, i): s = -1 iff bit l of (x0 | x1 << 32)
 *     of Philox(key, c0 = i, c1 = 0, c2 = (INIT << 28) | (sigma << 12) | g,
 *     c3 = 0) is set.
 *   Potts update random: r = x_{s & 3} of Philox(key, c0 = i,
 *     c1 = t & 0xffffffff, c2 = (POTTS << 28) | (sigma << 16) | (s >> 2),
 *     c3 = t >> 32).
 *   Potts initial state: x_{s & 3} >> 30 of Philox(key, c0 = i, c1 = 0,
 *     c2 = (PINIT << 28) | (sigma << 16) | (s >> 2), c3 = 0).
 *   Permutation couplings (IANUS_POTTS4_PERM, Eq. (3)): bond (d, i) of
 *     sample s carries permutation number p = floor(24 x / 2^32), x = x_{s & 3}
 *     of Philox(key, c0 = i, c1 = d, c2 = (PERM << 28) | (s >> 2), c3 = 0),
 *     where permutations of (0,1,2,3) are numbered in lexicographic order
 *     (0 = (0,1,2,3), 23 = (3,2,1,0)).  It is stored and exchanged as the
 *     8-bit code pi(0) | pi(1) << 2 | pi(2) << 4 | pi(3) << 6.
 *     (IANUS_DISORDER_FERRO: every pi is the identity.)
 *   Parallel-tempering random for chain (s, a), temperature pair k, swap
 *     step tau: x_{s & 3} of Philox(key, c0 = k, c1 = tau & 0xffffffff,
 *     c2 = (PT << 28) | (a << 16) | (s >> 2), c3 = tau >> 32).
 *   Field limits: slots < 4096, groups < 4096, samples < 2^18.
 *
 * ------------------------------------------------------------------------
 * Acceptance tables (the look-up table of Sec. 3.2, 32-bit randoms Sec. 3.3)
 * ------------------------------------------------------------------------
 *   Built once per beta on the host in IEEE double precision, in exactly
 *   this order, with std::exp, std::ldexp and std::floor; values lie in
 *   [0, 2^32] and the decision is (uint64)r < T, so a probability p is
 *   applied as floor(2^32 p) / 2^32.
 *   Metropolis (Sec. 2.2): dE <= 0 always flips (no random compare);
 *     for dE in {4, 8, 12} (2D: {4, 8}):
 *     T_M(dE) = floor(ldexp(exp(-beta * dE), 32)); flip iff r < T_M(dE).
 *   Heat bath (Sec. 2.2, Eq. (4)), x = s_i h_i in {-2D, ..., 2D} step 2:
 *     T_H(x) = floor(ldexp(1.0 / (1.0 + exp(-2.0 * beta * x)), 32));
 *     keep s_i iff r < T_H(x), else flip.  This is Eq. (4) written for the
 *     current spin value, so a gauge transformation maps trajectories onto
 *     each other bit for bit.
 *   Potts heat bath, n_k = sum_j J_ij [s_j == k] in -6..6:
 *     w_k = exp(beta * n_k); S0 = w0; S1 = S0 + w1; S2 = S1 + w2;
 *     Z = S2 + w3; T_k = floor(ldexp(S_k / Z, 32)) for k = 0, 1, 2;
 *     new state = smallest k in 0..2 with r < T_k, else 3.
 *   Permutation Potts heat bath (Eq. (3)): n_k = number of bonds of site i
 *     satisfied when s_i = k, in 0..2D: a forward bond (i, i + e_d) with
 *     permutation pi is satisfied iff k = pi(s_{i+e_d}), a backward bond
 *     (i - e_d, i) with permutation pi iff s_{i-e_d} = pi(k).  Same
 *     thresholds and selection as above.  Temperatures with 2 D beta > 700
 *     are rejected (EINVAL).
 *   Parallel tempering (pair k of temperatures k and k+1):
 *     db = beta[k] - beta[k+1]; energies of the configurations at
 *     temperatures k and k+1 are E_A and E_B, d = E_B - E_A (a multiple of 4
 *     in the +-J model); swap iff db * d <= 0, else iff
 *     r < T_PT(k, |d|) = floor(ldexp(exp(-|db| * |d|), 32)).  This is the
 *     usual acceptance min(1, exp(db * (E_A - E_B))).  Pairs are visited for
 *     k = 0 .. n_temps-2 in ascending order within one swap step.
 *
 * Ising-like models with fields and dilution (Eq. (2): RFIM, DAFF).  An
 * empty site (x_i = 0) carries no spin and is never updated.  For an occupied
 * site, v = s_i sum_j J_ij x_j s_j (an integer in -2D..2D) and
 * x = (double)v + w with w = +|h| when s_i h_i > 0 and w = -|h| otherwise
 * (w = +0.0 when |h| = 0); dE = 2.0 * x.
 *   Metropolis: flip iff dE <= 0 or r < floor(ldexp(exp(-beta * dE), 32));
 *   heat bath: keep iff r < floor(ldexp(1.0 / (1.0 + exp(-2.0 * beta * x)), 32)).
 * With |h| = 0 and x_i = 1 these are the EA tables above (v = 2D - 2u).
 *
 * Measurements (Sec. 4.1): exact int64 values.
 *   Ising: E = -sum_bonds J s s, M = sum_i s_i, Q = sum_i s_i^0 s_i^1.
 *   Potts: E = -sum_bonds J delta(s_i, s_j); "magnetisation" = the four
 *     state counts n_k; Q = sum_i delta(s_i^0, s_i^1).
 *   Permutation Potts: E = -sum_bonds delta(s_i, pi_ij(s_j)) over forward
 *     bonds (i, j = i + e_d); counts and Q as for Potts.
 *   RFIM / DAFF: "energy" = the bond part E_J = -sum_bonds J x_i x_j s_i s_j;
 *     "magnetisation" = two values, M = sum_i x_i s_i and the field sum
 *     F = sum_i sign(h_i) x_i s_i, so that E = E_J - |h| F;
 *     Q = sum_i x_i s_i^0 s_i^1.
 */
#ifndef IANUS_H
#define IANUS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IANUS_ABI_VERSION 3u

typedef struct ianus_lattice ianus_lattice; /* opaque, library-owned */

typedef enum {
  IANUS_OK = 0,
  IANUS_EINVAL = 1,      /* invalid argument or configuration            */
  IANUS_ENOMEM = 2,      /* device or host allocation failed              */
  IANUS_ECUDA = 3,       /* a CUDA runtime call failed                    */
  IANUS_ETIMEOUT = 4,    /* a bounded device wait expired                 */
  IANUS_EUNSUPPORTED = 5,/* valid request this build does not implement   */
  IANUS_ESTATE = 6       /* lattice is in an error state / bad state blob */
} ianus_status;

typedef enum {
  IANUS_EA_PM_J = 0,     /* Ising-like models of Eq. (2): EA +-J, RFIM, DAFF      */
  IANUS_POTTS4_J = 1,    /* q = 4 Potts glass H = -sum J_ij delta(s_i, s_j)      */
  IANUS_POTTS4_PERM = 2  /* glassy Potts model of Eq. (3), permutation couplings */
} ianus_model;
typedef enum { IANUS_METROPOLIS = 0, IANUS_HEATBATH = 1 } ianus_algo;
typedef enum {
  IANUS_LAYOUT_AUTO = 0,   /* BITS64 for Ising, U8X4 for Potts              */
  IANUS_LAYOUT_I8 = 1,     /* Ising: one int8 per spin (the plain kernel)   */
  IANUS_LAYOUT_BITS64 = 2, /* Ising: one uint64 per site holds 64 samples   */
  IANUS_LAYOUT_U8X4 = 3    /* Potts: one uint32 per site holds 4 samples    */
} ianus_layout;
typedef enum {
  IANUS_DISORDER_PM_J = 0,   /* EA: J = +-1 i.i.d., no field, no dilution        */
  IANUS_DISORDER_FERRO = 1,  /* J = +1, no field, no dilution (tests)             */
  IANUS_DISORDER_RFIM = 2,   /* random-field Ising model: J = +1, h_i = +-|h|     */
  IANUS_DISORDER_DAFF = 3    /* diluted antiferromagnet in a field: J = -1,
                                h_i = |h|, x_i = 1 with probability occupation */
} ianus_disorder;

/* Random stream of the Ising-like update (see the stream definitions). */
typedef enum {
  IANUS_RNG_PHILOX = 0,  /* the counter-based plane stream (every layout)       */
  IANUS_RNG_WHEEL = 1    /* Parisi-Rapuano wheels, Eq. (5) (layout I8 only)     */
} ianus_rng;

typedef struct {
  uint32_t abi_version;     /* must equal IANUS_ABI_VERSION                 */
  int32_t model;            /* ianus_model                                  */
  int32_t dim;              /* 2 or 3 (IANUS_POTTS4_PERM: 2, 3 or 4)         */
  int32_t L;                /* even, >= 2                                   */
  int32_t n_samples;        /* disorder samples, >= 1                       */
  int32_t n_replicas;       /* real replicas per sample and temperature     */
  int32_t n_temps;          /* temperatures; > 1 enables parallel tempering */
  int32_t layout;           /* ianus_layout                                 */
  int32_t disorder;         /* ianus_disorder                               */
  uint32_t series_capacity; /* rows kept by the device measurement series   */
  uint64_t seed;
  void* device_buffer;      /* optional caller-owned device memory, >= ianus_required_bytes */
  size_t device_buffer_bytes;
  void* cuda_stream;        /* cudaStream_t; NULL = the legacy default stream */
  double field;             /* |h| >= 0 (RFIM, DAFF); must be 0 otherwise      */
  double occupation;        /* DAFF site occupation probability in [0, 1]      */
  int32_t rng;              /* ianus_rng; WHEEL needs the Ising-like model and
                               layout I8 (AUTO picks I8), else EUNSUPPORTED    */
} ianus_config;

/* Device bytes a lattice with this configuration uses (state, couplings,
 * tables, series).  Returns 0 for an invalid configuration.  Host only. */
size_t ianus_required_bytes(const ianus_config* cfg);

/* Validates cfg, takes device memory (cfg->device_buffer if non-NULL, which
 * the caller keeps alive until ianus_destroy; else cudaMalloc), and fills
 * the couplings and the initial configuration from the seed on the device
 * (Sec. 2.1: quenched J_ij; initial state from the INIT/PINIT streams).
 * Sweep and swap counters start at 0, temperatures at the identity order.
 * Errors: EINVAL (bad cfg, out NULL, buffer too small; field not finite or
 * < 0, field != 0 for PM_J/FERRO, occupation outside [0, 1] for DAFF, Potts
 * with RFIM/DAFF), ENOMEM, ECUDA, EUNSUPPORTED (e.g. Potts with layout
 * I8/BITS64, DAFF with layout BITS64; AUTO picks I8 for DAFF).  On error
 * *out = NULL. */
ianus_status ianus_lattice_create(const ianus_config* cfg, ianus_lattice** out);

/* Runs nsweeps full sweeps (Sec. 2.2: every site once; Sec. 3.1: colour 0
 * then colour 1) of Metropolis or heat bath (algo) at inverse temperatures
 * beta[0..n_temps-1] (host array, indexed by temperature, not slot).
 * Acceptance tables are rebuilt on the host when beta or algo changes and
 * uploaded on the lattice stream.  If measure_every > 0, E, M and Q are
 * appended to the device series after every sweep whose absolute sweep
 * count is a multiple of measure_every.  Asynchronous.  Errors: EINVAL
 * (NULL, beta not finite or negative, algo out of range), EUNSUPPORTED
 * (Potts Metropolis), ECUDA, ESTATE. */
ianus_status ianus_sweep(ianus_lattice* lat, int32_t algo, const double* beta,
                         uint64_t nsweeps, uint32_t measure_every);

/* One parallel-tempering swap step (Sec. 2.2 names PT; rules in the header
 * comment above): measures the exact energies on the device (or takes them
 * from a measurement of the same state, when no sweep or state change came
 * after it), then every chain (sample, replica) visits its temperature pairs
 * in ascending order.
 * Uses the beta array of the last ianus_sweep.  Asynchronous.  Errors:
 * EINVAL (n_temps == 1 or no prior sweep), EUNSUPPORTED (Potts, RFIM,
 * DAFF: their energies E_J - |h| F are not on the integer grid of the swap
 * table), ECUDA. */
ianus_status ianus_pt_swap(ianus_lattice* lat);

/* Fused loop: repeats { ianus_sweep(swap_every sweeps, measure_every);
 * ianus_pt_swap } until nsweeps sweeps are done (nsweeps must be a multiple
 * of swap_every).  Same results as the separate calls. */
ianus_status ianus_sweep_pt(ianus_lattice* lat, int32_t algo, const double* beta,
                            uint64_t nsweeps, uint32_t swap_every,
                            uint32_t measure_every);

/* Measures the current configuration (Sec. 4.1 observables) and copies it
 * to host arrays (any may be NULL).  Synchronous.  Layouts, indexed by
 * temperature k (not slot):
 *   energy        int64 [n_samples][n_temps][n_replicas]
 *   magnetisation int64 [n_samples][n_temps][n_replicas]      (Ising)
 *                 int64 [n_samples][n_temps][n_replicas][4]   (Potts counts)
 *                 int64 [n_samples][n_temps][n_replicas][2]   (RFIM, DAFF: M, F)
 *   overlap       int64 [n_samples][n_temps]  (replicas 0 and 1; needs
 *                 n_replicas >= 2, else EINVAL when non-NULL). */
ianus_status ianus_measure(ianus_lattice* lat, int64_t* energy,
                           int64_t* magnetisation, int64_t* overlap);

/* Copies the device measurement series to the host.  Synchronous.  Row r
 * holds the absolute sweep count in sweep[r] and arrays laid out as in
 * ianus_measure; energy row r starts at energy + r * S*K*R, etc.  At most
 * cap_rows rows (the oldest kept rows first) are written; *n_rows receives
 * the number written.  If more rows were recorded than series_capacity,
 * only the last series_capacity are kept.  clear != 0 empties the series
 * afterwards. */
ianus_status ianus_read_series(ianus_lattice* lat, uint64_t* sweep,
                               int64_t* energy, int64_t* magnetisation,
                               int64_t* overlap, size_t cap_rows,
                               size_t* n_rows, int32_t clear);

/* Spins of every slot in natural site order: int8 [n_samples][slots][N]
 * with slots = n_temps * n_replicas; Ising values +-1, Potts 0..3.
 * Synchronous. */
ianus_status ianus_get_spins_i8(ianus_lattice* lat, int8_t* host);
/* Overwrites every slot's spins from the same layout (Ising values must be
 * +-1, Potts 0..3; else EINVAL).  Asynchronous w.r.t. the device. */
ianus_status ianus_set_spins_i8(ianus_lattice* lat, const int8_t* host);
/* Couplings: int8 [n_samples][dim][N], J_d(i) in {+1,-1} (permutation
 * Potts: the 8-bit permutation code as int8).  Synchronous. */
ianus_status ianus_get_couplings_i8(ianus_lattice* lat, int8_t* host);
/* Overwrites the couplings (values must be +-1, or permutation codes for the
 * permutation Potts model; else EINVAL).  Used for gauge tests. */
ianus_status ianus_set_couplings_i8(ianus_lattice* lat, const int8_t* host);
/* Site disorder of the Ising-like models (Eq. (2)): hsign int8 [n_samples][N]
 * = sign of h_i (+-1; +1 everywhere unless RFIM) and occupied int8
 * [n_samples][N] = x_i (0 or 1; 1 everywhere unless DAFF).  Either pointer
 * may be NULL.  Potts lattices: EUNSUPPORTED.  Synchronous. */
ianus_status ianus_get_sites_i8(ianus_lattice* lat, int8_t* hsign, int8_t* occupied);
/* Overwrites the site disorder of a field model (RFIM, DAFF; else
 * EUNSUPPORTED).  hsign values must be +-1 and occupied values 0 or 1 (else
 * EINVAL); the bit-sliced layout holds no dilution, so occupied must be all
 * 1 there (else EUNSUPPORTED).  Either pointer may be NULL (kept).  Used for
 * the global-flip and gauge tests. */
ianus_status ianus_set_sites_i8(ianus_lattice* lat, const int8_t* hsign, const int8_t* occupied);

/* ---- Fused serving (several jobs in the lanes of one lattice) ----
 * A pool is a bit-sliced EA lattice with n_replicas = n_temps = 1; each of
 * its n_samples / 64 groups holds up to 64 lanes.  A segment is up to 64
 * samples of a job, 64 job_group + b for b = 0..n-1, in lanes lane0 + b of one
 * group; it runs at the job's algorithm and beta.  (A job of more than 64
 * samples takes one segment per 64.)  Its lanes get the couplings and initial
 * spins that the job's own lattice (its seed, one replica, one temperature)
 * gives those samples, and each sweep draws their random planes from that
 * lattice's stream (key = the job's seed, group job_group, slot 0, sweep =
 * the segment's own sweep count).  So a job's trajectory is that
 * of its own lattice, bit for bit, whatever else the pool holds.  Once a
 * pool has a segment, ianus_sweep and ianus_pt_swap return EINVAL and
 * ianus_get_state EUNSUPPORTED on it; ianus_measure reports every lane
 * (sample index 64 group + lane). */

/* Loads samples 64 job_group .. 64 job_group + n - 1 of a job into lanes
 * [lane0, lane0 + n) of group `group`: couplings and spins from `seed`,
 * per-lane thresholds of (algo, beta), nsweeps sweeps to run (the lanes
 * freeze after them).  Errors: EINVAL (bad group, lanes, job_group (< 4096)
 * or arguments, lanes already taken, 64 segments in the group),
 * EUNSUPPORTED (not a pool-capable lattice), ECUDA.  Synchronous. */
ianus_status ianus_segment_load(ianus_lattice* lat, int32_t group, int32_t lane0, int32_t n, uint64_t seed,
                                int32_t job_group, int32_t algo, double beta, uint64_t nsweeps);
/* Frees the job whose lanes start at lane0 of `group` (its lanes freeze
 * until reused).  EINVAL if there is none.  Synchronous. */
ianus_status ianus_segment_release(ianus_lattice* lat, int32_t group, int32_t lane0);
/* Sweeps done and requested of the job at (group, lane0).  Host only. */
ianus_status ianus_segment_state(ianus_lattice* lat, int32_t group, int32_t lane0, uint64_t* sweeps_done,
                                 uint64_t* sweeps_requested);
/* Runs nsweeps sweeps of every live job of the pool (a job whose count has
 * reached its request stays frozen), as one launch per colour plus a counter
 * advance per sweep, replayed from CUDA graphs.  Asynchronous. */
ianus_status ianus_sweep_segments(ianus_lattice* lat, uint64_t nsweeps);

/* Parallel-tempering state: slot_at int32 [n_samples][n_replicas][n_temps]
 * (the temperature slot tslot holding temperature k), accepted uint64
 * [n_samples][n_replicas][n_temps-1] (swaps accepted per pair so far),
 * *swap_steps = number of swap steps done.  Any pointer may be NULL.
 * Synchronous. */
ianus_status ianus_get_pt_state(ianus_lattice* lat, int32_t* slot_at,
                                uint64_t* accepted, uint64_t* swap_steps);

/* Absolute number of sweeps done so far. */
ianus_status ianus_get_sweeps(ianus_lattice* lat, uint64_t* sweeps);

/* Checkpoint (Sec. 4.1: configurations dumped to the host).  The blob holds
 * a versioned header with the configuration, sweep and swap counters, the
 * temperature permutation, the couplings and the spins.  With host_buf NULL,
 * *n receives the size needed.  Synchronous.  ianus_set_state restores a
 * blob taken from a lattice of the same configuration (else ESTATE) and
 * clears a previous error state.  The acceptance tables of the last beta and
 * algorithm, the kernels specialised for them and captured sweep graphs are
 * kept (per-lane threshold planes are rebuilt for the restored temperature
 * permutation), so a restore into a running lattice costs only the copies. */
ianus_status ianus_get_state(ianus_lattice* lat, void* host_buf, size_t cap,
                             size_t* n);
ianus_status ianus_set_state(ianus_lattice* lat, const void* host_buf,
                             size_t n);

/* Blocks until all work queued for the lattice is done and reports a device
 * error recorded by a kernel (ETIMEOUT) or the CUDA runtime (ECUDA). */
ianus_status ianus_synchronize(ianus_lattice* lat);

/* Kernel variant for the bit-sliced sweep (results are identical; only speed
 * differs).  With one temperature the thresholds are the same in every lane
 * and the sweep kernel can be specialised for them at run time (NVRTC, a
 * fraction of a second per new table set, cached per device).
 *   0 = automatic: a lattice small enough for shared memory sweeps
 *       resident (ianus_set_resident); otherwise, with one temperature and
 *       one or two replicas, the lane-queue kernel (variant 24, below), the
 *       fastest shape measured on every lattice from L = 8 to L = 128; else
 *       the kernel with
 *       per-lane threshold bit-planes, compiled at run time for the
 *       lattice's geometry (also with several temperatures and for parallel
 *       tempering);
 *   1 = always the precompiled per-lane kernel (geometry from the launch
 *       parameters);
 *   2..9 = a specialised kernel shape: 2, 3 = lockstep plane loop with 3 or 4
 *       blocks per SM; 4..7 = a per-warp queue of the words still undecided
 *       after 4, 4, 3 or 5 lockstep plane pairs, finished 32 at a time, with
 *       3, 4, 3 or 3 blocks per SM; 8, 9 =
 *       lockstep with the two replicas interleaved in one thread, 2 or 3
 *       blocks per SM (needs two replicas; otherwise shape 2 is used);
 *   10..12 = shapes 2, 4 and a queue after 6 pairs, with the Philox blocks
 *       of two consecutive plane pairs computed together (two independent
 *       round chains in flight), 3 blocks per SM;
 *   13..16 = with 4 blocks per SM, each replica reading its coupling words
 *       again instead of holding them: the queue after 4 pairs and lockstep,
 *       each with two and with one Philox chain (13, 14 two; 15 lockstep
 *       one; 16 queue one);
 *   17..19 = two Philox chains, the class planes of both replicas computed
 *       before the first plane loop (all loads of a site in flight at once):
 *       the queue after 4 pairs with 3 blocks per SM, lockstep with 4 and
 *       with 3 blocks per SM;
 *   20, 21 = shape 17 in blocks of 128 threads, 7 or 6 blocks per SM;
 *   22..24 = the lane-queue kernel: Philox rounds 0 and 1 split into a site
 *       part and a block-uniform part, plane pairs 0..3 for every word, the
 *       lanes still undecided queued per warp and finished 32 at a time one
 *       plane pair per round; 8 or 6 blocks of 128 threads per SM (22, 23),
 *       4 blocks of 256 (24).  With no explicit launch shape its grid is one
 *       wave of about that many blocks per SM;
 *   25..27 = the persistent form of the lane-queue kernel: one cooperative
 *       launch runs every sweep between two measurements.  Each block owns
 *       a fixed range of rows and starts a colour pass once the blocks that
 *       own its sites' neighbours have finished the previous pass (bounded
 *       waits, ianus_set_persistent_wait), so there is no kernel boundary
 *       between colours; blocks of 128 threads with at least 512 (25) or
 *       128 (26) colour words, or of 256 threads with at least 512 (27), at
 *       most as many blocks as are resident at once.  Where that
 *       launch cannot run it falls back to variant 22's per-pass kernel.
 * The fastest shape depends on the lattice and the algorithm: on the L=64,
 * 256-sample x 2-replica heat-bath lattice it is the automatic one (24 in
 * its one-wave grid), which takes a fifth less time per sweep than 21 with
 * 256 words per block (ianus_set_block_words), the fastest shape before the
 * lane-queue kernel.  The
 * Python autotuner (tune.py) times the shapes on the caller's lattice.
 * The plain one-byte-per-spin layout (IANUS_LAYOUT_I8) has four sweep
 * kernels.  Variant 0 (automatic), with L = 32, 64 or 128: a block reads a
 * tile of a 64-sample group as bytes, turns it into 64-lane words in shared
 * memory (warp bit transposes of the sign bits), runs the bit-sliced update
 * there and writes the tile back as bytes (the random number of sample s
 * is bit s mod 64 of its group's plane stream, so the trajectory is the
 * same).  Variant 1: one thread per update, each drawing its own random
 * planes.  Other values, and variant 0 at other sides: a block draws the
 * planes of a site once for the site's 64-sample group and each update
 * compares an 8-bit prefix of its random number from shared memory, in
 * the word kernel (four spins of one sample per 32-bit load) when L is a
 * multiple of 4, else in the tiled kernel (one byte per thread).
 * With several temperatures every variant but 1 uses the per-lane kernel
 * compiled for the geometry.  If run-time compilation is unavailable, the
 * precompiled kernel runs.  EINVAL for other values. */
ianus_status ianus_set_variant(ianus_lattice* lat, int32_t variant);

/* Launch shape of the bit-sliced sweep: colour words handled by one block of
 * 256 threads (rounded up to a multiple of 32, whole warps); 0 restores the
 * default, a multiple of 256 that sizes the grid to about 8 blocks per SM
 * (for the lane-queue kernels 22..24: a multiple of 32 that makes the grid
 * one wave of resident blocks).
 * EINVAL above 2^24. */
ianus_status ianus_set_block_words(ianus_lattice* lat, uint32_t words_per_block);

/* Compiles (or finds in the per-process cache) the kernel that a sweep of
 * this lattice at (algo, beta[0]) under kernel variant `variant` would
 * specialise for its acceptance thresholds (the Metropolis and heat-bath
 * rules of Sec. 2.2 and Eq. (4), as the look-up table of Sec. 3.2), without
 * launching anything and without changing the lattice.  A sweep that finds no kernel compiles it on the
 * calling thread first, a fraction of a second; a server calls this on a
 * worker thread instead and runs the job meanwhile under variant 1 (the
 * precompiled kernel, same results), switching to `variant` once *ready.
 * Reads only the lattice's shape, fixed at creation, so it may run while
 * other threads sweep this or other lattices (the lattice must not be
 * destroyed before the call returns); concurrent calls compile different
 * kernels in parallel and wait for one another on the same one.
 * beta: one inverse temperature per temperature of the lattice (n_temps),
 * finite and >= 0.  *ready = 1 when the specialised kernel is now cached,
 * 0 when the variant selects none on this lattice (several temperatures,
 * a field or Potts model, the plain layout, variant 1) or run-time
 * compilation is unavailable or failed (the sweep then uses a per-lane
 * kernel, as it would anyway).  EINVAL for a null pointer, an unknown algo,
 * a variant outside 0..27 or a bad beta; ECUDA when the lattice's device
 * cannot be made current. */
ianus_status ianus_prepare_sweep(ianus_lattice* lat, int32_t algo, const double* beta, int32_t variant,
                                 int32_t* ready);

/* Waits of the persistent sweep (variants 25..27): each wait of a block for
 * its neighbours' progress is bounded by timeout_ns (default 2 s).  A wait
 * that runs out sets the device error word and the block returns; the next
 * ianus_synchronize reports IANUS_ETIMEOUT and the lattice is ESTATE
 * (restore it with ianus_set_state).  absent_block >= 0 makes that block of
 * the next launches return at once without doing its work: a wait that
 * nothing ends, for testing the timeout path (-1: none).  EINVAL for
 * timeout_ns = 0 or absent_block < -1. */
ianus_status ianus_set_persistent_wait(ianus_lattice* lat, uint64_t timeout_ns, int32_t absent_block);

/* Sweep blocks through CUDA graphs (default on): runs of at least 4 sweeps
 * between measurements are replayed from graphs of up to 64 sweeps, captured
 * on a private stream the first time each block length occurs and dropped
 * when the tables, the variant or the launch shape change.  Captured kernels
 * read the sweep index from a device counter, so results are identical with
 * and without graphs.  enable = 0 launches every kernel directly. */
ianus_status ianus_set_graphs(ianus_lattice* lat, int32_t enable);

/* Resident mode for small lattices (default on).
 *
 * Bit-sliced layout (IANUS_LAYOUT_BITS64, models of Eq. (2) without fields):
 * under the automatic kernel variant (0), a lattice whose state per (group,
 * temperature slot) fits in 220 KiB of shared memory -- R spin words and dim
 * coupling words per site and R x 33 x 8 threshold-plane words, 8 (R + dim)
 * L^dim + 2112 R bytes: 3D L <= 17 with two replicas and L <= 19 with one,
 * 2D L <= 83 and L <= 96 -- can run every block of two or more sweeps
 * between measurements in launches of up to 4096 sweeps, one thread block
 * per (group, temperature slot) holding that state, the colours separated
 * by block barriers (Sec. 3.1); measurements run between the launches as
 * usual.  A pool lattice (ianus_segment_load) sweeps the same way, one
 * block per group, when N + dim N + 264 words fit; each block advances its
 * jobs' sweep counters itself.  Same results, bit for bit, as the
 * launch-per-colour path.  enable = 1 (default) takes it where it is the
 * faster sweep: at most 512 word updates per block and sweep (R N), or
 * 1024 with at least 32 blocks (3D L = 8; 2D L <= 22 with one replica);
 * enable = 2 or 3 takes it wherever it fits; enable = 0: off.
 *
 * Plain layout: with layout I8, one
 * temperature, (1 + dim) L^dim bytes <= 200 KiB, and either one replica or no
 * measurements, each configuration is held in shared memory by one launch
 * that runs all requested sweeps (the two colours separated by barriers,
 * Sec. 3.1) and records E and M itself.  Same results as the
 * launch-per-colour path.
 *   enable = 1 (default): with few configurations (at most two blocks per SM
 *            when each is split) a thread-block cluster of C blocks holds
 *            one configuration, C the largest divisor of L in 2..16 that
 *            can be scheduled; block r owns the slab of L/C planes along the
 *            last axis, neighbours across a face come from the neighbouring
 *            block's shared memory, cluster barriers separate the colours.
 *            Otherwise one thread block per configuration.
 *   enable = 2: one thread block per configuration always.
 *   enable = 3: a cluster per configuration whenever L has a divisor in
 *            2..16 for which a cluster can be scheduled, however many
 *            configurations there are.
 *   enable = 0: off.
 * Other values: IANUS_EINVAL. */
ianus_status ianus_set_resident(ianus_lattice* lat, int32_t enable);

/* Frees what the lattice allocated.  NULL is accepted.  The caller-owned
 * device buffer, if any, is not freed. */
ianus_status ianus_destroy(ianus_lattice* lat);

/* Static, NUL-terminated description of a status code. */
const char* ianus_status_string(int32_t status);

/* ---- Measurement for callers that cannot allocate device memory ----
 *
 * The paper has no counterpart to this entry point.  It serves callers that
 * must not call cudaMalloc: code embedded in a framework that owns all device
 * memory through its own pool (a direct allocation bypasses the pool and can
 * fail when the pool has reserved the device), and serving loops where
 * cudaMalloc / cudaFree would synchronise the device and stall other streams.
 * It allocates nothing: it calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * It computes, for bit-sliced configurations in the BITS64 layout, the energy
 * E = -sum_bonds J s s and the magnetisation M = sum_i s_i of every (sample,
 * slot), the same values ianus_measure reports for a BITS64 lattice.
 *   spins          device uint64 [ceil(n_samples/64)][n_slots][L^dim], lane
 *                  l of a word = sample 64 g + l, bit 1 = spin -1, sites in
 *                  checkerboard-split order (2 (y + L z) + colour) L/2 + x/2
 *   couplings      device uint64 [ceil(n_samples/64)][dim][L^dim], same
 *                  order, bit 1 = coupling -1, J_d(i) joins i and i + e_d
 *   energy, magnetisation  device int64 [n_samples][n_slots] (written)
 *   cuda_stream    cudaStream_t the work is enqueued on (NULL = legacy stream)
 * Working storage is a fixed device array inside the library: 2 counters for
 * each of at most IANUS_NOALLOC_MAX_CONFIGS (sample, slot) pairs, 512 KiB
 * that every GPU which loads the library holds until the process exits.
 * n_samples * n_slots above that limit returns IANUS_EINVAL, as do NULL
 * pointers and invalid dim / L; a CUDA failure returns IANUS_ECUDA.
 * The first call on a device looks up that array's device address (with the
 * device current) and caches it; make that first call before any stream
 * capture.  Each call clears the counters it uses before counting, but all
 * calls share the one array: calls that may overlap on the GPU (different
 * streams, or different host threads) race and give wrong results, so
 * serialise them.  Asynchronous: results are ready when the stream is. */
#define IANUS_NOALLOC_MAX_CONFIGS 32768
ianus_status ianus_measure_bits64_noalloc(const uint64_t* spins, const uint64_t* couplings, int32_t dim,
                                          int32_t L, int32_t n_samples, int32_t n_slots, int64_t* energy,
                                          int64_t* magnetisation, void* cuda_stream);

/* ---- Host-only table builders (the look-up tables of Sec. 3.2).  These
 * need no GPU; tests compare them with an independent builder. ---- */

/* Metropolis (algo 0): out[j] = T_M(4 (j+1)) for j = 0..dim-1 (dE = 4, 8,
 * 12 in 3D).  Heat bath (algo 1): out[j] = T_H(-2 dim + 2 j) for
 * j = 0..2 dim.  Values in [0, 2^32].  n = capacity of out.  Returns the
 * count written, or 0 on bad arguments. */
size_t ianus_table_ising(int32_t dim, int32_t algo, double beta, uint64_t* out,
                         size_t n);
/* Potts heat bath: out[idx*3 + k] = T_k(n0..n3), idx = (((n0+6)*13 + n1+6)
 * *13 + n2+6)*13 + n3+6, for all 13^4 tuples (also unreachable ones).
 * n must be >= 3 * 13^4.  Returns the count written or 0. */
size_t ianus_table_potts(double beta, uint64_t* out, size_t n);
/* Potts heat bath for one tuple of counts n[0..3] (any integers, the
 * permutation model's n_k in 0..2D included): T[k] as above for k = 0..2.
 * Returns 3, or 0 on bad arguments (NULL, beta not finite or < 0). */
size_t ianus_table_potts_counts(double beta, const int32_t* n, uint64_t* T);
/* PT: out[m-1] = T_PT(|d| = 4 m) = floor(ldexp(exp(-|db| * 4m), 32)) for
 * m = 1..n, db = beta_k - beta_k1.  Returns n, or 0 on bad arguments. */
size_t ianus_table_pt(double beta_k, double beta_k1, uint64_t* out, size_t n);
/* Field models (Eq. (2), RFIM / DAFF rules above): out[(v + 2 dim) * 2 + f]
 * for v = -2 dim..2 dim and f = 1 when s_i h_i > 0, else 0; field = |h|.
 * Metropolis (algo 0): the flip threshold, 2^32 where dE = 2x <= 0.  Heat
 * bath (algo 1): the keep threshold.  n must be >= 2 (4 dim + 1).  Returns
 * the count written, or 0 on bad arguments. */
size_t ianus_table_field(int32_t dim, int32_t algo, double beta, double field, uint64_t* out, size_t n);

#ifdef __cplusplus
}
#endif

#endif /* IANUS_H */
