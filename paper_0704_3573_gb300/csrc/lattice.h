// lattice.h -- host-side definition of a lattice object and the kernel
// launchers each translation unit provides.  Internal to libianus.so.
#pragma once
#include <cstddef>
#include <algorithm>
#include <cstdint>
#include <map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ianus.h"
#include "common.cuh"

namespace ianus {

constexpr int kAccStride = 8;    // int64 accumulators per (sample, slot)
constexpr uint64_t kTwo32 = 1ull << 32;
// Field models (Eq. 2 with random fields or dilution): the I8 class of a site
// is (v + 2D) * 2 + f, v = s_i sum_j J_ij x_j s_j in -2D..2D and f = 1 when
// s_i h_i > 0; the bit-sliced class is 8 f + u with v = 2D - 2u.
constexpr int kFieldClasses = 32;
constexpr int kFieldPlaneClasses = 16;
// With dilution (DAFF) the bit-sliced local field is t = v + 2D in 0..4D,
// summed as 4 bit-planes from per-neighbour contributions c_j + 1 in {0,1,2};
// plane class 16 f + t.
constexpr int kDiluteClasses = 32;

// Truth tables of the lane-uniform threshold path: t[p] bit u = bit (31-p)
// of the class-u threshold; always bit u = (T(u) == 2^32); need bit u = the
// class compares against a random number.
struct UniformLut {
  uint8_t t[32];
  uint8_t always, need, pad0, pad1;
};

// The same for the random-field model, one table set per f = [s_i h_i > 0]
// (bit u = the class (u, f)); t[f] is laid out as the 64 bytes the field
// kernel's tail reads.
struct FieldLut {
  uint8_t t[2][2][32];            // [f][t3 (dilute models; 0 otherwise)][plane]
  uint8_t always[2][2], need[2][2];
};

// Fused serving: a job occupies the lanes [lane0, lane0 + n) of one 64-lane
// group of a pool lattice (bit-sliced, one replica, one temperature).  Its
// lanes draw the random planes of the job's own stream (key from its seed,
// its own sweep counter t), so its trajectory equals that of the job run on
// its own lattice.
struct Segment {
  uint64_t mask;      // lanes of the segment
  uint64_t t;         // sweeps done
  uint64_t t_end;     // sweeps requested
  uint32_t key_lo, key_hi;
  uint32_t lane0;
  uint32_t inv;       // heat bath: 1
  uint32_t jgroup;    // the lanes are samples 64 jgroup + (lane - lane0) of the job
  uint32_t pad;
};
constexpr int kMaxSegs = 64;  // per group

struct Lattice {
  ianus_config cfg;
  int model, D, L, S, R, K, slots, layout;
  int G;        // 64-sample groups (BITS64)
  int Q4;       // 4-sample quads (U8X4)
  uint32_t N;
  Geom geom;
  cudaStream_t stream;
  bool owns_buffer;
  uint8_t* base;
  size_t bytes;

  // device arrays (carved from base)
  void* spins;          // I8: int8 [slots][S][N]; BITS64: u64 [G][slots][N]; U8X4: u32 [slots][Q4][N]
  void* J;              // I8: int8 [S][D][N];     BITS64: u64 [G][D][N];     U8X4: u32 [Q4][D][N]
  uint64_t* thr;        // Ising: u64 [K][kMaxClasses] threshold per class u
  uint64_t* tp;         // BITS64: u64 [G][slots][kMaxClasses][kPlanes]
  uint4* ptab;          // Potts: uint4 [K][65536]; permutation Potts: [K][(2D+1)^3]
  uint64_t* pttab;      // PT: u64 [K-1][pt_len], T_PT(|d| = 4m) at m-1
  int8_t* pt_sign;      // PT: sign of beta[k] - beta[k+1], [K-1]
  int32_t* slot_at;     // [S][R][K]
  int32_t* temp_of;     // [S][R][K]
  uint64_t* accepted;   // [S][R][K-1]
  int64_t* acc;         // [S][slots][kAccStride] measurement accumulators
  int64_t* out_E;       // [S][K][R]
  int64_t* out_M;       // [S][K][R][mq]
  int64_t* out_Q;       // [S][K]
  uint64_t* ser_sweep;  // [cap]
  int64_t* ser_E;       // [cap][S*K*R]
  int64_t* ser_M;       // [cap][S*K*R*mq]
  int64_t* ser_Q;       // [cap][S*K]
  uint32_t* err;        // device error word
  uint32_t* flags;      // progress flags of the persistent sweep [kMaxPersistBlocks]
  uint64_t persist_timeout_ns;  // bound of each wait of the persistent sweep
  int32_t persist_absent;       // block told to return at once (tests), -1 = none

  // field models (RFIM, DAFF)
  int disorder;         // IANUS_DISORDER_*
  bool field;           // disorder is RFIM or DAFF
  double hmag;          // |h|
  uint64_t* fthr;       // u64 [K][kFieldClasses] threshold per field class
  uint64_t* ftp;        // BITS64 field: u64 [G][slots][kPlanes][kFieldPlaneClasses]
  int8_t* hs;           // I8 field: sign of h_i, int8 [S][N]
  int8_t* occ;          // I8 field: x_i in {0, 1}, int8 [S][N]
  uint64_t* hbits;      // BITS64 field: lane bit set where h_i < 0, u64 [G][N]
  uint64_t* xbits;      // BITS64 field: lane bit set where x_i = 1 (occupied), u64 [G][N]
  bool dilute;          // BITS64 DAFF: local field from the 4-bit sum t (plane classes kDiluteClasses)
  int fpc;              // plane classes of the field planes (kFieldPlaneClasses or kDiluteClasses)
  FieldLut flut;        // valid when flut_ok (BITS64 field model, one temperature)
  bool flut_ok;
  cudaKernel_t jitf;    // field sweep specialised for flut (null: per-lane planes)
  int jitf_algo;        // algorithm it was requested for; -1 = not yet
  // Parisi-Rapuano wheels (IANUS_RNG_WHEEL, I8 only): ring of 64 words per
  // (slot, sample, colour, row), I(k) at ring index k mod 64;
  // u32 [slots * S][2][64][rows], rows = N / L
  int rng;
  uint32_t* wheels;
  uint32_t rows;
  // fused serving (pool lattices): segment tables [G][kMaxSegs], counts [G]
  bool pool;
  Segment* segs;
  uint32_t* nseg;
  std::vector<Segment>* segs_host;
  std::vector<uint32_t>* nseg_host;
  std::vector<uint64_t>* tp_host;  // per-lane planes [G][kPlanes][kMaxClasses]

  int mq;               // magnetisation entries per configuration (1 Ising, 4 Potts, 2 field models)
  uint32_t cap;         // series capacity
  uint64_t ser_count;   // rows recorded so far (ring position = ser_count % cap)
  uint64_t ser_first;   // first row still readable
  uint32_t pt_len;      // entries per PT pair table (<= pt_cap)
  uint32_t pt_cap;      // allocated entries per pair
  uint64_t sweeps;      // absolute sweep counter
  uint64_t steps;       // PT swap steps done
  PhiloxKeys keys;
  std::vector<double> beta;  // last beta array (tables are valid for it)
  int algo;                  // last algo; -1 = none
  bool tables_ok;
  bool pt_tables_ok;
  int sticky;                // sticky error status (ESTATE after a failure)
  int variant;               // kernel variant knob (tuner), 0 = default
  int dev;                   // CUDA device current when the lattice was created
  UniformLut ulut;           // valid when ulut_ok (n_temps == 1)
  bool ulut_ok;
  cudaKernel_t jit;          // sweep kernel specialised for ulut (null: use the per-lane planes)
  cudaKernel_t jitp[2];      // per-lane-plane sweep compiled for the geometry, per algorithm (null: precompiled)
  bool jitp_tried[2];
  int jit_algo;              // algorithm the specialisation was requested for; -1 = not yet
  int jit_variant;           // variant it was built for
  uint32_t block_words;      // words per block of the bit-sliced sweep; 0 = heuristic
  // CUDA graphs of sweep blocks: the kernels of B sweeps and a counter
  // advance, captured once on a private stream and replayed on `stream`.
  uint64_t* t_dev;           // device sweep counter read by captured kernels
  bool capturing;            // launchers pass t_dev (and an offset) while true
  bool use_graphs;
  bool use_resident;         // resident mode for small I8 lattices (default on)
  int resident_mode;         // 1 = clusters when few configurations, 2 = one block each, 3 = clusters
  // The accumulators hold the measurement of the state at (acc_sweeps,
  // acc_mut) when acc_ok; mut counts changes of the state other than sweeps.
  uint64_t mut, acc_sweeps, acc_mut;
  bool acc_ok;
  bool t_dev_valid;          // *t_dev == sweeps
  cudaStream_t cap_stream;
  std::map<uint32_t, cudaGraphExec_t>* graphs;  // by block length
};

// ---- host table builders (tables.cpp) ----
size_t table_ising(int dim, int algo, double beta, uint64_t* out, size_t n);
size_t table_potts(double beta, uint64_t* out, size_t n);
// Potts heat-bath thresholds T[0..2] for one tuple of counts n[0..3].
void potts_thresholds(double beta, const int* n, uint64_t* T);
size_t table_pt(double beta_k, double beta_k1, uint64_t* out, size_t n);
// Threshold per class u = 0..2D for the unified rule "flip iff (r < T) != inv":
// Metropolis: u < D -> T_M(4D - 4u), u >= D -> 2^32 (always); inv = 0.
// Heat bath: T_H(2D - 2u), inv = 1 (keep iff r < T).
void class_thresholds(int dim, int algo, double beta, uint64_t* thr /*[kMaxClasses]*/);
// Field models: threshold per class (v + 2D) * 2 + f for the same unified
// rule; Metropolis classes with dE <= 0 get 2^32.  Unused entries are 0.
void field_thresholds(int dim, int algo, double beta, double hmag, uint64_t* thr /*[kFieldClasses]*/);

// Run-time specialised bit-sliced sweep for lat.ulut (jit.cu); null when
// runtime compilation is unavailable.  Its queued shape takes kJitSmemBytes
// of dynamic shared memory: one queue of 64 entries (5 x 8 + 3 x 4 bytes) for
// each of its 8 warps.
constexpr size_t kJitSmemBytes = 8 * 64 * (5 * 8 + 3 * 4);
cudaKernel_t jit_kernel(const Lattice& lat, const UniformLut& u, int algo, int mode, int phase_a, int min_blocks,
                        int group, int jreload, int ufirst, int block);
// The lane-queue shape of the same sweep (jit_sweep_lt.cuh): shared Philox
// rounds 0..1, four plane pairs for every word, undecided lanes queued.
cudaKernel_t jit_lt_kernel(const Lattice& lat, const UniformLut& u, int algo, int min_blocks, int block);
// Its persistent form (IANUS_JIT_PERSIST): many sweeps per launch.
cudaKernel_t jit_ltp_kernel(const Lattice& lat, const UniformLut& u, int algo, int min_blocks, int block);
// The specialised shape (>= 2) that `variant` selects on this lattice when
// its tables are lane-uniform, or 1 when it selects none (k_msc.cu).
int specialised_variant(const Lattice& lat, int variant);
// The kernel of shape v (>= 2) specialised for tables u and algorithm algo
// (0 Metropolis, 1 heat bath); null when run-time compilation is
// unavailable or fails.  Reads only the lattice's shape (D, L, R, K,
// geometry), which is fixed at creation, so any thread may call it.
cudaKernel_t specialised_sweep_kernel(const Lattice& lat, const UniformLut& u, int algo, int v);
// Lane-uniform tables of one temperature from the class thresholds
// thr[0..2D] (api.cu).
UniformLut uniform_lut(int dim, int algo, const uint64_t* thr);
constexpr int kMaxVariant = 27;  // ianus_set_variant accepts 0..kMaxVariant
constexpr int kMaxPersistBlocks = 4096;
// True when the selected variant is the persistent sweep and the lattice
// qualifies (one temperature, one or two replicas, lane-uniform tables).
bool persistent_variant(const Lattice& lat);
// Runs nsweeps sweeps from sweep t0 in one cooperative launch of the
// persistent sweep.  *ran = false (and cudaSuccess) when it cannot run here
// (no run-time compiler, or too many blocks to be resident at once): the
// caller then sweeps with the per-pass kernels.
cudaError_t launch_sweep_persistent(Lattice& lat, int inv, uint64_t t0, uint32_t nsweeps, bool* ran);
// Run-time specialised random-field sweep for lat.flut (jit.cu; null when
// unavailable).
cudaKernel_t jit_field_kernel(const Lattice& lat, int algo, int min_blocks);
// The per-lane-plane sweep (sweep_planes.cuh) compiled for the lattice's
// geometry: rt replicas at compile time (0: run time), per-warp queues.
cudaKernel_t jit_planes_kernel(const Lattice& lat, int algo, int rt, bool queue, int min_blocks, size_t smem);

// ---- launchers; each returns cudaGetLastError() of its launches ----
// I8 (k_plain.cu)
// Coupling modes of the initialisers: 0 = the J stream, 1 = every J = +1,
// 2 = every J = -1.
cudaError_t launch_init_i8(Lattice& lat, int jmode);
cudaError_t launch_init_sites_i8(Lattice& lat, double occupation);  // hs, occ from the H and X streams
cudaError_t launch_get_sites_i8(Lattice& lat, int8_t* dev_hs, int8_t* dev_occ);  // [S][N] each
cudaError_t launch_set_sites_i8(Lattice& lat, const int8_t* dev_hs, const int8_t* dev_occ);
cudaError_t launch_init_wheels(Lattice& lat);  // starting values of every wheel
cudaError_t launch_sweep_i8(Lattice& lat, int colour, uint64_t t, int inv);
cudaError_t launch_measure_i8(Lattice& lat, int want_q);
// Resident mode (one block per configuration in shared memory, many sweeps
// per launch, E/M written to the series ring): n_temps == 1, I8 layout,
// (1 + D) N bytes <= kResidentSmemMax.
constexpr size_t kResidentSmemMax = 200 * 1024;
bool resident_i8_fits(const Lattice& lat);
// Resident bit-sliced sweeps (k_resident_bits.cu): one block per (group,
// temperature slot) -- or per group of a fused pool -- holding its spins,
// couplings and threshold planes in shared memory for many sweeps.  The
// *_fits tests also ask that the resident sweep be the faster one, unless
// resident_mode >= 2 forces it wherever it fits.
bool resident_bits_fits(const Lattice& lat);
bool resident_fused_fits(const Lattice& lat);
// nsweeps sweeps t0, t0 + 1, ... of every configuration (no measurements).
cudaError_t launch_resident_bits(Lattice& lat, int inv, uint64_t t0, uint32_t nsweeps);
// nsweeps sweeps of a pool, each advancing its running segments by one.
cudaError_t launch_resident_fused(Lattice& lat, uint32_t nsweeps);
cudaError_t launch_resident_i8(Lattice& lat, int inv, uint32_t nsweeps, uint32_t measure_every);
cudaError_t launch_get_spins_i8(Lattice& lat, int8_t* dev_out);       // [S][slots][N]
cudaError_t launch_set_spins_i8(Lattice& lat, const int8_t* dev_in);
cudaError_t launch_get_couplings_i8(Lattice& lat, int8_t* dev_out);   // [S][D][N]
cudaError_t launch_set_couplings_i8(Lattice& lat, const int8_t* dev_in);
// BITS64 (k_msc.cu)
cudaError_t launch_init_bits(Lattice& lat, int jmode);
cudaError_t launch_init_sites_bits(Lattice& lat, double occupation);  // hbits (H stream), xbits (X stream)
cudaError_t launch_get_sites_bits(Lattice& lat, int8_t* dev_hs, int8_t* dev_occ);  // [S][N] each
cudaError_t launch_set_sites_bits(Lattice& lat, const int8_t* dev_hs, const int8_t* dev_occ);
cudaError_t launch_build_field_planes(Lattice& lat);                 // ftp from fthr and temp_of
// fused serving (k_msc.cu)
cudaError_t launch_load_segment(Lattice& lat, int group, uint32_t lane0, uint32_t n, uint32_t jgroup,
                                PhiloxKeys job_keys);
cudaError_t launch_sweep_fused(Lattice& lat, int colour);
cudaError_t launch_advance_segments(Lattice& lat);
cudaError_t launch_sweep_bits(Lattice& lat, int colour, uint64_t t, int inv);
// Launch with programmatic stream serialisation, for sweep kernels that
// begin with dependent_launch_entry() (k_msc.cu)
cudaError_t launch_dependent(const void* k, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t s);
size_t sweep_bits_smem(int R);  // least shared memory of the per-lane-plane sweep for R replicas
// energy_only: U of every configuration only (the PT swap needs no more)
cudaError_t launch_measure_bits(Lattice& lat, int want_q, bool energy_only = false);
cudaError_t launch_build_planes(Lattice& lat);  // tp from thr and temp_of
cudaError_t launch_get_spins_bits(Lattice& lat, int8_t* dev_out);
cudaError_t launch_set_spins_bits(Lattice& lat, const int8_t* dev_in);
cudaError_t launch_get_couplings_bits(Lattice& lat, int8_t* dev_out);
cudaError_t launch_set_couplings_bits(Lattice& lat, const int8_t* dev_in);
// U8X4 Potts (k_potts.cu)
cudaError_t launch_init_potts(Lattice& lat, int jmode);
cudaError_t launch_sweep_potts(Lattice& lat, int colour, uint64_t t);
cudaError_t launch_measure_potts(Lattice& lat, int want_q);
cudaError_t launch_get_spins_potts(Lattice& lat, int8_t* dev_out);
cudaError_t launch_set_spins_potts(Lattice& lat, const int8_t* dev_in);
cudaError_t launch_get_couplings_potts(Lattice& lat, int8_t* dev_out);
cudaError_t launch_set_couplings_potts(Lattice& lat, const int8_t* dev_in);
cudaError_t launch_overlap_potts(Lattice& lat);  // Q into acc (both Potts models)
// Permutation Potts model of Eq. (3), U8X4 storage, D = 2..4 (k_perm.cu).
// The Potts launchers above forward to these for IANUS_POTTS4_PERM.
cudaError_t launch_init_perm(Lattice& lat, int jmode);
cudaError_t launch_sweep_perm(Lattice& lat, int colour, uint64_t t);
cudaError_t launch_measure_perm(Lattice& lat, int want_q);
cudaError_t launch_get_spins_perm(Lattice& lat, int8_t* dev_out);
cudaError_t launch_set_spins_perm(Lattice& lat, const int8_t* dev_in);
cudaError_t launch_get_couplings_perm(Lattice& lat, int8_t* dev_out);
cudaError_t launch_set_couplings_perm(Lattice& lat, const int8_t* dev_in);
// compact permutation-model table: entry n0 + B (n1 + B n2), B = 2D + 1
inline uint32_t perm_table_entries(int D) { return (uint32_t)(2 * D + 1) * (2 * D + 1) * (2 * D + 1); }
// shared (k_pt.cu)
cudaError_t launch_finalize(Lattice& lat, int64_t* E, int64_t* M, int64_t* Q, uint64_t* sweep_out, int want_q);
cudaError_t launch_pt_swap(Lattice& lat);
cudaError_t launch_set_tick(Lattice& lat, uint64_t value);
cudaError_t launch_advance_tick(Lattice& lat, uint64_t by);
// Compiles the specialised bit-sliced kernel if the next sweep will use it
// (so that no compilation happens during stream capture).
void prepare_sweep_bits(Lattice& lat, int inv);

}  // namespace ianus
