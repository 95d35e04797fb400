// kernels.h -- host-side launchers of the libsoma kernels (internal).
#pragma once

#include <string>
#include <vector>

#include "common.cuh"

namespace soma {

// Launch shape of the sweep kernel for chains of N particles: Q pairs of
// particles per lane, G whole chains per 32-lane tile.
struct SweepShape {
  int Q;
  uint32_t G;
  uint64_t n_tiles;
  bool vec;
  bool pair;  // even N <= 64: one even and one odd particle per lane
  bool big;   // 64-bit particle indices (M >= 2^32)
  int move;   // 0 uniform, 1 smart Monte Carlo, 2 learned
  bool learned_tc;  // learned move with the network on the tensor cores
  bool learned_umma;  // ... through tcgen05 (else warp-level mma.sync)
  bool molecule;      // molecule-parallel iteration (one thread per chain)
  size_t smem;        // dynamic shared memory of the sweep kernel
  int block;
  int grid;
};

SweepShape sweep_shape(uint64_t n_chains, uint32_t N, int sm_count, int grid_dtype, int move,
                       bool learned_fp32 = false, bool learned_umma = false,
                       bool molecule = false);
cudaError_t launch_sweep_uniform(const SweepArgs& a, const SweepShape& s, int grid_dtype,
                                 cudaStream_t st);

cudaError_t launch_init(const Geom& g, float* x, float* y, float* z, double sigma, int sm_count,
                        cudaStream_t st);
// Re-label whole chains in Morton order of the 8^3-cell block of their first
// particle: src and dst are 3-plane position buffers, keys holds n_pad >=
// n_chains (a power of two) 64-bit words of scratch.
cudaError_t launch_sort_chains(const Geom& g, const float* src, uint64_t src_plane, float* dst,
                               uint64_t dst_plane, uint64_t* keys, uint64_t n_pad, int sm_count,
                               cudaStream_t st);
// seq/arch: the per-chain type sequences of a mixture (NULL: diblocks of N_A A particles);
// alen: particles of each architecture (NULL: all N), absent slots not counted
cudaError_t launch_histogram(const Geom& g, const float* x, const float* y, const float* z,
                             uint32_t* n, int sm_count, cudaStream_t st,
                             const uint64_t* seq = nullptr, const uint8_t* arch = nullptr,
                             const uint8_t* alen = nullptr);
cudaError_t launch_range_check(const float* p, uint64_t n, float lim, unsigned* flag, int sm_count,
                               cudaStream_t st);
cudaError_t launch_fields(const FieldArgs& a, unsigned* arrive, int grid_dtype, int sm_count,
                          cudaStream_t st);
cudaError_t launch_convert_fields(const void* w, int grid_dtype, float* dst, uint64_t n,
                                  cudaStream_t st);

// FP64 observables: partial sums per block into part, then one block folds
// them in a fixed order into out (device).
//   out[0] = sum over bonds |b|^2, out[1] = sum over chains |R_e|^2,
//   out[2] = sum over cells of K(c) (Eq. discrete-ham, without rho dL^3/N),
//   out[3] = max over cells of n_A + n_B.
constexpr int OBS_BLOCKS = 1024;
// part: 5 * OBS_BLOCKS doubles; out: b2, Re2 sums, K sum, max cell, external energy
cudaError_t launch_observables(const Geom& g, const float* x, const float* y, const float* z,
                               const uint32_t* n, double inv_rho, double kappaN, double chiN,
                               int hamiltonian, const float* ext, double* part, double* out,
                               cudaStream_t st);

// S(q) for k <= SQ_MAX wave vectors; tw holds per q the FP64 twiddles
// (cos, sin) of the three axes, laid out [q][nx + ny + nz][2].
constexpr int SQ_MAX = 32;
constexpr int SQ_BLOCKS = 512;
cudaError_t launch_structure_factor(const Geom& g, const uint32_t* n, const double* tw, int k,
                                    double* part, double* out, cudaStream_t st);

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n,
                          cudaStream_t st);
// out[4i..4i+3] = the three normals and ln u a smart Monte Carlo move takes
// from draw words[4i..4i+3]
cudaError_t launch_smc_draws(const uint32_t* words, float* out, size_t n, int sm_count,
                             cudaStream_t st);

cudaError_t launch_sweep_batch(const BatchArgs& a, int grid, int block, int grid_dtype,
                               cudaStream_t st);
cudaError_t launch_fields_batch(const BatchArgs& a, uint32_t total_cells, unsigned* arrive,
                                unsigned* err, int grid_dtype, int sm_count, cudaStream_t st);
int batch_kernel_blocks_per_sm(int block, int grid_dtype);

cudaError_t launch_sweep_learned(const SweepArgs& a, const SweepShape& s, int grid_dtype,
                                 const void* wq, cudaStream_t st);
cudaError_t launch_esjd_grad(const TrainArgs& t, int grid_dtype, int sm_count, cudaStream_t st);
cudaError_t launch_adam(float* w, float* m, float* v, const float* grad, void* wq, float lr,
                        float b1, float b2, float eps, int step, float inv_n, cudaStream_t st);
cudaError_t launch_quantize(const float* w, void* wq, cudaStream_t st);
const void* learned_kernel_ptr(int Q, int grid_dtype);
const void* learned_tc_kernel_ptr(int grid_dtype, bool umma);
// one warp waits (at most limit polls) for an mbarrier phase nobody completes
cudaError_t launch_wait_probe(uint32_t limit, unsigned* err, cudaStream_t st);
// molecule-parallel sweep kernel for chains of N particles (one thread per
// chain, MOL_BLOCK threads and chains per block); *smem receives its dynamic
// shared memory (prepare: allow the kernel that much, once at create)
constexpr int MOL_BLOCK = 128;
const void* molecule_kernel_ptr(uint32_t N, int grid_dtype, size_t* smem, bool prepare);
// smart Monte Carlo sweep kernel: paired layout (even N <= 64, 32-bit indices) or general
const void* smc_kernel_ptr(int Q, bool pair, int grid_dtype);
// Smart Monte Carlo table (omega and the central-difference field force per
// type and cell, float4, A then B) from the omega planes of storage type
// grid_dtype; rebuilt after every field update of a smart Monte Carlo system.
cudaError_t launch_smc_table(const Geom& g, const void* wA, const void* wB, float4* tab,
                             int grid_dtype, int sm_count, cudaStream_t st);
// the same for n_t types: one float4 plane per type from the FP32 planes w
cudaError_t launch_smc_table_planes(const Geom& g, const float* w, uint32_t planes, float4* tab,
                                    int sm_count, cudaStream_t st);

// Molecules of any architecture (topology.cu): the architecture array of
// Sec. 3.2.1 and the independent sets derived from it.
// The bond lists of the array are re-encoded per particle: one 32-bit word
// with its degree, its first three partners, type, set and the number of sets,
// and a 64-bit mask of all its partners (bit j: bonded to particle j of the
// molecule) read only for particles with more than three.
struct TopoArgs {
  SweepArgs s;               // geometry, positions, fields, tile shape (G = 64/N)
  const uint64_t* pmask;     // partners of particle i of architecture a: [a*64 + i]
  const uint32_t* ptab;      // [a*64 + i]: degree, first three partners, type, set, sets
  const uint8_t* mol_arch;   // architecture of every molecule
  const uint8_t* alen;       // particles of each architecture (the slots past it are absent)
  // n_t types: type of particle i of architecture a ([a*64 + i]), the field
  // planes (n_types * cells) and the count planes of both parities
  const uint8_t* ttab;
  const float* wt;
  uint32_t* nt0;
  uint32_t* nt1;
};
struct TopologyTables {
  std::vector<uint64_t> pmask;   // n_arch * 64
  std::vector<uint32_t> ptab;    // n_arch * 64
  std::vector<uint8_t> ttab;     // n_arch * 64, type of each particle
  uint32_t max_type = 0;
  std::vector<uint8_t> nsets;    // n_arch
  std::vector<uint64_t> seq;     // type bits (bit i: particle i is B)
  std::vector<uint32_t> bonds;   // bonds per architecture
  std::vector<uint8_t> len;      // particles per architecture (<= N; the rest absent)
};
// Checks an architecture array against a system of N particle slots per
// molecule (an architecture holds 1..N particles, the first slots of its
// molecules) and derives the tables -- an absent slot has table word 0 (no
// sets), no partners and type byte 0xFF; returns an empty string or what is
// wrong.
std::string topology_tables(const uint32_t* words, uint64_t n_words, const uint32_t* start,
                            uint32_t n_arch, uint32_t N, TopologyTables* out,
                            uint32_t n_types = 2);
// smc: the smart Monte Carlo move (the table s.smc_tab holds one plane per type)
int topology_grid(int grid_dtype, bool big, int sm_count, uint64_t n_tiles, bool types = false,
                  bool smc = false);
cudaError_t launch_sweep_topology(const TopoArgs& a, int grid, int grid_dtype, bool big,
                                  cudaStream_t st, bool types = false, bool smc = false);
// the molecule-parallel iteration for molecules of any architecture (N <= 64);
// the grid helper also allows the kernel its shared memory (call it before
// the first launch, outside stream capture)
int molecule_topology_grid(uint32_t N, int grid_dtype, int sm_count, uint64_t n_chains);
cudaError_t launch_molecule_topology(const TopoArgs& a, int grid, int grid_dtype, cudaStream_t st,
                                     bool types = false);
// out[0] = sum over the bonds of the architectures of |b|^2, out[1] = sum over
// the molecules of |r_last - r_0|^2 with r_last the last particle of each
// molecule's architecture (lengths alen) (FP64); part: 2 OBS_BLOCKS doubles
cudaError_t launch_topology_bonds(const Geom& g, const float* x, const float* y, const float* z,
                                  const uint64_t* pmask, const uint8_t* mol_arch,
                                  const uint8_t* alen, double* part, double* out, cudaStream_t st);

// n_t particle types (types.cu).
constexpr int TYPES_MAX = 8;
struct TypesArgs {
  Geom g;
  uint32_t* n0;              // count planes, n_types * cells each; the sweep of step s
  uint32_t* n1;              // counts into planes (s+1)&1
  float* w;                  // field planes, n_types * cells
  unsigned long long* d_sweep;
  uint32_t n_types;
  int after_sweep;           // as FieldArgs
  int hamiltonian;           // 0: K^0_inter, 1: K^1_inter
  float inv_rho;             // 1/(rho_0 dL^3)
  float kappa0;              // kappaN/N
  double inv_rho_f64;
  float chi0[TYPES_MAX * TYPES_MAX];    // chi_ij N / N
  double chiN[TYPES_MAX * TYPES_MAX];   // chi_ij N
};
cudaError_t launch_fields_types(const TypesArgs& a, unsigned* arrive, int sm_count,
                                cudaStream_t st);
cudaError_t launch_histogram_types(const Geom& g, const float* x, const float* y, const float* z,
                                   const uint8_t* ttab, const uint8_t* mol_arch, uint32_t* n,
                                   int sm_count, cudaStream_t st);
// n_i | n_j << 16 per cell from the type planes n (for the composition S(q))
cudaError_t launch_pack_type_pair(const uint32_t* n, uint32_t cells, uint32_t ti, uint32_t tj,
                                  uint32_t* out, unsigned* err, int sm_count, cudaStream_t st);
// out[2] = sum over cells of the energy per cell, out[3] = largest total count,
// out[4] = 0 (no external potential); part: 2 * OBS_BLOCKS doubles
cudaError_t launch_observables_types(const TypesArgs& a, double kappaN, const uint32_t* n,
                                     double* part, double* out, cudaStream_t st);

// Entry-point helpers implemented in api.cu (messages go to soma_last_error).
}  // namespace soma
#include "../../include/soma.h"
namespace soma {
soma_status describe(const soma_system_desc* d, Geom* g);
soma_status report(soma_status st, const char* msg);
soma_status report_cuda(cudaError_t e, const char* what);
}  // namespace soma
