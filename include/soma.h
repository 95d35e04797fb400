/*
 * soma.h -- C ABI of libsoma: single-chain-in-mean-field (SCMF) Monte-Carlo
 * simulation of soft, coarse-grained diblock copolymer melts on one GB300
 * (sm_103a), after "SOMA: Soft coarse grained Monte-Carlo Acceleration"
 * (arXiv:1711.03828).
 *
 * One SCMF cycle (Sec. 2.2 of the paper) is
 *   1. an independent-set Monte-Carlo step of every particle against frozen
 *      quasi-instantaneous fields omega_t(c) (Sec. 2.2 move + Eq. delta-e; the
 *      "SET" iteration of Sec. 3.1.2: even then odd chain positions, or the
 *      reverse, the order drawn per chain and step),
 *   2. the integer occupation numbers n_t(c) on the collocation grid
 *      (Eq. density-characteristics, Sec. 3.1.1),
 *   3. the field update omega_A/B (Eq. omega-fields, option K^0).
 *
 * Units and layout (fixed for every entry point):
 *   - lengths are in units of the grid spacing dL; the grid is cubic
 *     (Sec. 2.1), so box_Re[d] / grid[d] must agree on the three axes;
 *   - positions are FP32, structure of arrays: one buffer of 3*M floats holds
 *     x[0..M), y[0..M), z[0..M); particle m = chain*N + i; positions are
 *     unwrapped (periodic images are folded only to find the cell) and must
 *     stay within |x| < 2^18 dL, where the cell fold is exact;
 *   - particle i of a chain is type A iff i < N_A = floor(f*N + 1/2);
 *   - the cell of a position is (floor(x) mod grid_x, ...), index
 *     (cz*grid_y + cy)*grid_x + cx;
 *   - occupation numbers are packed per cell: n_A in bits 0..15, n_B in bits
 *     16..31 (the paper stores them as 16-bit integers, Sec. 3.1.1);
 *   - omega_t(c) is the per-particle field energy in kT of Eq. (omega-fields):
 *     omega_A/B = (kappaN/N)(phi_A + phi_B - 1) -/+ (chiN/(2N))(phi_A - phi_B),
 *     phi_t = n_t / (rho_0 dL^3), rho_0 dL^3 = M / cells.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) with counter
 * (id lo32, id hi32, w, purpose<<24 | replica_id) and key (seed lo32, seed
 * hi32); a move of particle m in sweep s uses purpose 1, id m, w s.  There is
 * no generator state (the paper's Sec. 3.2.3 stores a PCG state per thread).
 *
 * Execution: every call is asynchronous on the handle's stream unless it says
 * otherwise; calls that return data to the host synchronise that stream.  No
 * call aborts the process: each returns a soma_status, and soma_last_error()
 * gives a message for the calling thread.  Device-side conditions (a 16-bit
 * count saturating) are recorded in a sticky device word and reported by the
 * next synchronising call.
 *
 * Ownership: a soma_t owns every device buffer it allocates (in soma_create)
 * and frees them in soma_destroy.  Buffers passed by the caller are borrowed
 * for the duration of the call and never retained.
 */
#ifndef SOMA_H
#define SOMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SOMA_ABI_VERSION 2

typedef enum {
  SOMA_OK = 0,
  SOMA_EINVAL = -1,     /* invalid argument or description; nothing was done */
  SOMA_ENOMEM = -2,     /* a device or host allocation failed */
  SOMA_ECUDA = -3,      /* a CUDA runtime call failed (message in soma_last_error) */
  SOMA_EOVERFLOW = -4,  /* a 16-bit occupation number reached 0xC000 (sticky) */
  SOMA_ETIMEOUT = -5,   /* a bounded device wait gave up (sticky) */
  SOMA_ESTATE = -6      /* call not valid in the handle's current state */
} soma_status;

typedef enum { SOMA_MOVE_UNIFORM = 0, SOMA_MOVE_SMC = 1, SOMA_MOVE_LEARNED = 2 } soma_move;
/* How a sweep visits the particles (Sec. 3.1.2).  The SET scheme moves the
 * even and then the odd chain positions (or the reverse) as two sets of
 * independent particles: the order is drawn per chain and step (RANDOM) or
 * always even first (FIXED).  SOMA_ITERATION_MOLECULE is the molecule-
 * parallel scheme: one thread per chain makes the chain's N attempts one after
 * another, each on a particle chosen at random (Philox purpose 3, id
 * chain*N + attempt; the particle is ((word 3 & 0xFF) * N) >> 8, the
 * acceptance uniform the top 24 bits of word 3); uniform moves only. */
typedef enum { SOMA_SET_ORDER_RANDOM = 0, SOMA_SET_ORDER_FIXED = 1,
               SOMA_ITERATION_MOLECULE = 2 } soma_set_order;
typedef enum { SOMA_GRID_F32 = 0, SOMA_GRID_BF16 = 1, SOMA_GRID_F16 = 2 } soma_grid_dtype;

/* desc.flags bits.  By default soma_create labels the chains in spatial order:
 * increasing Morton code of the 8^3-cell block holding each chain's first
 * particle (ties keep the drawing order), so that chains with nearby labels
 * are near each other and share field values in cache.  Labels of molecules
 * are arbitrary (the paper distributes whole molecules freely, Sec. 3.1.1);
 * the label decides the particle indices and so the Philox streams.
 * SOMA_FLAG_NO_SORT keeps the drawing order (chain k = k-th draw). */
#define SOMA_FLAG_NO_SORT 1
/* The learned proposal's network runs on the tensor cores (BF16 operands and
 * activations, FP32 accumulation) for even N <= 64: by default as warp-level
 * mma.sync products (32 feature rows per warp, weights held in registers).
 * SOMA_FLAG_LEARNED_UMMA evaluates it as one tcgen05.mma product per layer
 * over a 4-warp block's 128 rows with the accumulator in tensor memory
 * (correct, but slower here: the block's warps must meet for every one of the
 * twelve dependent products of a tile).  SOMA_FLAG_LEARNED_FP32 evaluates it
 * on the CUDA cores in FP32 (the precision the parity tests use). */
#define SOMA_FLAG_LEARNED_FP32 2
#define SOMA_FLAG_LEARNED_UMMA 4

/* Description of one system: a melt of n_chains linear A-B diblock chains.
 * struct_size must be sizeof(soma_system_desc) (ABI versioning). */
typedef struct soma_system_desc {
  uint32_t struct_size;
  uint32_t N;            /* particles per chain, 1..256 */
  uint64_t n_chains;     /* >= 1; M = n_chains*N < 2^40 */
  double f;              /* A fraction of a chain, 0..1 */
  double box_Re[3];      /* box edges in units of R_e0 (> 0) */
  uint32_t grid[3];      /* cells per axis, 1..4096; dL = box/grid equal on all axes */
  uint32_t hamiltonian;  /* interaction option of Eq. (hamil-pair): 0 K^0_inter,
                            1 K^1_inter (omega_A/B = kappa_0 (phi_A + phi_B - 1)
                            + chi_0 phi_B/A, Eq. omega-fields second line) */
  double chiN;           /* Flory-Huggins chi_0 N (Eq. hamil-pair) */
  double kappaN;         /* inverse compressibility kappa_0 N (Eq. hamil-comp) */
  double a_Re;           /* maximal trial displacement per axis in R_e0;
                            <= 0 selects 0.5/sqrt(N-1) (0.5 for N = 1) */
  int32_t move;          /* soma_move */
  int32_t set_order;     /* soma_set_order */
  int32_t grid_dtype;    /* soma_grid_dtype: storage type of omega */
  int32_t flags;         /* SOMA_FLAG_* bits */
  uint64_t seed;         /* Philox key */
  uint32_t replica_id;   /* Philox counter word 3, low 24 bits */
  uint32_t reserved1;
  void* stream;          /* cudaStream_t to run on; NULL: the handle creates its own */
  /* Chain sharding (see soma_shard_sweep): this handle holds chains
     [chain_offset, chain_offset + n_chains) of a system of n_chains_total
     chains.  n_chains_total = 0: the handle holds the whole system
     (chain_offset must then be 0). */
  uint64_t chain_offset;
  uint64_t n_chains_total;
} soma_system_desc;

typedef struct soma_t soma_t;

/* Observables, reduced in FP64 on the device.  Energies in kT, lengths in dL. */
typedef struct soma_obs {
  double E_b;        /* sum over bonds of (k0/2)|b|^2, Eq. (h-bond), (V-harmonic) */
  double E_nb;       /* Eq. (discrete-ham) with K_fluc + K_inter of the current n */
  double E_tot;      /* E_b + E_nb + E_ext */
  double Re2;        /* mean over chains of |r_{N-1} - r_0|^2 */
  double Re2_rel;    /* Re2 / R_e0^2 */
  double b2;         /* mean over bonds of |r_{i+1} - r_i|^2 */
  uint64_t accepted; /* accepted moves since creation */
  uint64_t attempted;/* attempted moves since creation */
  uint64_t sweeps;   /* completed SCMF cycles since creation */
  uint32_t max_cell; /* largest n_A + n_B of any cell */
  uint32_t reserved;
  double E_ext;      /* sum over cells of n_A ext_A + n_B ext_B (soma_set_external);
                        E_tot = E_b + E_nb + E_ext */
} soma_obs;

/* Accumulated device time per kernel while timing is on (soma_set_timing). */
typedef struct soma_timing {
  double ms_sweep;        /* MC sweep kernel (move + fused occupation count) */
  double ms_fields;       /* field-update kernel */
  uint64_t sweep_launches;  /* launches since timing was last enabled (or creation) */
  uint64_t field_launches;
  uint64_t kernel_launches; /* every kernel this handle launched since creation */
} soma_timing;

/* Create a system: validate desc, allocate device state, draw the initial
 * configuration (first particle of each chain uniform in the box, then
 * Gaussian bonds with <b^2> = R_e0^2/(N-1); Sec. 2.1 with b0 = sqrt(3/k0)),
 * label the chains in spatial order unless desc.flags has SOMA_FLAG_NO_SORT,
 * then compute n and omega (first stage of the SCMF cycle, Sec. 2.2).
 * Returns SOMA_EINVAL before touching the GPU when desc is invalid.
 * On success *out owns the state; on failure *out is NULL. */
soma_status soma_create(const soma_system_desc* desc, soma_t** out);

/* Free all device state of h (synchronises h's stream).  NULL is a no-op. */
soma_status soma_destroy(soma_t* h);

/* Run n SCMF cycles: n x (MC step of every particle against the frozen
 * fields with the occupation count fused into it, then the field update).
 * Asynchronous.  Sec. 2.2 cycle; Sec. 3.1.2 SET iteration; Eq. (delta-e). */
soma_status soma_sweep(soma_t* h, uint32_t n);

/* Recompute n and omega from the current positions (first stage of the SCMF
 * cycle, Eqs. density-characteristics and omega-fields).  Asynchronous. */
soma_status soma_update_fields(soma_t* h);

/* Chain sharding over ranks (Sec. 3.1.1: whole molecules are distributed over
 * the ranks, every rank moves its own molecules against the same fields, and
 * the one exchange of a cycle is the sum of the occupation numbers over the
 * ranks before each rank computes the fields itself).
 *
 * A shard is a handle whose desc has n_chains_total > 0: it holds chains
 * [chain_offset, chain_offset + n_chains) of a system of n_chains_total
 * chains (n_chains_total * N < 2^32) on the whole system's box and grid.
 * Every random number is keyed on the whole system's chain and particle
 * indices and rho_0 dL^3 counts all n_chains_total * N particles, so shards
 * that hold every chain once, driven through the three calls below with
 * their counts summed, reproduce bit for bit the handle that holds the whole
 * system (given the same positions: soma_create labels each shard's chains
 * in spatial order by itself, which is a different labelling of the same
 * system; soma_set_positions gives any other).  A shard takes the uniform,
 * smart Monte Carlo and learned moves, the SET and the molecule-parallel
 * iterations and molecular architectures (soma_set_topology); not n_t types
 * nor batches.  soma_sweep and soma_update_fields refuse a shard
 * (SOMA_ESTATE): they would use its own particles' counts alone.
 *
 * One cycle of a shard h, on h's stream:
 *   soma_shard_sweep(h, buf, cells)     MC step of h's particles; their packed
 *                                       occupation numbers are copied to buf
 *   <sum buf over all shards, in place> e.g. ncclAllReduce(buf, buf, cells,
 *                                       ncclUint32, ncclSum, comm, stream): the
 *                                       packed A | B<<16 halves add exactly
 *                                       while every global count is < 2^16
 *   soma_shard_fields(h, buf, cells)    n := buf, omega from it, cycle done
 * After soma_create or soma_set_positions the fields are those of h's own
 * particles; start with soma_shard_counts(h, buf, cells), the sum, and
 * soma_shard_fields(h, buf, cells).  The calls must alternate in that order
 * (a counts or sweep call, then a fields call): SOMA_ESTATE otherwise.
 * buf holds cells = grid cells uint32 entries, device or host memory (the
 * copies use cudaMemcpyDefault; with host memory the call returns after its
 * copy); it is borrowed for the call only.  SOMA_EINVAL: NULL argument or
 * cells differs from the grid size.  Overflow of a summed count is reported
 * as for soma_sweep (SOMA_EOVERFLOW, sticky). */
soma_status soma_shard_counts(soma_t* h, uint32_t* counts, size_t cells);
soma_status soma_shard_sweep(soma_t* h, uint32_t* counts, size_t cells);
soma_status soma_shard_fields(soma_t* h, const uint32_t* summed, size_t cells);

/* Copy the packed occupation numbers (n_cells = grid cells entries; bits 0..15
 * n_A, 16..31 n_B) to dst (device pointer if dst_on_device, else host).
 * Synchronises.  SOMA_EINVAL if n_cells differs from the grid size. */
soma_status soma_get_density(soma_t* h, uint32_t* dst, size_t n_cells, int dst_on_device);

/* Copy omega as FP32: dst[0..cells) = omega_A, dst[cells..2 cells) = omega_B
 * (converted from the storage type).  n must be 2*cells.  Synchronises. */
soma_status soma_get_fields(soma_t* h, float* dst, size_t n, int dst_on_device);

/* Copy positions (3*M floats, SoA x|y|z, dL units).  Synchronises. */
soma_status soma_get_positions(soma_t* h, float* dst, size_t n, int dst_on_device);

/* Replace positions (3*M floats, SoA).  Does not recompute the fields: call
 * soma_update_fields to make n and omega follow.  Every coordinate must be
 * finite with |x| < 2^18 dL (the range in which the cell fold is exact;
 * chains diffuse far less than that in any feasible run).  The check runs on
 * the device after the copy: on a violation the call returns SOMA_EINVAL and
 * the handle refuses soma_sweep, soma_update_fields and training (SOMA_ESTATE)
 * until a later call sets valid positions.  Synchronises. */
soma_status soma_set_positions(soma_t* h, const float* src, size_t n, int src_on_device);

/* External fields (Sec. 4): ext (2*cells floats: the potential of an A
 * particle in each cell, then of a B particle, kT per particle) is added to
 * omega at every field update, e.g. a linear attraction of one type to a
 * surface; forbidden (cells bytes, nonzero = no particle may enter the cell,
 * e.g. a confining wall) makes omega +inf there, so every move into such a
 * cell is rejected.  Either pointer may be NULL (that field is removed).
 * Forbidden cells take uniform moves only (SOMA_EINVAL otherwise: the smart
 * Monte Carlo and learned proposals use field gradients).  A particle already
 * inside a forbidden cell may leave it but none enters one.  Takes effect at
 * the next field update (soma_update_fields applies it at once); the
 * handle keeps its own copies.  Synchronises. */
soma_status soma_set_external(soma_t* h, const float* ext, const uint8_t* forbidden,
                              int src_on_device);

/* Mixture of linear architectures (Sec. 2.1: any mixture of molecular
 * architectures; here linear chains of N particles with any A/B sequence,
 * e.g. homopolymer blends or triblocks): seq holds n_arch (1..256) type
 * sequences, bit i of seq[a] set meaning particle i of architecture a is B,
 * and arch (n_chains bytes) the architecture of every chain.  Replaces the
 * diblock derived from desc.f for the sweep and the occupation count; call
 * soma_update_fields to recount at once.  N <= 64.  Uniform moves: even N
 * for the SET scheme (any N <= 64 with SOMA_ITERATION_MOLECULE).  Smart
 * Monte Carlo moves (any N <= 64): the mixture is set as linear
 * architectures through soma_set_topology (particle i of type bit i, bonded
 * to i - 1 and i + 1), whose sweep moves a linear chain as the linear path
 * does.  The learned proposal: SOMA_EINVAL.  seq = NULL
 * returns to the diblock.  Every arch entry is checked against n_arch
 * (SOMA_EINVAL).  The handle keeps its own copies.  Synchronises. */
soma_status soma_set_architectures(soma_t* h, const uint64_t* seq, uint32_t n_arch,
                                   const uint8_t* arch, int src_on_device);

/* Molecules of any architecture (Sec. 2.1: branched molecules, rings, any
 * mixture; Sec. 3.2.1: the architecture array; Sec. 3.1.2: independent sets).
 *   words (n_words uint32): one block per architecture, starting at
 *     start[a] (n_arch = 1..256 entries): word 0 = n, the architecture's
 *     particles, 1 <= n <= N (the system's N, <= 64): a molecule of n < N
 *     particles holds the first n of its N slots (molecules of several
 *     lengths in one system, Sec. 2.1); its other slots are absent -- never
 *     moved, counted or bonded, their positions kept as they are;
 *     word 1 + i = (index in words of particle i's first bond word << 8) |
 *     type (0 A, 1 B; 0..n_types-1 after soma_set_types), index 0xFFFFFF for
 *     a particle without bonds; a bond
 *     word = (signed 27-bit offset j - i of the partner j << 5) | (bond type
 *     << 1) | last, where bond type 0 (harmonic, the system's spring) is the
 *     only one and the list of a particle ends at the word with last = 1.
 *     Every bond is listed at both ends, once.
 *   mol_arch (n_chains bytes): the architecture of every molecule.
 * The independent sets are derived here: particles in index order take the
 * smallest set index that none of their earlier partners holds (at most 8
 * sets).  Each sweep a molecule visits its sets in a random order: two sets
 * as the linear chain (bit 0 of the acceptance word of particle 0's move
 * draw puts set 1 first), more by an inside-out Fisher-Yates shuffle whose
 * k-th step (k = 1..n-1) takes j = (h_k (k+1)) >> 16, h_k the k-th 16-bit half
 * (low half first) of the words of the Philox draw with counter (molecule lo,
 * molecule hi, sweep, 6 << 24 | replica_id); SOMA_SET_ORDER_FIXED visits them
 * in index order.  Replaces the diblock (and any mixture) for the sweep, the
 * occupation count and the bond observables (E_b and b2 over the listed
 * bonds; Re2 = |r_{n-1} - r_0|^2 with n the molecule's particles); rho_0 dL^3,
 * the attempted moves and the normalisation of S(q) count the molecules'
 * particles, while kappa_0 = kappaN/N and chi_0 = chiN/N keep the system's N
 * as the reference length; call soma_update_fields to recount at
 * once.  Uniform moves, in the SET scheme or the molecule-parallel iteration
 * (SOMA_ITERATION_MOLECULE: each molecule makes n attempts, on particles
 * ((word 3 & 0xFF) * n) >> 8 of its own n; partners from the same tables),
 * or smart Monte Carlo moves in the SET scheme (Sec. 2.2; the draws and the
 * acceptance of the linear chain's move, the bonded force -2 K_b sum_q (r -
 * r_q) over the listed partners q at the time the particle's set moves); the
 * learned proposal takes linear chains only (SOMA_EINVAL).
 * A shard (desc.n_chains_total > 0) takes only architectures of N particles
 * (SOMA_EINVAL otherwise: its density counts the whole system).
 * src_on_device: all three
 * arrays are device memory (else host).  SOMA_EINVAL, with the reason in
 * soma_last_error, for a block that does not fit the array, a type outside
 * 0/1 (0..n_types-1 with n_t types), a bond type other than 0, a partner
 * outside the molecule or listed
 * twice, a bond listed at one end only, more than 8 sets, or a mol_arch entry
 * >= n_arch.  words = NULL returns to the diblock.  The handle keeps its own
 * copies.  Synchronises. */
soma_status soma_set_topology(soma_t* h, const uint32_t* words, uint64_t n_words,
                              const uint32_t* start, uint32_t n_arch, const uint8_t* mol_arch,
                              int src_on_device);

/* n_t particle types (Sec. 2.1: Eq. hamil-comp, hamil-pair, omega-fields for
 * n_t types).  n_types = 2..8 with chiN[i*n_types + j] = chi_ij N (finite,
 * symmetric, zero diagonal); the option K^0 / K^1 is desc.hamiltonian:
 *   K^0: omega_i = kappa_0 (sum_k phi_k - 1) - sum_{k != i} chi_ik/(2N) (phi_i - phi_k)
 *   K^1: omega_i = kappa_0 (sum_k phi_k - 1) + sum_{k != i} chi_ik/N phi_k
 * and E_nb per cell kappaN/2 (sum phi - 1)^2 - sum_{i<j} chi_ij N/4 (phi_i -
 * phi_j)^2 (K^0) or + sum_{i<j} chi_ij N phi_i phi_j (K^1), every pair of
 * types counted once.  Particle types are the type bytes of the architecture
 * array (soma_set_topology, types < n_types), so the system runs the
 * architecture path (SET or molecule-parallel, uniform moves, or SET with
 * smart Monte Carlo moves whose field and field force come from the plane of
 * the particle's type; FP32 fields, no external fields); the occupation
 * numbers become one 32-bit plane per type.
 * soma_get_density, soma_get_fields and soma_structure_factor then refuse
 * (SOMA_EINVAL): use soma_get_type_counts / soma_get_type_fields /
 * soma_structure_factor_types.  Recomputes
 * counts and fields when architectures are set.  n_types = 0 returns to the
 * two types A, B (SOMA_ESTATE while the architectures use a type >= 2).
 * SOMA_EINVAL for a bad n_types or chiN or an incompatible description.
 * Synchronises. */
soma_status soma_set_types(soma_t* h, uint32_t n_types, const double* chiN);
/* Composition structure factor of types ti and tj (Sec. 5.6 for A, B):
 * S_ij(q) = |sum_c (n_ti(c) - n_tj(c)) exp(-i q.c)|^2 / M on grid wave vectors
 * q = 2 pi m / n (m: k x 3 int32, k <= 4096); with the two types A, B it is
 * soma_structure_factor.  SOMA_EINVAL for equal or out-of-range types;
 * SOMA_EOVERFLOW if a count exceeds 65535.  Synchronises. */
soma_status soma_structure_factor_types(soma_t* h, uint32_t ti, uint32_t tj, const int32_t* m,
                                        size_t k, double* out);
/* Occupation numbers per type, n[t*cells + c] (n = n_types*cells), and the
 * FP32 fields per type, w[t*cells + c], of the current state.  Synchronise. */
soma_status soma_get_type_counts(soma_t* h, uint32_t* dst, size_t n, int dst_on_device);
soma_status soma_get_type_fields(soma_t* h, float* dst, size_t n, int dst_on_device);

/* Relabels the molecules in the order soma_create gives its own chains: by
 * the Morton (Z-curve) code of the 8^3-cell block holding each molecule's
 * particle 0, ties by the previous label (the labels of molecules are
 * arbitrary, Sec. 3.1.1).  Positions and the architectures of
 * soma_set_architectures / soma_set_topology follow their molecules; the
 * occupation numbers and fields do not change.  Molecules that are neighbours
 * in space then share warps, so the field gathers and count atomics of a warp
 * hit nearby cells: call it after soma_set_positions with positions in an
 * arbitrary order.  perm (optional, host, n_chains entries) receives the
 * previous label of each new label.  SOMA_EINVAL for n_chains >= 2^32,
 * SOMA_ESTATE for a batch member.  Synchronises. */
soma_status soma_sort_molecules(soma_t* h, uint64_t* perm);

/* The check and the independent sets of soma_set_topology on their own, on
 * the host (no handle, no device): words / start / n_arch as there (host
 * memory), N the particle slots per molecule; writes the set of particle i of
 * architecture a to sets[a*N + i] (n_arch*N bytes; 0xFF for the absent slots
 * of an architecture of fewer than N particles) and the number of sets of
 * each architecture to n_sets (n_arch bytes).  Types 0..7 are accepted (the
 * sets do not depend on them; soma_set_topology checks them against the
 * system's types).  SOMA_EINVAL for an array soma_set_topology would refuse
 * otherwise, with the reason in soma_last_error. */
soma_status soma_topology_sets(const uint32_t* words, uint64_t n_words, const uint32_t* start,
                               uint32_t n_arch, uint32_t N, uint8_t* sets, uint8_t* n_sets);

/* FP64 observables of the current state (Eq. h-bond, Eq. discrete-ham).
 * Synchronises.  For a shard, E_b, Re2, b2 and the move counts cover its own
 * chains (sum E_b and the counts over the shards, weight Re2 and b2 by the
 * chains and bonds); E_nb, E_ext and max_cell are those of the current
 * occupation numbers, i.e. of the whole system after soma_shard_fields. */
soma_status soma_observables(soma_t* h, soma_obs* out);

/* Derived parameters of a system (Sec. 2.1), all in the units used by the
 * library (lengths in dL, energies in kT). */
typedef struct soma_params {
  double Re;          /* R_e0 in dL */
  double a;           /* maximal trial displacement per axis, dL */
  double K_b;         /* k0/2 = 3(N-1)/(2 R_e0^2), kT/dL^2 */
  double b0;          /* bond length R_e0/sqrt(N-1), dL */
  double rho_cell;    /* rho_0 dL^3 = M / cells, particles per cell */
  double sqrt_Nbar;   /* invariant degree of polymerisation: rho_0 R_e0^3 / N */
  double epsilon;     /* SCMF accuracy (b0/dL)^3 / sqrt(N Nbar) (quasi-instantaneous
                         field approximation; small is accurate, Sec. 2.2) */
  uint64_t M;         /* particles */
  uint32_t cells;     /* grid cells */
  uint32_t N_A;       /* A particles of a diblock */
} soma_params;
soma_status soma_get_parameters(soma_t* h, soma_params* out);

/* Diagnostic of the bounded device waits (the tcgen05 network evaluator waits
 * for its tensor-core products on an mbarrier with an iteration limit and
 * reports a wait that gives up as SOMA_ETIMEOUT instead of hanging): one warp
 * waits, at most limit polls, for an mbarrier phase that nothing completes.
 * Returns SOMA_ETIMEOUT (the expected outcome), after which the context stays
 * usable.  No counterpart in the paper.  Synchronises stream (NULL: legacy). */
soma_status soma_check_bounded_wait(uint32_t limit, void* stream);

/* Composition structure factor S(q) = |sum_c (n_A - n_B)(c) e^{-i q.c}|^2 / M
 * at q = 2 pi (m_x/grid_x, m_y/grid_y, m_z/grid_z) for k integer triples m
 * (host array, k x 3); FP64 on the device; out is a host array of k doubles.
 * The radial S(q,t) of Sec. 5.6 is the shell average of these values.
 * Synchronises.  k <= 4096. */
soma_status soma_structure_factor(soma_t* h, const int32_t* m, size_t k, double* out);

/* Sweep counter: the Philox counter word w of the next MC step.  Setting it
 * (with soma_set_positions) resumes a run bit-exactly: there is no RNG state. */
soma_status soma_get_sweep(soma_t* h, uint64_t* out);
soma_status soma_set_sweep(soma_t* h, uint64_t sweep);

/* Per-kernel device timing with CUDA events on the handle's stream (on != 0
 * enables; enabling resets the sums and the launch counts).  soma_get_timing
 * synchronises. */
soma_status soma_set_timing(soma_t* h, int on);
soma_status soma_get_timing(soma_t* h, soma_timing* out);

/* Block until all work queued by h has finished; reports sticky device errors. */
soma_status soma_sync(soma_t* h);

/* The cudaStream_t the handle runs on. */
void* soma_stream(soma_t* h);

/* Evaluate the device Philox4x32-10 on n counters: ctr (4n words), key (2n
 * words), out (4n words), all device pointers; asynchronous on stream.  Used
 * to check the generator against independent implementations. */
soma_status soma_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n,
                        void* stream);

/* What the smart Monte Carlo move (Sec. 2.2) makes of its Philox draw, for n
 * draws of four words each (words, 4n uint32) into out (4n floats): the three
 * standard normals of the Box-Muller transform of the uniforms (k + 1/2)/2^24
 * of the top 24 bits k of words (0, 1) and (2, 3) -- radius sqrt(-2 ln u1)
 * with ln u1 accurate to about an FP32 ulp, angle 2 pi u2 by the hardware
 * sincos -- and ln u of the acceptance uniform, k = the low bytes of words 0,
 * 1, 2 (word 0's lowest), by the hardware log.  The same device functions as
 * the sweeps.  Both pointers device memory; asynchronous on stream.
 * SOMA_EINVAL for a NULL pointer with n > 0.  Used to check the transforms
 * against independent implementations. */
soma_status soma_smc_draws(const uint32_t* words, float* out, size_t n, void* stream);

/* ------------------------------------------------------------------------
 * Learned proposal (desc.move = SOMA_MOVE_LEARNED; no counterpart in the
 * paper, whose force-biased proposal is the smart Monte Carlo move, Sec. 2.2).
 *
 * A multilayer perceptron 12 -> 32 -> 32 -> 4 (ReLU hidden units) maps the
 * features of a particle -- the bond vectors r - r_{i-1} and r_{i+1} - r (zero
 * without that partner), the gradient of omega_t at r (per axis, the face
 * differences of its cell interpolated linearly inside the cell), is_A,
 * has_prev, has_next -- to a drift mu and a log step scale s = 2 tanh(o3/2).
 * Trial move r' = r + mu + (a/sqrt 3) e^s xi, xi standard normal; accepted
 * with min(1, exp(-dE) q(r|r')/q(r'|r)), the reverse density evaluating the
 * network at r', so the move samples the same distribution for any weights.
 * Parameters (SOMA_MLP_PARAMS floats): W1[32][12], b1[32], W2[32][32], b2[32],
 * W3[4][32], b3[4].  The sweep uses a BF16 copy with FP32 arithmetic; the
 * FP32 master copy is trained.  A new handle starts with all weights zero
 * (a Gaussian random-walk proposal of the uniform move's variance).
 * ------------------------------------------------------------------------ */
#define SOMA_MLP_PARAMS 1604

/* Replace the parameters (FP32; host or device source); resets Adam. */
soma_status soma_proposal_set_weights(soma_t* h, const float* w, size_t n, int src_on_device);
/* Copy the FP32 master parameters out.  Synchronises. */
soma_status soma_proposal_get_weights(soma_t* h, float* w, size_t n, int dst_on_device);

/* Expected squared jump J = alpha |r' - r|^2 of n given samples and its
 * gradient with respect to the parameters (FP32), the training objective:
 * samples (device, n pairs chain, i), xi (device, 3n normals), w (device FP32
 * parameters, or NULL for the handle's), grad (device, SOMA_MLP_PARAMS,
 * overwritten with the sum over samples), J and log_alpha (device, n each,
 * optional).  The trial position is not rounded to FP32 here (a smooth
 * surrogate of the move).  Asynchronous. */
soma_status soma_proposal_grad(soma_t* h, const float* w, const uint32_t* samples, const float* xi,
                               uint32_t n, float* grad, float* J, float* log_alpha);

typedef struct soma_train_cfg {
  uint32_t steps;           /* gradient steps */
  uint32_t batch;           /* samples per step (particles of the current state) */
  uint32_t sweeps_between;  /* plain (uniform-move) cycles before each step */
  float lr, beta1, beta2, eps;  /* Adam */
} soma_train_cfg;

typedef struct soma_train_log {
  double mean_J_first;      /* mean objective of the first batch */
  double mean_J_last;       /* ... of the last batch */
  double mean_alpha_last;   /* mean acceptance probability of the last batch */
  uint32_t steps_done;
  uint32_t reserved;
} soma_train_log;

/* Train the proposal on configurations the plain method generates: per step,
 * sweeps_between uniform-move cycles of this system, then one Adam step on
 * -mean J over `batch` particles drawn with Philox (purpose 5).  The system's
 * state advances.  Synchronises. */
soma_status soma_proposal_train(soma_t* h, const soma_train_cfg* cfg, soma_train_log* log);

/* ------------------------------------------------------------------------
 * Batches: many independent systems advanced together, one sweep launch and
 * one field launch per cycle for the whole batch (no counterpart in the
 * paper, which runs one system per MPI rank; the launch shape is chosen by
 * an autotuner in the spirit of Sec. 3.2.2).
 *
 * Members are created as by soma_create and evolve bit-identically to the
 * same system run alone.  Requirements: even N <= 64, uniform moves, one seed
 * and one grid_dtype for all members (distinguish members by replica_id),
 * M < 2^32 per member, at most SOMA_BATCH_MAX members.  soma_batch_system
 * lends the member's handle for getters and observables; soma_sweep on a lent
 * handle returns SOMA_ESTATE.  All members run on the batch's stream (NULL:
 * the batch creates its own).
 * ------------------------------------------------------------------------ */
#define SOMA_BATCH_MAX 4096
typedef struct soma_batch_t soma_batch_t;

/* One launch shape of the batched sweep and its measured time. */
typedef struct soma_tune_entry {
  int32_t block;          /* threads per block */
  int32_t blocks_per_sm;  /* resident blocks per SM (persistent grid) */
  int32_t item_tiles;     /* 32-lane tiles per work item, taken by the blocks
                             in turn; 0 (the default): every block takes one
                             contiguous range of the members' concatenated
                             tiles, equal to within a tile */
  int32_t reserved;
  double ms_per_cycle;    /* sweep + field update, CUDA events */
} soma_tune_entry;

soma_status soma_batch_create(const soma_system_desc* descs, uint32_t n, void* stream,
                              soma_batch_t** out);
soma_status soma_batch_destroy(soma_batch_t* b);
/* n cycles of every member: n x (one sweep launch, one field launch). */
soma_status soma_batch_sweep(soma_batch_t* b, uint32_t n);
soma_status soma_batch_sync(soma_batch_t* b);
soma_status soma_batch_system(soma_batch_t* b, uint32_t i, soma_t** out);
/* Time every launch shape (block 128/256/512 threads that fit the kernel x
 * 1..8 resident blocks per SM that fit x work items of 16/64/256 tiles or the
 * equal contiguous range per block) over cycles_per_candidate real cycles
 * (the members advance), keep the fastest.  table (optional) receives up to
 * table_len entries; *n_written the number of shapes tried.  The paper tunes
 * its parallel regions the same way, by timing candidates (Sec. 3.2.2). */
soma_status soma_batch_autotune(soma_batch_t* b, uint32_t cycles_per_candidate,
                                soma_tune_entry* table, uint32_t table_len, uint32_t* n_written);
/* The work items of the batched sweep, computed on the host only (no CUDA
 * call): what soma_batch_* launches for members of member_tiles[k] warp tiles
 * (ceil(n_chains / floor(64 / N)) for member k) on a grid of `grid` blocks.
 * Block j takes items j, j + grid, j + 2 grid, ...
 *   item_tiles > 0: runs of at most item_tiles tiles of each member in turn
 *                   (grid unused);
 *   item_tiles = 0: block j's items cover tiles [T j / grid, T (j+1) / grid)
 *                   of the members' concatenation (T tiles in all), cut at
 *                   member boundaries; piece r of block j is item r * grid + j
 *                   and blocks with fewer pieces get empty items.
 * items:    host array of 3 * capacity words (member, first tile, end tile) or
 *           NULL to ask for the count only; *n_items receives the count.
 * SOMA_EINVAL for NULL member_tiles / n_items, n_members outside
 * 1..SOMA_BATCH_MAX, item_tiles < 0, grid outside 1..2^20 with item_tiles = 0,
 * or capacity below the count (nothing written). */
soma_status soma_batch_plan(const uint32_t* member_tiles, uint32_t n_members, uint32_t grid,
                            int32_t item_tiles, uint32_t* items, size_t capacity, size_t* n_items);
/* Use a given launch shape (e.g. one tuned earlier; ms_per_cycle ignored).
 * SOMA_EINVAL unless block is a multiple of 32 the kernel accepts,
 * blocks_per_sm of that block fit on one SM and item_tiles >= 0.  Results do
 * not depend on the shape: every member evolves as it would alone. */
soma_status soma_batch_set_shape(soma_batch_t* b, const soma_tune_entry* shape);
soma_status soma_batch_get_shape(soma_batch_t* b, soma_tune_entry* out);
soma_status soma_batch_set_timing(soma_batch_t* b, int on);
soma_status soma_batch_get_timing(soma_batch_t* b, soma_timing* out);

/* S(q) for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this is a library convenience.  It computes
 * exactly what soma_structure_factor computes, but allocates nothing after
 * its first call on a device (below): no cudaMalloc, no cudaFree, no host
 * heap, on success or failure.  It is meant for code that cannot allocate at
 * the moment it wants S(q), e.g. an analysis hook inside a host application
 * whose memory pool owns all free device memory, or code that must not
 * synchronise the device (cudaMalloc and cudaFree may).
 *
 * desc:     the system (validated like soma_create; desc->stream is ignored).
 * density:  device pointer to the packed occupation numbers of that system
 *           (cells words, n_A | n_B << 16, e.g. from soma_get_density).
 * m, k:     host array of k integer wave-vector triples, k <= SOMA_SQ_NOALLOC_MAX_K.
 * out:      host array of k doubles; returns after the results are there.
 * stream:   cudaStream_t to run on (NULL: legacy default stream).
 *
 * Scratch (twiddle tables and block partial sums, about 768 KB) lives in one
 * file-scope device array of libsoma.  The first call on each device sets it
 * up: it looks up the array's device address, and with CUDA's lazy module
 * loading (the default) that lookup is what loads this part of the library
 * onto the device and allocates the array there -- so make the first call
 * at a time when device memory can still be allocated (for instance right
 * after soma_create).  The address is kept for
 * the rest of the process: after a cudaDeviceReset of that device the kept
 * address is stale and this entry point must not be called on it again.  The
 * array stays allocated on every device that made a call until the process
 * exits.  Every call synchronises its stream before returning (the results
 * are copied to the host array out), so no call may be made on a stream that
 * is being captured into a graph.  All calls share the array: two calls
 * that overlap on the GPU (different streams, or different host threads
 * without ordering) race and may return wrong values.  Every call overwrites
 * all of the scratch it reads.
 * Returns SOMA_EINVAL when k exceeds SOMA_SQ_NOALLOC_MAX_K or grid_x + grid_y +
 * grid_z exceeds SOMA_SQ_NOALLOC_MAX_AXES, and SOMA_ECUDA on a CUDA error. */
#define SOMA_SQ_NOALLOC_MAX_K 32
#define SOMA_SQ_NOALLOC_MAX_AXES 1024
soma_status soma_structure_factor_noalloc(const soma_system_desc* desc, const uint32_t* density,
                                          const int32_t* m, size_t k, double* out, void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* soma_last_error(void);

/* SOMA_ABI_VERSION of the loaded library. */
int soma_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SOMA_H */
