/*
 * soma_oracle.h -- plain, slow, FP64 CPU oracle for the SCMF Monte-Carlo cycle
 * of Daoulas/Mueller-type soft coarse-grained polymer melts as implemented by
 * SOMA (arXiv:1711.03828).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py may load this library.  It
 * shares no code, header, constant table or helper with the CUDA library under
 * paper_1711_03828_gb300/csrc; neither includes the other.
 *
 * Conventions (where the paper leaves a choice open, the reading taken):
 *   - lengths in units of the grid spacing dL (cubic cells, Sec. 2.1), so the
 *     cell of a particle is floor(x) taken modulo the grid extent;
 *   - energies in kT; omega_t(c) is the per-particle field energy of Eq.
 *     (omega-fields), i.e. kappa_0 = kappaN/N and chi_0 = chiN/N;
 *   - linear diblock chains: monomer i of a chain is type A iff i < N_A;
 *   - positions are stored FP32 structure-of-arrays (x[M], y[M], z[M]),
 *     monomer m = chain*N + i, unwrapped (only the cell index is wrapped);
 *   - every arithmetic decision is taken in FP64 from the FP32 stored state.
 *
 * Parity pins: see tests/test_oracle_*.py.  Functions whose parity is not
 * pinned by anything outside the oracle say "parity unpinned" below.
 */
#ifndef SOMA_ORACLE_H
#define SOMA_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox stream purposes (the fourth counter word holds purpose<<24 | replica). */
enum { OR_PURPOSE_INIT = 0, OR_PURPOSE_MOVE = 1, OR_PURPOSE_MOVE2 = 2,
       OR_PURPOSE_ATTEMPT = 3, OR_PURPOSE_CONFIG = 4, OR_PURPOSE_TRAIN = 5,
       OR_PURPOSE_SETS = 6 };

typedef struct {
  uint64_t n_chains;
  uint32_t N;        /* particles per chain */
  uint32_t N_A;      /* floor(f*N + 1/2) */
  uint32_t grid[3];  /* collocation cells per axis */
  double   Re;       /* R_e0 in units of dL */
  double   kappaN, chiN;
  double   a;        /* maximal displacement per axis, units of dL (FP64) */
  float    a32;      /* the same, rounded to FP32: the move uses this value */
  double   K_b;      /* k0/2 = 3(N-1)/(2 Re^2), kT / dL^2 */
  double   rho_cell; /* rho_0 dL^3 = M / n_cells */
  uint64_t seed;
  uint32_t replica;
  int      set_order;  /* 0: random per (chain, sweep); 1: fixed even->odd;
                          2: molecule-parallel iteration (no sets, below) */
  int      move;       /* 0 uniform (Metropolis), 1 smart MC (force biased), 2 learned */
  const double* mlp;   /* learned proposal parameters (move 2), OR_MLP_PARAMS doubles */
  uint32_t* chosen;    /* optional: particle chosen by each attempt of the
                          molecule-parallel iteration (set_order 2), M entries */
  int hamiltonian;     /* 0: K^0_inter (default), 1: K^1_inter (Eq. hamil-pair) */
  const double* ext;   /* optional external field per type and cell (cells of A,
                          then cells of B), kT per particle, added to omega */
  const uint8_t* forbidden;  /* optional: nonzero cells no particle may enter */
  const uint64_t* seq; /* optional mixture of linear architectures (N <= 64): bit i of
                          seq[a] set means particle i of architecture a is type B */
  const uint8_t* arch; /* architecture of every chain (with seq or topo; n_chains entries) */
  /* optional molecular architectures in the array layout of Sec. 3.2.1 (below);
     arch[] then gives the architecture of every molecule and seq must be NULL */
  const uint32_t* topo;       /* the architecture array */
  const uint32_t* topo_start; /* index of the first word of each architecture's block */
  uint32_t n_topo;            /* architectures */
  const uint8_t* topo_set;    /* independent set of particle i of architecture a: [a*N + i] */
  const uint8_t* topo_nsets;  /* number of independent sets of each architecture */
  /* optional n_t particle types (Sec. 2.1, Eq. hamil-pair and omega-fields for
     n_t types): with topo, particle types are the architecture's type bytes
     0..n_types-1; chi_types[i*8 + j] = chi_ij N (symmetric, zero diagonal);
     the sweep then takes the field of type t from w_types[t] */
  uint32_t n_types;           /* 0: the two types A, B of wA / wB */
  double chi_types[64];
  const double* const* w_types;
  /* learned proposal in the tensor-core reading (mlp_bf16 = 1): features,
     weights, biases and the two hidden layers' activations rounded to BF16
     (nearest, ties to even) where the GPU's tensor-core evaluators round them,
     sums exact (FP64); mlp_slack (optional, M doubles) receives per move the
     smallest distance of a rounded value to a BF16 rounding boundary in units
     of the magnitude of the terms that formed it (or_bf16_slack) */
  int mlp_bf16;
  double* mlp_slack;
} or_system;

/* --- Molecular architectures (Sec. 3.2.1, Fig. polyarch) ---------------------
 * One block per architecture: word 0 = n, its number of particles (1 <= n <=
 * N: molecules of several lengths in one system; a molecule of n < N
 * particles occupies the first n of its N slots, the others are absent --
 * never moved, counted or bonded); word 1 + i = (offset << 8) | type of
 * particle i, where offset is the index in the whole array of the particle's
 * first bond word (OR_TOPO_NO_BONDS: no bonds) and type 0 = A, 1 = B; bond
 * words = (signed 27-bit partner offset j - i) << 5 | (bond type << 1) | last,
 * the list of a particle ending at the word whose last bit is 1.  Bond type 0
 * is the harmonic bond of the system (the only one).  Readings where the
 * figure is silent: "first bytes / bits" are the most significant ones, and
 * a particle without bonds carries the offset 0xFFFFFF. */
#define OR_TOPO_NO_BONDS 0xFFFFFFu
/* type (0 A, 1 B) of particle i of the block starting at start */
uint32_t or_topo_type(const uint32_t* topo, uint32_t start, uint32_t i);
/* bond partners of particle i in list order into out (cap entries at most);
 * returns their number */
uint32_t or_topo_partners(const uint32_t* topo, uint32_t start, uint32_t i, uint32_t* out,
                          uint32_t cap);
/* Independent sets of one architecture (Sec. 3.1.2, set generation by a simple
 * heuristic): particles in index order each take the smallest set index that
 * none of their already placed bond partners holds.  Writes set_of[0..N) and
 * returns the number of sets. */
uint32_t or_topology_sets(const uint32_t* topo, uint32_t start, uint8_t* set_of);
/* Order in which a molecule visits its n_sets sets in one sweep (Sec. 3.1.2:
 * a random permutation per molecule and sweep).  Two sets: the linear-chain
 * rule (bit 0 of the fourth word of the move draw of particle 0 puts set 1
 * first).  More sets (up to 8): an inside-out Fisher-Yates shuffle whose k-th
 * step (k = 1..n-1) takes j = (h_k (k+1)) >> 16, h_k the k-th 16-bit half
 * (low half first) of the words of the draw (OR_PURPOSE_SETS, molecule,
 * sweep).  set_order 1: sets in index order. */
void or_set_order(const or_system* s, uint64_t chain, uint32_t sweep, uint32_t n_sets,
                  uint32_t* order);

/* Particles of a molecule (its architecture's n, else N) and of the system. */
uint32_t or_length(const or_system* s, uint64_t chain);
double or_particles(const or_system* s);
/* Type of particle i of a chain: 1 for B, 0 for A (the diblock boundary N_A,
 * or the chain's architecture in a mixture). */
int or_is_B(const or_system* s, uint64_t chain, uint32_t i);
/* Type 0..n_t-1 of particle i of a chain (the architecture's type byte, else
 * or_is_B). */
uint32_t or_type(const or_system* s, uint64_t chain, uint32_t i);

typedef struct {
  uint64_t attempted, accepted;
  uint64_t near_ties;   /* moves with |dE + ln u| < 1e-4 */
} or_sweep_stats;

/* --- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Draw for (purpose, id, w) of a system: ctr = (id lo, id hi, w, purpose<<24|replica),
 * key = (seed lo, seed hi). */
void or_draw(const or_system* s, uint32_t purpose, uint64_t id, uint32_t w, uint32_t out[4]);
double or_uniform_sym(uint32_t r);   /* (2k+1)/2^24 - 1, k = r>>8, in (-1,1) */
double or_uniform_open(uint32_t r);  /* (k+1/2)/2^24,      k = r>>8, in (0,1)  */

/* --- System description ---------------------------------------------------- */
int or_system_init(or_system* s, uint64_t n_chains, uint32_t N, double f,
                   const double box_Re[3], const uint32_t grid[3],
                   double chiN, double kappaN, double a_Re, uint64_t seed,
                   uint32_t replica, int set_order, int move);

/* --- a0: initial configuration --------------------------------------------- */
void or_init_chains(const or_system* s, float* x, float* y, float* z);
void or_init_chain_range(const or_system* s, uint64_t c0, uint64_t c1,
                         float* x, float* y, float* z);

/* Spatial labelling of chains: chains are re-labelled in increasing order of
 * the Morton code of the coarse block (OR_SORT_BLOCK^3 cells) holding their
 * first particle, ties by the previous label.  The labels of molecules are
 * arbitrary (Sec. 3.1.1 distributes whole molecules freely at
 * initialisation); this only fixes which particle index, and so which random
 * stream, each chain uses.  perm (optional, n_chains) receives the old label
 * of each new label. */
#define OR_SORT_BLOCK 8
uint64_t or_chain_key(const or_system* s, float x0, float y0, float z0);
void or_sort_chains(const or_system* s, float* x, float* y, float* z, uint64_t* perm);

/* --- a3: occupation numbers, Eq. (density-characteristics) ----------------- */
void or_histogram(const or_system* s, const float* x, const float* y, const float* z,
                  uint32_t* nA, uint32_t* nB);

/* --- a4: interaction fields, Eq. (omega-fields) with K^0 -------------------- */
/* round_mode: 0 FP64 result, 1 rounded to FP32, 2 to BF16 (RNE), 3 to FP16 (RNE).
 * For 2/3 the value is first rounded to FP32 (the storage path of the GPU). */
void or_fields(const or_system* s, const uint32_t* nA, const uint32_t* nB,
               double* wA, double* wB, int round_mode);

/* --- n_t particle types (Sec. 2.1) ------------------------------------------
 * Occupation numbers per type, n[t*cells + c]; fields per type,
 * w[t*cells + c]:
 *   K^0: omega_i = kappa_0 (sum_k phi_k - 1) - sum_{k != i} chi_0ik/2 (phi_i - phi_k)
 *   K^1: omega_i = kappa_0 (sum_k phi_k - 1) + sum_{k != i} chi_0ik phi_k
 * (Eq. omega-fields), the derivatives of the energy per cell
 *   kappaN/2 (sum phi - 1)^2 - sum_{i<j} chi_ij N/4 (phi_i - phi_j)^2   (K^0)
 *   kappaN/2 (sum phi - 1)^2 + sum_{i<j} chi_ij N phi_i phi_j           (K^1)
 * counting every pair of types once (as for two types); or_energy_types
 * returns E_nb = rho_0 dL^3 / N times its sum over cells.  round_mode as for
 * or_fields (no external potential). */
void or_histogram_types(const or_system* s, const float* x, const float* y, const float* z,
                        uint32_t* n);
void or_fields_types(const or_system* s, const uint32_t* n, double* w, int round_mode);
double or_energy_types(const or_system* s, const uint32_t* n);

/* --- a2: one SET sweep with frozen fields (Sec. 3.1.2, Listing 2 scheme) --- */
/* margin (optional, M doubles): ln u - ln(acceptance ratio) of each attempted
 * move (dE + ln u for the uniform move); the move is accepted iff it is < 0.
 * accepted (optional, M bytes): 1 if the move was accepted.
 * chain range [c0, c1) lets tests run a sample of chains. */
void or_sweep(const or_system* s, float* x, float* y, float* z,
              const double* wA, const double* wB, uint32_t sweep,
              uint64_t c0, uint64_t c1,
              double* margin, uint8_t* accepted, or_sweep_stats* st);

/* The same, also recording the trial position of every attempted move in
 * trial (optional, 3*M floats, x|y|z planes). */
void or_sweep_trial(const or_system* s, float* x, float* y, float* z,
                    const double* wA, const double* wB, uint32_t sweep,
                    uint64_t c0, uint64_t c1,
                    double* margin, uint8_t* accepted, float* trial, or_sweep_stats* st);

/* --- a7/a8: learned Metropolis-Hastings proposal ----------------------------
 * A multilayer perceptron 12 -> 32 -> 32 -> 4 (ReLU hidden units) maps the
 * features of a particle to a drift mu (3) and a log step scale; the trial
 * move is r' = r + mu + sigma xi with sigma = sigma0 exp(2 tanh(o3/2)),
 * sigma0 = a/sqrt(3), xi standard normal (Box-Muller of the move draw, as for
 * the smart Monte Carlo move), accepted with min(1, exp(-dE) q(r|r')/q(r'|r))
 * where the reverse density evaluates the network at r'.  Features: the bond
 * vectors r - r_{i-1} and r_{i+1} - r (zero without that partner), the
 * gradient of omega_t at r (per axis, the face differences of the cell and its
 * neighbour interpolated linearly in the position inside the cell), is_A,
 * has_prev, has_next.  Parameters (1604, flat): W1[32][12], b1[32],
 * W2[32][32], b2[32], W3[4][32], b3[4].  There is no counterpart in the paper
 * (SMC is its force-biased proposal, Sec. 2.2).  Pins: the forward pass by
 * a closed form on hand-built weights, the features by a hand-placed chain in
 * a field with known face differences, the gradient by finite differences,
 * exactness of the move by brute force. */
#define OR_MLP_PARAMS 1604
void or_mlp_forward(const double* W, const double x[12], double out[4]);
void or_learned_features(const or_system* s, const float* x, const float* y, const float* z,
                         const double* w_t, uint64_t chain, uint32_t i, const double r[3],
                         double feat[12]);
void or_set_mlp(or_system* s, const double* W);
/* The network in the BF16 reading (see mlp_bf16): x rounded to BF16, weights
 * and biases rounded FP64 -> FP32 -> BF16, each hidden pre-activation summed
 * exactly, passed through the ReLU and rounded to BF16, outputs summed
 * exactly.  Tx (optional, 12): magnitude of the terms each input was formed
 * from (0: the input is reproduced exactly); *slack (optional) is lowered to
 * the smallest or_bf16_slack of the rounded inputs and activations. */
void or_mlp_forward_bf16(const double* W, const double x[12], const double* Tx,
                         double out[4], double* slack);
/* Distance of v from the nearest BF16 rounding boundary (the midpoint of two
 * adjacent BF16 values, applied to the FP32 value of v) divided by T: how far,
 * in units of T, v may move before its BF16 value changes.  +inf for v = 0,
 * T <= 0, or where the BF16 spacing at v is below 2^-16 T (a change of the
 * rounded value there is negligible). */
double or_bf16_slack(double v, double T);
/* Expected-squared-jump objective of one sample (chain, i) with normals xi:
 * J = alpha |r'-r|^2, alpha = min(1, exp(log_alpha)); returns J and adds dJ/dW
 * to grad (1604, optional).  Fields frozen, neighbours at their positions. */
double or_esjd_sample(const or_system* s, const double* W, const float* x, const float* y,
                      const float* z, const double* wA, const double* wB, uint64_t chain,
                      uint32_t i, const double xi[3], double* grad, double* log_alpha);

/* One full SCMF cycle: sweep all chains, then histogram, then fields. */
void or_cycle(const or_system* s, float* x, float* y, float* z,
              uint32_t* nA, uint32_t* nB, double* wA, double* wB,
              uint32_t sweep, int round_mode, or_sweep_stats* st);

/* --- a5: observables --------------------------------------------------------- */
typedef struct {
  double E_b;     /* sum over bonds of K_b |b|^2, Eq. (h-bond)+(V-harmonic) */
  double E_nb;    /* Eq. (discrete-ham) with K_fluc + K^0_inter (or K^1_inter) */
  double Re2;     /* mean |r_{N-1} - r_0|^2 over chains, dL^2 */
  double b2;      /* mean |r_{i+1} - r_i|^2 over bonds, dL^2 */
  double E_ext;   /* sum over cells and types of n_t(c) * ext_t(c) */
} or_obs;
void or_observables(const or_system* s, const float* x, const float* y, const float* z,
                    const uint32_t* nA, const uint32_t* nB, or_obs* out);

/* S(q) = |sum_c (nA-nB)(c) exp(-i q.c)|^2 / M with q = 2 pi m / grid, for
 * k wave-vector index triples m (k x 3 int32). */
void or_structure_factor(const or_system* s, const uint32_t* nA, const uint32_t* nB,
                         const int32_t* m, size_t k, double* out);

/* Threads the OpenMP parts use (1 when built without OpenMP). */
int or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
