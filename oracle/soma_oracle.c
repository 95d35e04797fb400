/*
 * soma_oracle.c -- FP64 CPU oracle of the SCMF Monte-Carlo cycle
 * (arXiv:1711.03828, Sec. 2 and Sec. 3.1.2).  Test infrastructure only: the
 * product path never loads it.  Every function follows the paper's steps in
 * the paper's order; nothing is blocked, fused or reordered.
 */
#include "soma_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, the counter-based generator of Salmon et al., "Parallel     */
/* random numbers: as easy as 1, 2, 3" (SC'11).  The paper's own generator is  */
/* a stored-state PCG (Sec. 3.2.3); a counter-based generator needs no stored  */
/* state at all, which is the property Sec. 3.2.3 argues for.                  */
/* One round: two 32x32->64 products of counter words 0 and 2 by the round     */
/* multipliers; the high halves are xored with the other two counter words and */
/* the round key; the low halves pass through; the key is bumped by the Weyl   */
/* constants between rounds.                                                    */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = M0 * (uint64_t)c0;
    uint64_t p1 = M1 * (uint64_t)c2;
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

void or_draw(const or_system* s, uint32_t purpose, uint64_t id, uint32_t w, uint32_t out[4]) {
  uint32_t ctr[4] = { (uint32_t)id, (uint32_t)(id >> 32), w,
                      (purpose << 24) | (s->replica & 0xFFFFFFu) };
  uint32_t key[2] = { (uint32_t)s->seed, (uint32_t)(s->seed >> 32) };
  or_philox4x32_10(ctr, key, out);
}

/* The 24 leading bits k of a word give the symmetric uniform (2k+1)/2^24 - 1
 * (never 0, exact in FP32) and the open uniform (k+1/2)/2^24 (never 0 or 1). */
double or_uniform_sym(uint32_t r) {
  double k = (double)(r >> 8);
  return (2.0 * k + 1.0) / 16777216.0 - 1.0;
}
double or_uniform_open(uint32_t r) {
  double k = (double)(r >> 8);
  return (k + 0.5) / 16777216.0;
}

/* ------------------------------------------------------------------------- */
/* System parameters.                                                          */
/*   R_e0 in dL units follows from the box: grid cells / box length in R_e0.   */
/*   k0/2 = 3/(2 b0^2) with b0^2 = R_e0^2/(N-1) (Sec. 2.1, b0 = sqrt(3/k0)).    */
/*   rho_0 dL^3 = particles per cell on average (Sec. 3.1.1).                   */
/* ------------------------------------------------------------------------- */
int or_system_init(or_system* s, uint64_t n_chains, uint32_t N, double f,
                   const double box_Re[3], const uint32_t grid[3],
                   double chiN, double kappaN, double a_Re, uint64_t seed,
                   uint32_t replica, int set_order, int move) {
  memset(s, 0, sizeof(*s));
  if (n_chains == 0 || N == 0) return -1;
  if (set_order == 2 && (move != 0 || N > 256)) return -1;  /* uniform moves, N <= 256 */
  s->n_chains = n_chains;
  s->N = N;
  s->N_A = (uint32_t)floor(f * (double)N + 0.5);
  if (s->N_A > N) s->N_A = N;
  for (int d = 0; d < 3; ++d) s->grid[d] = grid[d];
  s->Re = (double)grid[0] / box_Re[0];
  s->kappaN = kappaN;
  s->chiN = chiN;
  if (!(a_Re > 0.0)) a_Re = (N > 1) ? 0.5 / sqrt((double)(N - 1)) : 0.5;
  s->a = a_Re * s->Re;
  s->a32 = (float)s->a;
  s->K_b = (N > 1) ? 3.0 * (double)(N - 1) / (2.0 * s->Re * s->Re) : 0.0;
  double cells = (double)grid[0] * (double)grid[1] * (double)grid[2];
  s->rho_cell = (double)n_chains * (double)N / cells;
  s->seed = seed;
  s->replica = replica;
  s->set_order = set_order;
  s->move = move;
  return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* a0: first particle uniform in the box, then Gaussian bond vectors with      */
/* per-component variance R_e0^2 / (3 (N-1)), i.e. <b^2> = b0^2 (Sec. 2.1).    */
/* Gaussians by the Box-Muller transform of pairs of open uniforms.            */
/* ------------------------------------------------------------------------- */
static double or_init_gauss(const or_system* s, uint64_t chain, uint32_t j) {
  uint32_t w[4];
  or_draw(s, OR_PURPOSE_INIT, chain, 1u + j / 4u, w);
  uint32_t p = (j % 4u) / 2u;
  double u1 = or_uniform_open(w[2 * p]);
  double u2 = or_uniform_open(w[2 * p + 1]);
  double rad = sqrt(-2.0 * log(u1));
  double th = 2.0 * M_PI * u2;
  return (j % 2u == 0u) ? rad * cos(th) : rad * sin(th);
}

void or_init_chain_range(const or_system* s, uint64_t c0, uint64_t c1,
                         float* x, float* y, float* z) {
  const uint32_t N = s->N;
  const double sigma = (N > 1) ? s->Re / sqrt(3.0 * (double)(N - 1)) : 0.0;
  long long i0 = (long long)c0, i1 = (long long)c1;
#pragma omp parallel for schedule(static)
  for (long long cc = i0; cc < i1; ++cc) {
    uint64_t chain = (uint64_t)cc;
    uint32_t w[4];
    or_draw(s, OR_PURPOSE_INIT, chain, 0u, w);
    double r[3];
    for (int d = 0; d < 3; ++d) r[d] = or_uniform_open(w[d]) * (double)s->grid[d];
    uint64_t m = chain * N;
    x[m] = (float)r[0]; y[m] = (float)r[1]; z[m] = (float)r[2];
    for (uint32_t i = 0; i + 1 < N; ++i) {
      for (int d = 0; d < 3; ++d) r[d] += sigma * or_init_gauss(s, chain, 3u * i + (uint32_t)d);
      x[m + i + 1] = (float)r[0]; y[m + i + 1] = (float)r[1]; z[m + i + 1] = (float)r[2];
    }
  }
}

void or_init_chains(const or_system* s, float* x, float* y, float* z) {
  or_init_chain_range(s, 0, s->n_chains, x, y, z);
}

/* ------------------------------------------------------------------------- */
/* Cell of a position: the characteristic function Pi_c of Eq.                 */
/* (density-characteristics) with half-open cells [c, c+1) in dL units and     */
/* periodic images folded back into the box.                                    */
/* ------------------------------------------------------------------------- */
static uint64_t or_cell(const or_system* s, double x, double y, double z) {
  long long c[3];
  double p[3] = { x, y, z };
  for (int d = 0; d < 3; ++d) {
    long long n = (long long)s->grid[d];
    long long f = (long long)floor(p[d]);
    long long r = f % n;
    if (r < 0) r += n;
    c[d] = r;
  }
  return ((uint64_t)c[2] * s->grid[1] + (uint64_t)c[1]) * s->grid[0] + (uint64_t)c[0];
}

/* Morton code of the coarse block holding a position: the bits of the block
 * coordinates bx, by, bz (10 each) interleaved as ...z1y1x1z0y0x0. */
uint64_t or_chain_key(const or_system* s, float x0, float y0, float z0) {
  double p[3] = { x0, y0, z0 };
  uint64_t b[3];
  for (int d = 0; d < 3; ++d) {
    long long n = (long long)s->grid[d];
    long long c = (long long)floor(p[d]) % n;
    if (c < 0) c += n;
    b[d] = (uint64_t)(c / OR_SORT_BLOCK);
  }
  uint64_t key = 0;
  for (int bit = 0; bit < 10; ++bit)
    for (int d = 0; d < 3; ++d) key |= ((b[d] >> bit) & 1u) << (3 * bit + d);
  return key;
}

static int or_cmp_u64(const void* a, const void* b) {
  uint64_t u = *(const uint64_t*)a, v = *(const uint64_t*)b;
  return (u > v) - (u < v);
}

void or_sort_chains(const or_system* s, float* x, float* y, float* z, uint64_t* perm) {
  const uint64_t n = s->n_chains, N = s->N;
  uint64_t* kv = (uint64_t*)malloc(n * sizeof(uint64_t));
  float* tmp = (float*)malloc(n * N * sizeof(float));
  for (uint64_t k = 0; k < n; ++k)
    kv[k] = (or_chain_key(s, x[k * N], y[k * N], z[k * N]) << 32) | k;
  qsort(kv, n, sizeof(uint64_t), or_cmp_u64);
  float* axes[3] = { x, y, z };
  for (int d = 0; d < 3; ++d) {
    for (uint64_t j = 0; j < n; ++j) {
      uint64_t old = kv[j] & 0xFFFFFFFFu;
      memcpy(tmp + j * N, axes[d] + old * N, N * sizeof(float));
    }
    memcpy(axes[d], tmp, n * N * sizeof(float));
  }
  if (perm)
    for (uint64_t j = 0; j < n; ++j) perm[j] = kv[j] & 0xFFFFFFFFu;
  free(kv);
  free(tmp);
}

int or_is_B(const or_system* s, uint64_t chain, uint32_t i) {
  if (s->topo && s->arch) return or_topo_type(s->topo, s->topo_start[s->arch[chain]], i) == 1u;
  if (s->seq && s->arch) return (int)((s->seq[s->arch[chain]] >> i) & 1u);
  return i >= s->N_A;
}

/* Particles of a molecule: its architecture's count (the first word of the
 * block, at most N; the slots from there to N-1 are absent), else N. */
uint32_t or_length(const or_system* s, uint64_t chain) {
  if (s->topo && s->arch) return s->topo[s->topo_start[s->arch[chain]]];
  return s->N;
}

/* Particles of the system: the molecules' counts summed. */
double or_particles(const or_system* s) {
  if (!(s->topo && s->arch)) return (double)s->n_chains * (double)s->N;
  double n = 0.0;
  for (uint64_t k = 0; k < s->n_chains; ++k) n += (double)or_length(s, k);
  return n;
}

uint32_t or_type(const or_system* s, uint64_t chain, uint32_t i) {
  if (s->topo && s->arch) return or_topo_type(s->topo, s->topo_start[s->arch[chain]], i);
  return (uint32_t)or_is_B(s, chain, i);
}

/* ------------------------------------------------------------------------- */
/* Molecular architectures in the array layout of Sec. 3.2.1.                  */
/* ------------------------------------------------------------------------- */
uint32_t or_topo_type(const uint32_t* topo, uint32_t start, uint32_t i) {
  return topo[start + 1u + i] & 0xFFu;
}

uint32_t or_topo_partners(const uint32_t* topo, uint32_t start, uint32_t i, uint32_t* out,
                          uint32_t cap) {
  const uint32_t first = topo[start + 1u + i] >> 8;
  if (first == OR_TOPO_NO_BONDS) return 0u;
  uint32_t k = 0;
  for (uint32_t b = first;; ++b) {
    const uint32_t w = topo[b];
    /* the top 27 bits are the signed offset to the partner */
    const int32_t off = (int32_t)w >> 5;
    if (k < cap) out[k] = (uint32_t)((int64_t)i + off);
    ++k;
    if (w & 1u) break;
  }
  return k < cap ? k : cap;
}

uint32_t or_topology_sets(const uint32_t* topo, uint32_t start, uint8_t* set_of) {
  const uint32_t N = topo[start];
  uint32_t partners[256];
  uint32_t n_sets = 0;
  for (uint32_t i = 0; i < N; ++i) {
    const uint32_t k = or_topo_partners(topo, start, i, partners, 256u);
    uint32_t taken = 0;   /* bit c: a partner already placed holds set c */
    for (uint32_t b = 0; b < k; ++b)
      if (partners[b] < i) taken |= 1u << set_of[partners[b]];
    uint32_t c = 0;
    while (taken & (1u << c)) ++c;
    set_of[i] = (uint8_t)c;
    if (c + 1u > n_sets) n_sets = c + 1u;
  }
  return n_sets;
}

void or_set_order(const or_system* s, uint64_t chain, uint32_t sweep, uint32_t n_sets,
                  uint32_t* order) {
  for (uint32_t k = 0; k < n_sets; ++k) order[k] = k;
  if (s->set_order != 0 || n_sets < 2) return;
  uint32_t w[4];
  if (n_sets == 2) {
    or_draw(s, OR_PURPOSE_MOVE, chain * s->N, sweep, w);
    const uint32_t first = w[3] & 1u;
    order[0] = first;
    order[1] = 1u - first;
    return;
  }
  or_draw(s, OR_PURPOSE_SETS, chain, sweep, w);
  order[0] = 0;
  for (uint32_t k = 1; k < n_sets; ++k) {
    const uint32_t h = (w[(k - 1u) / 2u] >> (16u * ((k - 1u) % 2u))) & 0xFFFFu;
    const uint32_t j = (h * (k + 1u)) >> 16;
    order[k] = order[j];
    order[j] = k;
  }
}

/* Bond partners of particle i of a chain: the linear neighbours i-1, i+1, or
 * the bond list of the molecule's architecture. */
static uint32_t or_partners(const or_system* s, uint64_t chain, uint32_t i, uint32_t* out) {
  if (s->topo && s->arch)
    return or_topo_partners(s->topo, s->topo_start[s->arch[chain]], i, out, 256u);
  uint32_t k = 0;
  if (i > 0) out[k++] = i - 1u;
  if (i + 1u < s->N) out[k++] = i + 1u;
  return k;
}

/* a3: n_i(c) = number of particles of type i in cell c (Eq.                    */
/* density-characteristics times rho_0 dL^3; Sec. 3.1.1 occupation numbers).    */
void or_histogram(const or_system* s, const float* x, const float* y, const float* z,
                  uint32_t* nA, uint32_t* nB) {
  const uint64_t cells = (uint64_t)s->grid[0] * s->grid[1] * s->grid[2];
  memset(nA, 0, cells * sizeof(uint32_t));
  memset(nB, 0, cells * sizeof(uint32_t));
  for (uint64_t k = 0; k < s->n_chains; ++k) {
    const uint32_t n_k = or_length(s, k);
    for (uint32_t i = 0; i < n_k; ++i) {
      uint64_t m = k * s->N + i;
      uint64_t c = or_cell(s, x[m], y[m], z[m]);
      if (!or_is_B(s, k, i)) nA[c] += 1u; else nB[c] += 1u;
    }
  }
}

/* Round-to-nearest-even of an FP32 value to BF16 / FP16, returned as double. */
static double or_round_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  u &= 0xFFFF0000u;
  float g;
  memcpy(&g, &u, 4);
  return (double)g;
}
static double or_round_fp16(float f) {
  _Float16 h = (_Float16)f;
  return (double)(float)h;
}

/* a4: omega_i(c) = kappa_0 (sum_k phi_k(c) - 1) - sum_{k != i} chi_0/2 (phi_i - phi_k)  */
/* (option K^0) or kappa_0 (sum_k phi_k(c) - 1) + sum_{k != i} chi_0 phi_k (option K^1), */
/* with phi_k = n_k / (rho_0 dL^3), kappa_0 = kappaN/N, chi_0 = chiN/N            */
/* (Eq. omega-fields; two types A, B).  The external fields of Sec. 4 are added:   */
/* a per-type, per-cell potential, and cells no particle may enter (omega = +inf, */
/* so that every move into them is rejected).                                      */
void or_fields(const or_system* s, const uint32_t* nA, const uint32_t* nB,
               double* wA, double* wB, int round_mode) {
  const uint64_t cells = (uint64_t)s->grid[0] * s->grid[1] * s->grid[2];
  const double kappa0 = s->kappaN / (double)s->N;
  const double chi0 = s->chiN / (double)s->N;
  for (uint64_t c = 0; c < cells; ++c) {
    double phiA = (double)nA[c] / s->rho_cell;
    double phiB = (double)nB[c] / s->rho_cell;
    double comp = kappa0 * (phiA + phiB - 1.0);
    double a, b;
    if (s->hamiltonian == 1) {       /* K^1: + sum_{k != i} chi0 phi_k */
      a = comp + chi0 * phiB;
      b = comp + chi0 * phiA;
    } else {                         /* K^0: - sum_{k != i} chi0/2 (phi_i - phi_k) */
      a = comp - 0.5 * chi0 * (phiA - phiB);
      b = comp - 0.5 * chi0 * (phiB - phiA);
    }
    if (s->ext) { a += s->ext[c]; b += s->ext[cells + c]; }
    if (s->forbidden && s->forbidden[c]) { a = INFINITY; b = INFINITY; }
    if (round_mode == 1) { a = (double)(float)a; b = (double)(float)b; }
    else if (round_mode == 2) { a = or_round_bf16((float)a); b = or_round_bf16((float)b); }
    else if (round_mode == 3) { a = or_round_fp16((float)a); b = or_round_fp16((float)b); }
    wA[c] = a;
    wB[c] = b;
  }
}

/* n_t particle types: occupation numbers and fields per type (Sec. 2.1, Eq.    */
/* density-characteristics, hamil-comp, hamil-pair and omega-fields).          */
void or_histogram_types(const or_system* s, const float* x, const float* y, const float* z,
                        uint32_t* n) {
  const uint64_t cells = (uint64_t)s->grid[0] * s->grid[1] * s->grid[2];
  memset(n, 0, (size_t)s->n_types * cells * sizeof(uint32_t));
  for (uint64_t k = 0; k < s->n_chains; ++k)
    for (uint32_t i = 0; i < or_length(s, k); ++i) {
      const uint64_t m = k * s->N + i;
      n[(uint64_t)or_type(s, k, i) * cells + or_cell(s, x[m], y[m], z[m])] += 1u;
    }
}

void or_fields_types(const or_system* s, const uint32_t* n, double* w, int round_mode) {
  const uint64_t cells = (uint64_t)s->grid[0] * s->grid[1] * s->grid[2];
  const uint32_t T = s->n_types;
  const double kappa0 = s->kappaN / (double)s->N;
  for (uint64_t c = 0; c < cells; ++c) {
    double phi[8], total = 0.0;
    for (uint32_t t = 0; t < T; ++t) {
      phi[t] = (double)n[t * cells + c] / s->rho_cell;
      total += phi[t];
    }
    const double comp = kappa0 * (total - 1.0);
    for (uint32_t i = 0; i < T; ++i) {
      double v = comp;
      for (uint32_t k = 0; k < T; ++k) {
        if (k == i) continue;
        const double chi0 = s->chi_types[i * 8 + k] / (double)s->N;
        if (s->hamiltonian == 1) v = v + chi0 * phi[k];
        else v = v - 0.5 * chi0 * (phi[i] - phi[k]);
      }
      if (round_mode == 1) v = (double)(float)v;
      else if (round_mode == 2) v = or_round_bf16((float)v);
      else if (round_mode == 3) v = or_round_fp16((float)v);
      w[i * cells + c] = v;
    }
  }
}

double or_energy_types(const or_system* s, const uint32_t* n) {
  const uint64_t cells = (uint64_t)s->grid[0] * s->grid[1] * s->grid[2];
  const uint32_t T = s->n_types;
  double K = 0.0;
  for (uint64_t c = 0; c < cells; ++c) {
    double phi[8], total = 0.0;
    for (uint32_t t = 0; t < T; ++t) {
      phi[t] = (double)n[t * cells + c] / s->rho_cell;
      total += phi[t];
    }
    const double fl = total - 1.0;
    double k = 0.5 * s->kappaN * fl * fl;
    for (uint32_t i = 0; i < T; ++i)
      for (uint32_t j = i + 1; j < T; ++j) {
        const double chi = s->chi_types[i * 8 + j];
        if (s->hamiltonian == 1) k += chi * phi[i] * phi[j];
        else k -= 0.25 * chi * (phi[i] - phi[j]) * (phi[i] - phi[j]);
      }
    K += k;
  }
  return s->rho_cell / (double)s->N * K;
}

/* ------------------------------------------------------------------------- */
/* a2: one Monte-Carlo step with the fields frozen (second stage of the SCMF    */
/* cycle, Sec. 2.2), iterating each molecule's independent sets in a random     */
/* order (the SET scheme of Sec. 3.1.2): for a linear chain the even particles  */
/* form set 0 and the odd ones set 1.                                           */
/* Move of particle j (Sec. 2.2): trial displacement uniform in [-a, a] per     */
/* axis; dE = bonded change (Eq. V-harmonic summed over the bonds of j) + the   */
/* field change omega_t(c') - omega_t(c) (Eq. delta-e); Metropolis acceptance    */
/* min(1, exp(-dE)), taken as: accept iff dE <= 0 or ln u < -dE.                 */
/* ------------------------------------------------------------------------- */
/* Uniform move of particle i of chain with the draw w (words 0-2: the
 * displacement, word 3: the acceptance uniform).  Diagnostics are stored at
 * index rec (the particle for the SET sweep, the attempt for the molecule-
 * parallel sweep). */
static void or_move_uniform_w(const or_system* s, float* x, float* y, float* z,
                              const double* wA, const double* wB, uint64_t chain, uint32_t i,
                              const uint32_t w[4], uint64_t rec, double* margin, uint8_t* accepted,
                              float* trial, uint64_t* acc, uint64_t* ties) {
  const uint32_t N = s->N;
  const uint64_t m = chain * N + i;
  /* trial position: r + a*v rounded once to FP32 (the stored precision of
   * positions); fmaf rounds the exact value of the fused multiply-add */
  double r_old[3] = { x[m], y[m], z[m] };
  double r_new[3];
  const float pos[3] = { x[m], y[m], z[m] };
  for (int d = 0; d < 3; ++d)
    r_new[d] = (double)fmaf(s->a32, (float)or_uniform_sym(w[d]), pos[d]);
  double u = or_uniform_open(w[3]);
  if (trial) {
    const uint64_t M = s->n_chains * N;
    for (int d = 0; d < 3; ++d) trial[d * M + rec] = (float)r_new[d];
  }
  /* bonded energy change over the bond partners (i-1 and i+1 of a linear
   * chain, in that order) */
  uint32_t partners[256];
  const uint32_t n_partners = or_partners(s, chain, i, partners);
  double dEb = 0.0;
  for (uint32_t b = 0; b < n_partners; ++b) {
    uint64_t n = chain * N + partners[b];
    double rn[3] = { x[n], y[n], z[n] };
    double d_new = 0.0, d_old = 0.0;
    for (int d = 0; d < 3; ++d) {
      d_new += (r_new[d] - rn[d]) * (r_new[d] - rn[d]);
      d_old += (r_old[d] - rn[d]) * (r_old[d] - rn[d]);
    }
    dEb += s->K_b * (d_new - d_old);
  }
  /* field energy change, Eq. (delta-e) */
  const double* w_t = or_is_B(s, chain, i) ? wB : wA;
  if (s->n_types && s->w_types) w_t = s->w_types[or_type(s, chain, i)];
  uint64_t c_old = or_cell(s, r_old[0], r_old[1], r_old[2]);
  uint64_t c_new = or_cell(s, r_new[0], r_new[1], r_new[2]);
  double dE = dEb + (w_t[c_new] - w_t[c_old]);
  double lnu = log(u);
  int acc_move = (dE <= 0.0) || (lnu < -dE);
  if (margin) margin[rec] = dE + lnu;
  if (fabs(dE + lnu) < 1e-4) (*ties)++;
  if (acc_move) {
    x[m] = (float)r_new[0]; y[m] = (float)r_new[1]; z[m] = (float)r_new[2];
    (*acc)++;
  }
  if (accepted) accepted[rec] = (uint8_t)acc_move;
}

static void or_move_uniform(const or_system* s, float* x, float* y, float* z,
                            const double* wA, const double* wB, uint32_t sweep,
                            uint64_t chain, uint32_t i, double* margin, uint8_t* accepted,
                            float* trial, uint64_t* acc, uint64_t* ties) {
  const uint64_t m = chain * s->N + i;
  uint32_t w[4];
  or_draw(s, OR_PURPOSE_MOVE, m, sweep, w);
  or_move_uniform_w(s, x, y, z, wA, wB, chain, i, w, m, margin, accepted, trial, acc, ties);
}

/* Molecule-parallel iteration (Sec. 3.1.2, the first scheme): the chain's N
 * attempts of one MC step are made one after another, each on a particle of
 * the chain chosen at random, so each particle is attempted once per step on
 * average.  Attempt j of chain k draws Philox purpose 3 with id k*N + j: the
 * particle is ((word 3 & 0xFF) * n) >> 8, n the molecule's particles (the low byte, which the acceptance
 * uniform of the top 24 bits does not use; a state-independent choice, so
 * balance holds for any choice probabilities), the move is the uniform move
 * with that draw.  Diagnostics (margin, accepted, trial) are per attempt. */
static void or_move_attempt(const or_system* s, float* x, float* y, float* z,
                            const double* wA, const double* wB, uint32_t sweep,
                            uint64_t chain, uint32_t j, double* margin, uint8_t* accepted,
                            float* trial, uint32_t* chosen, uint64_t* acc, uint64_t* ties) {
  const uint64_t a = chain * s->N + j;
  uint32_t w[4];
  or_draw(s, OR_PURPOSE_ATTEMPT, a, sweep, w);
  const uint32_t i = (uint32_t)(((uint64_t)(w[3] & 0xFFu) * or_length(s, chain)) >> 8);
  if (chosen) chosen[a] = i;
  or_move_uniform_w(s, x, y, z, wA, wB, chain, i, w, a, margin, accepted, trial, acc, ties);
}

/* ------------------------------------------------------------------------- */
/* Smart Monte Carlo (force-biased) move of Sec. 2.2 (Rossky, Doll, Friedman;  */
/* Pangali, Rao, Berne): trial displacement dr = A F(r) + sqrt(2A) xi with xi a */
/* vector of standard normals and F the force on the particle: the bonded      */
/* force -2 k0/2 sum_n (r - r_n) over its bond partners n (of any architecture) */
/* plus minus the field gradient of its type, taken by                          */
/* central differences of omega_t over the neighbouring cells.  Accepted with   */
/* min(1, exp(-dE) T(r'->r)/T(r->r')), T(r->r') = exp(-|r'-r-A F(r)|^2/(4A)),   */
/* which keeps the move exact for any force.  A = a^2/6, so that the per-axis    */
/* variance 2A equals that of the uniform move, a^2/3.                          */
/* Random numbers: one draw per move (purpose 1).  The normals come from the   */
/* Box-Muller transform of the uniforms of the top 24 bits of words (0,1) and  */
/* (2,3); the acceptance uniform from the 24 bits left over, the low bytes of   */
/* words 0, 1, 2 (word 0's lowest).                                              */
/* ------------------------------------------------------------------------- */
static uint64_t or_cell_shift(const or_system* s, uint64_t c, int axis, int step) {
  long long n[3] = { s->grid[0], s->grid[1], s->grid[2] };
  long long k[3] = { (long long)(c % s->grid[0]), (long long)((c / s->grid[0]) % s->grid[1]),
                     (long long)(c / ((uint64_t)s->grid[0] * s->grid[1])) };
  k[axis] = ((k[axis] + step) % n[axis] + n[axis]) % n[axis];
  return ((uint64_t)k[2] * s->grid[1] + (uint64_t)k[1]) * s->grid[0] + (uint64_t)k[0];
}

/* Force on particle i of chain at r: the harmonic bonds to its partners (the
 * linear neighbours i-1, i+1, or the bond list of the molecule's
 * architecture, Sec. 3.2.1) and the field force of its type's plane. */
static void or_force(const or_system* s, const float* x, const float* y, const float* z,
                     const double* w_t, uint64_t chain, uint32_t i, const double r[3],
                     double F[3]) {
  for (int d = 0; d < 3; ++d) F[d] = 0.0;
  uint32_t fpart[256];
  const uint32_t n_fpart = or_partners(s, chain, i, fpart);
  for (uint32_t b = 0; b < n_fpart; ++b) {
    uint64_t n = chain * s->N + fpart[b];
    double rn[3] = { x[n], y[n], z[n] };
    for (int d = 0; d < 3; ++d) F[d] -= 2.0 * s->K_b * (r[d] - rn[d]);
  }
  uint64_t c = or_cell(s, r[0], r[1], r[2]);
  for (int d = 0; d < 3; ++d)
    F[d] -= 0.5 * (w_t[or_cell_shift(s, c, d, +1)] - w_t[or_cell_shift(s, c, d, -1)]);
}

static void or_move_smc(const or_system* s, float* x, float* y, float* z,
                        const double* wA, const double* wB, uint32_t sweep,
                        uint64_t chain, uint32_t i, double* margin, uint8_t* accepted,
                        float* trial, uint64_t* acc, uint64_t* ties) {
  const uint32_t N = s->N;
  const uint64_t m = chain * N + i;
  /* the field plane of the particle's type (A / B, or one of n_t types) */
  const double* w_t = (s->n_types && s->w_types) ? s->w_types[or_type(s, chain, i)]
                                                  : (or_is_B(s, chain, i) ? wB : wA);
  uint32_t w1[4];
  or_draw(s, OR_PURPOSE_MOVE, m, sweep, w1);
  /* the acceptance uniform's 24 bits, as the top 24 bits of a word */
  const uint32_t w_acc = ((w1[0] & 0xFFu) | (w1[1] & 0xFFu) << 8 | (w1[2] & 0xFFu) << 16) << 8;
  double xi[4];
  for (int p = 0; p < 2; ++p) {
    double u1 = or_uniform_open(w1[2 * p]), u2 = or_uniform_open(w1[2 * p + 1]);
    double rad = sqrt(-2.0 * log(u1)), th = 2.0 * M_PI * u2;
    xi[2 * p] = rad * cos(th);
    xi[2 * p + 1] = rad * sin(th);
  }
  const double A = s->a * s->a / 6.0;
  double r_old[3] = { x[m], y[m], z[m] };
  double F_old[3], F_new[3], r_new[3];
  or_force(s, x, y, z, w_t, chain, i, r_old, F_old);
  for (int d = 0; d < 3; ++d) {
    float dx = (float)(A * F_old[d] + sqrt(2.0 * A) * xi[d]);
    r_new[d] = (double)(float)(r_old[d] + (double)dx);
  }
  if (trial) {
    const uint64_t M = s->n_chains * N;
    for (int d = 0; d < 3; ++d) trial[d * M + m] = (float)r_new[d];
  }
  or_force(s, x, y, z, w_t, chain, i, r_new, F_new);
  /* bonded energy change over the partners, as in the uniform move */
  uint32_t epart[256];
  const uint32_t n_epart = or_partners(s, chain, i, epart);
  double dEb = 0.0;
  for (uint32_t b = 0; b < n_epart; ++b) {
    uint64_t n = chain * N + epart[b];
    double rn[3] = { x[n], y[n], z[n] };
    for (int d = 0; d < 3; ++d)
      dEb += s->K_b * ((r_new[d] - rn[d]) * (r_new[d] - rn[d]) - (r_old[d] - rn[d]) * (r_old[d] - rn[d]));
  }
  double dE = dEb + (w_t[or_cell(s, r_new[0], r_new[1], r_new[2])] -
                     w_t[or_cell(s, r_old[0], r_old[1], r_old[2])]);
  double fwd = 0.0, rev = 0.0;
  for (int d = 0; d < 3; ++d) {
    double f = r_new[d] - r_old[d] - A * F_old[d];
    double b = r_old[d] - r_new[d] - A * F_new[d];
    fwd += f * f;
    rev += b * b;
  }
  const double log_alpha = -dE - rev / (4.0 * A) + fwd / (4.0 * A);
  const double lnu = log(or_uniform_open(w_acc));
  const int acc_move = (log_alpha >= 0.0) || (lnu < log_alpha);
  if (margin) margin[m] = lnu - log_alpha;
  if (fabs(lnu - log_alpha) < 1e-4) (*ties)++;
  if (acc_move) {
    x[m] = (float)r_new[0]; y[m] = (float)r_new[1]; z[m] = (float)r_new[2];
    (*acc)++;
  }
  if (accepted) accepted[m] = (uint8_t)acc_move;
}

/* ------------------------------------------------------------------------- */
/* Learned proposal (move 2).                                                   */
/* ------------------------------------------------------------------------- */
enum { L_W1 = 0, L_B1 = 384, L_W2 = 416, L_B2 = 1440, L_W3 = 1472, L_B3 = 1600 };

void or_set_mlp(or_system* s, const double* W) { s->mlp = W; }

typedef struct {
  double x[12], z1[32], h1[32], z2[32], h2[32], o[4];
} or_mlp_cache;

static void or_mlp_run(const double* W, const double x[12], or_mlp_cache* c) {
  for (int k = 0; k < 12; ++k) c->x[k] = x[k];
  for (int j = 0; j < 32; ++j) {
    double a = W[L_B1 + j];
    for (int k = 0; k < 12; ++k) a += W[L_W1 + 12 * j + k] * x[k];
    c->z1[j] = a;
    c->h1[j] = a > 0.0 ? a : 0.0;
  }
  for (int j = 0; j < 32; ++j) {
    double a = W[L_B2 + j];
    for (int k = 0; k < 32; ++k) a += W[L_W2 + 32 * j + k] * c->h1[k];
    c->z2[j] = a;
    c->h2[j] = a > 0.0 ? a : 0.0;
  }
  for (int j = 0; j < 4; ++j) {
    double a = W[L_B3 + j];
    for (int k = 0; k < 32; ++k) a += W[L_W3 + 32 * j + k] * c->h2[k];
    c->o[j] = a;
  }
}

void or_mlp_forward(const double* W, const double x[12], double out[4]) {
  or_mlp_cache c;
  or_mlp_run(W, x, &c);
  for (int j = 0; j < 4; ++j) out[j] = c.o[j];
}

/* BF16 reading of the network (the tensor-core evaluators of the library):
 * every operand of a product is a BF16 value -- the inputs, the weights and
 * biases (rounded from their FP32 value) and the hidden activations (the ReLU
 * of the exact sum, rounded) -- while the sums themselves are exact here (the
 * GPU accumulates in FP32, so a rounded value near a BF16 rounding boundary
 * may round the other way there: or_bf16_slack measures how near). */
double or_bf16_slack(double v, double T) {
  if (v == 0.0 || !(T > 0.0) || !isfinite(v)) return INFINITY;
  if (ldexp(1.0, ilogb(v) - 7) < ldexp(T, -16)) return INFINITY;
  const float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, 4);
  const uint32_t sign = u & 0x80000000u, mag = u & 0x7FFF0000u;
  double best = INFINITY;
  /* the boundaries below, inside and above the BF16 interval holding f */
  for (int k = -1; k <= 1; ++k) {
    const int64_t b = (int64_t)mag + 0x8000 + (int64_t)k * 0x10000;
    if (b < 0 || b >= 0x7F800000) continue;
    const uint32_t bu = sign | (uint32_t)b;
    float bf;
    memcpy(&bf, &bu, 4);
    const double d = fabs(v - (double)bf);
    if (d < best) best = d;
  }
  return best / T;
}

static double or_wbf(const double* W, int k) { return or_round_bf16((float)W[k]); }

/* T3 (optional, 4): magnitude of the terms of each output's sum */
static void or_mlp_bf16_run(const double* W, const double x[12], const double* Tx,
                            double out[4], double* T3, double* slack) {
  double sl = slack ? *slack : INFINITY;
  double xb[12], h1[32], h2[32];
  for (int k = 0; k < 12; ++k) {
    xb[k] = or_round_bf16((float)x[k]);
    if (Tx) sl = fmin(sl, or_bf16_slack(x[k], Tx[k]));
  }
  for (int j = 0; j < 32; ++j) {
    double a = or_wbf(W, L_B1 + j), T = fabs(a);
    for (int k = 0; k < 12; ++k) {
      const double t = or_wbf(W, L_W1 + 12 * j + k) * xb[k];
      a += t;
      T += fabs(t);
    }
    h1[j] = a > 0.0 ? or_round_bf16((float)a) : 0.0;
    if (a > 0.0) sl = fmin(sl, or_bf16_slack(a, T));
  }
  for (int j = 0; j < 32; ++j) {
    double a = or_wbf(W, L_B2 + j), T = fabs(a);
    for (int k = 0; k < 32; ++k) {
      const double t = or_wbf(W, L_W2 + 32 * j + k) * h1[k];
      a += t;
      T += fabs(t);
    }
    h2[j] = a > 0.0 ? or_round_bf16((float)a) : 0.0;
    if (a > 0.0) sl = fmin(sl, or_bf16_slack(a, T));
  }
  for (int j = 0; j < 4; ++j) {
    double a = or_wbf(W, L_B3 + j), T = fabs(a);
    for (int k = 0; k < 32; ++k) {
      const double t = or_wbf(W, L_W3 + 32 * j + k) * h2[k];
      a += t;
      T += fabs(t);
    }
    out[j] = a;
    if (T3) T3[j] = T;
  }
  if (slack) *slack = sl;
}

void or_mlp_forward_bf16(const double* W, const double x[12], const double* Tx,
                         double out[4], double* slack) {
  or_mlp_bf16_run(W, x, Tx, out, NULL, slack);
}

/* Back-propagation of output gradients go[4] through the cached run: adds
 * the parameter gradients to gW (optional) and returns input gradients gx. */
static void or_mlp_backward(const double* W, const or_mlp_cache* c, const double go[4],
                            double* gW, double gx[12]) {
  double gh2[32], gz2[32], gh1[32], gz1[32];
  for (int k = 0; k < 32; ++k) {
    double a = 0.0;
    for (int j = 0; j < 4; ++j) a += W[L_W3 + 32 * j + k] * go[j];
    gh2[k] = a;
  }
  for (int k = 0; k < 32; ++k) gz2[k] = c->z2[k] > 0.0 ? gh2[k] : 0.0;
  for (int k = 0; k < 32; ++k) {
    double a = 0.0;
    for (int j = 0; j < 32; ++j) a += W[L_W2 + 32 * j + k] * gz2[j];
    gh1[k] = a;
  }
  for (int k = 0; k < 32; ++k) gz1[k] = c->z1[k] > 0.0 ? gh1[k] : 0.0;
  for (int k = 0; k < 12; ++k) {
    double a = 0.0;
    for (int j = 0; j < 32; ++j) a += W[L_W1 + 12 * j + k] * gz1[j];
    gx[k] = a;
  }
  if (gW) {
    for (int j = 0; j < 4; ++j) {
      gW[L_B3 + j] += go[j];
      for (int k = 0; k < 32; ++k) gW[L_W3 + 32 * j + k] += go[j] * c->h2[k];
    }
    for (int j = 0; j < 32; ++j) {
      gW[L_B2 + j] += gz2[j];
      for (int k = 0; k < 32; ++k) gW[L_W2 + 32 * j + k] += gz2[j] * c->h1[k];
    }
    for (int j = 0; j < 32; ++j) {
      gW[L_B1 + j] += gz1[j];
      for (int k = 0; k < 12; ++k) gW[L_W1 + 12 * j + k] += gz1[j] * c->x[k];
    }
  }
}

/* Per-axis gradient of omega_t at r: the face differences omega(c) -
 * omega(c-e) and omega(c+e) - omega(c) interpolated linearly in the position
 * t = r - floor(r) inside the cell.  dgrad (optional, 3) receives the
 * derivative of each component with respect to its own coordinate. */
static void or_field_gradient(const or_system* s, const double* w_t, const double r[3],
                              double g[3], double dgrad[3]) {
  uint64_t c = or_cell(s, r[0], r[1], r[2]);
  for (int d = 0; d < 3; ++d) {
    double t = r[d] - floor(r[d]);
    double lo = w_t[c] - w_t[or_cell_shift(s, c, d, -1)];
    double hi = w_t[or_cell_shift(s, c, d, +1)] - w_t[c];
    g[d] = (1.0 - t) * lo + t * hi;
    if (dgrad) dgrad[d] = hi - lo;
  }
}

void or_learned_features(const or_system* s, const float* x, const float* y, const float* z,
                         const double* w_t, uint64_t chain, uint32_t i, const double r[3],
                         double feat[12]) {
  for (int k = 0; k < 12; ++k) feat[k] = 0.0;
  const uint64_t m0 = chain * s->N;
  if (i > 0) {
    uint64_t n = m0 + i - 1;
    feat[0] = r[0] - x[n]; feat[1] = r[1] - y[n]; feat[2] = r[2] - z[n];
  }
  if (i + 1 < s->N) {
    uint64_t n = m0 + i + 1;
    feat[3] = x[n] - r[0]; feat[4] = y[n] - r[1]; feat[5] = z[n] - r[2];
  }
  or_field_gradient(s, w_t, r, feat + 6, NULL);
  feat[9] = or_is_B(s, chain, i) ? 0.0 : 1.0;
  feat[10] = (i > 0) ? 1.0 : 0.0;
  feat[11] = (i + 1 < s->N) ? 1.0 : 0.0;
}

/* Magnitudes of the terms each feature at r is formed from, for the slack of
 * its BF16 rounding: dr[d] bounds (as a magnitude) how far the GPU's r may
 * lie from r -- 0 at the particle's own stored position, which both sides
 * hold exactly, so that its bond vectors (one FP32 rounding of an exact
 * difference on both sides) are reproduced exactly; the field gradient is
 * formed from three field values (and r when dr > 0); the flags are exact. */
static void or_feature_terms(const or_system* s, const double* w_t, uint32_t i,
                             const double r[3], const double dr[3], const double feat[12],
                             double T[12]) {
  for (int k = 0; k < 12; ++k) T[k] = 0.0;
  for (int d = 0; d < 3; ++d) {
    if (i > 0 && dr[d] > 0.0) T[d] = dr[d] + fabs(feat[d]);
    if (i + 1 < s->N && dr[d] > 0.0) T[3 + d] = dr[d] + fabs(feat[3 + d]);
  }
  const uint64_t c = or_cell(s, r[0], r[1], r[2]);
  for (int d = 0; d < 3; ++d) {
    const double wm = w_t[or_cell_shift(s, c, d, -1)], wp = w_t[or_cell_shift(s, c, d, +1)];
    const double lo = w_t[c] - wm, hi = wp - w_t[c];
    T[6 + d] = fabs(w_t[c]) + fabs(wm) + fabs(wp) + fabs(hi - lo) * dr[d];
  }
}

/* proposal parameters of the network outputs */
static double or_sigma0(const or_system* s) { return s->a / sqrt(3.0); }
static double or_logsig(const double o3) { return 2.0 * tanh(0.5 * o3); }

/* log q(to | from) up to a constant, for network outputs o at `from` */
static double or_log_q(const or_system* s, const double o[4], const double from[3],
                       const double to[3]) {
  double sig = or_sigma0(s) * exp(or_logsig(o[3]));
  double r2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    double e = to[d] - from[d] - o[d];
    r2 += e * e;
  }
  return -r2 / (2.0 * sig * sig) - 3.0 * log(sig);
}

static double or_bond_energy(const or_system* s, const float* x, const float* y, const float* z,
                             uint64_t chain, uint32_t i, const double r[3]) {
  double e = 0.0;
  for (int side = -1; side <= 1; side += 2) {
    long long jn = (long long)i + side;
    if (jn < 0 || jn >= (long long)s->N) continue;
    uint64_t n = chain * s->N + (uint64_t)jn;
    double rn[3] = { x[n], y[n], z[n] };
    for (int d = 0; d < 3; ++d) e += s->K_b * (r[d] - rn[d]) * (r[d] - rn[d]);
  }
  return e;
}

static void or_move_learned(const or_system* s, float* x, float* y, float* z,
                            const double* wA, const double* wB, uint32_t sweep,
                            uint64_t chain, uint32_t i, double* margin, uint8_t* accepted,
                            float* trial, uint64_t* acc, uint64_t* ties) {
  const uint64_t m = chain * s->N + i;
  const double* w_t = or_is_B(s, chain, i) ? wB : wA;
  uint32_t w1[4], w2[4];
  or_draw(s, OR_PURPOSE_MOVE, m, sweep, w1);
  or_draw(s, OR_PURPOSE_MOVE2, m, sweep, w2);
  double xi[4];
  for (int p = 0; p < 2; ++p) {
    double u1 = or_uniform_open(w1[2 * p]), u2 = or_uniform_open(w1[2 * p + 1]);
    double rad = sqrt(-2.0 * log(u1)), th = 2.0 * M_PI * u2;
    xi[2 * p] = rad * cos(th);
    xi[2 * p + 1] = rad * sin(th);
  }
  double r_old[3] = { x[m], y[m], z[m] }, r_new[3], f[12], o[4], o_rev[4];
  double T[12], T3[4], slack = INFINITY;
  const double dr0[3] = { 0.0, 0.0, 0.0 };
  or_learned_features(s, x, y, z, w_t, chain, i, r_old, f);
  if (s->mlp_bf16) {
    or_feature_terms(s, w_t, i, r_old, dr0, f, T);
    or_mlp_bf16_run(s->mlp, f, T, o, T3, &slack);
  } else {
    or_mlp_forward(s->mlp, f, o);
  }
  const double sig = or_sigma0(s) * exp(or_logsig(o[3]));
  for (int d = 0; d < 3; ++d) {
    float dx = (float)(o[d] + sig * xi[d]);
    r_new[d] = (double)(float)(r_old[d] + (double)dx);
  }
  if (trial) {
    const uint64_t M = s->n_chains * s->N;
    for (int d = 0; d < 3; ++d) trial[d * M + m] = (float)r_new[d];
  }
  or_learned_features(s, x, y, z, w_t, chain, i, r_new, f);
  if (s->mlp_bf16) {
    /* the trial position inherits the rounding of the outputs, the step
       scale and the normals on the GPU, and one rounding of the position
       itself (2^-4 |r'| carries it at the 2^-19 relative level of the rest) */
    double dr[3];
    for (int d = 0; d < 3; ++d)
      dr[d] = fabs(o[d]) + sig * fabs(xi[d]) + T3[d] + ldexp(fabs(r_new[d]), -4);
    or_feature_terms(s, w_t, i, r_new, dr, f, T);
    or_mlp_bf16_run(s->mlp, f, T, o_rev, NULL, &slack);
    if (s->mlp_slack) s->mlp_slack[m] = slack;
  } else {
    or_mlp_forward(s->mlp, f, o_rev);
  }
  double dE = or_bond_energy(s, x, y, z, chain, i, r_new) - or_bond_energy(s, x, y, z, chain, i, r_old)
              + (w_t[or_cell(s, r_new[0], r_new[1], r_new[2])] - w_t[or_cell(s, r_old[0], r_old[1], r_old[2])]);
  const double log_alpha = -dE + or_log_q(s, o_rev, r_new, r_old) - or_log_q(s, o, r_old, r_new);
  const double lnu = log(or_uniform_open(w2[0]));
  const int acc_move = (log_alpha >= 0.0) || (lnu < log_alpha);
  if (margin) margin[m] = lnu - log_alpha;
  if (fabs(lnu - log_alpha) < 1e-4) (*ties)++;
  if (acc_move) {
    x[m] = (float)r_new[0]; y[m] = (float)r_new[1]; z[m] = (float)r_new[2];
    (*acc)++;
  }
  if (accepted) accepted[m] = (uint8_t)acc_move;
}

/* Expected squared jump of one sample with its reparameterised gradient:
 * r' = r + mu(x) + sigma(x) xi,  D = |r'-r|^2,
 * l = -dE(r') + log q(r|r') - log q(r'|r),  J = min(1, e^l) D.
 * The field term of dE is piecewise constant in r' (zero derivative); the
 * features at r' depend on r' through the bond vectors and the interpolated
 * field gradient.  Positions are not rounded to FP32 here (a smooth surrogate
 * of the move used for training). */
double or_esjd_sample(const or_system* s, const double* W, const float* x, const float* y,
                      const float* z, const double* wA, const double* wB, uint64_t chain,
                      uint32_t i, const double xi[3], double* grad, double* log_alpha_out) {
  const uint64_t m = chain * s->N + i;
  const double* w_t = or_is_B(s, chain, i) ? wB : wA;
  const double r[3] = { x[m], y[m], z[m] };
  double f[12], fr[12];
  or_mlp_cache cf, cr;
  or_learned_features(s, x, y, z, w_t, chain, i, r, f);
  or_mlp_run(W, f, &cf);
  const double ls = or_logsig(cf.o[3]);
  const double sig = or_sigma0(s) * exp(ls);
  double rp[3], dvec[3];
  for (int d = 0; d < 3; ++d) {
    dvec[d] = cf.o[d] + sig * xi[d];
    rp[d] = r[d] + dvec[d];
  }
  or_learned_features(s, x, y, z, w_t, chain, i, rp, fr);
  or_mlp_run(W, fr, &cr);
  const double lsr = or_logsig(cr.o[3]);
  const double sigr = or_sigma0(s) * exp(lsr);
  double e[3], e2 = 0.0, D = 0.0;
  for (int d = 0; d < 3; ++d) {
    e[d] = r[d] - rp[d] - cr.o[d];  /* reverse residual */
    e2 += e[d] * e[d];
    D += dvec[d] * dvec[d];
  }
  double xi2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
  double dE = or_bond_energy(s, x, y, z, chain, i, rp) - or_bond_energy(s, x, y, z, chain, i, r)
              + (w_t[or_cell(s, rp[0], rp[1], rp[2])] - w_t[or_cell(s, r[0], r[1], r[2])]);
  double lq_rev = -e2 / (2.0 * sigr * sigr) - 3.0 * log(sigr);
  double lq_fwd = -0.5 * xi2 - 3.0 * log(sig);
  double l = -dE + lq_rev - lq_fwd;
  if (log_alpha_out) *log_alpha_out = l;
  double alpha = l >= 0.0 ? 1.0 : exp(l);
  double J = alpha * D;
  if (!grad) return J;
  /* dJ = alpha dD + [l < 0] alpha D dl */
  const double cl = (l < 0.0) ? alpha * D : 0.0;
  /* gradient with respect to r' (through D, -dE, lq_rev's residual and features) */
  double g_rp[3];
  for (int d = 0; d < 3; ++d) g_rp[d] = alpha * 2.0 * dvec[d];
  /* -dE: bond part */
  for (int side = -1; side <= 1; side += 2) {
    long long jn = (long long)i + side;
    if (jn < 0 || jn >= (long long)s->N) continue;
    uint64_t n = chain * s->N + (uint64_t)jn;
    double rn[3] = { x[n], y[n], z[n] };
    for (int d = 0; d < 3; ++d) g_rp[d] += cl * (-2.0 * s->K_b * (rp[d] - rn[d]));
  }
  /* lq_rev: explicit residual e = r - r' - mu_r(r'): de/dr' = -I */
  for (int d = 0; d < 3; ++d) g_rp[d] += cl * (e[d] / (sigr * sigr));
  /* lq_rev through the reverse network outputs */
  double go_r[4];
  for (int d = 0; d < 3; ++d) go_r[d] = cl * (e[d] / (sigr * sigr));  /* d lq/d mu_r */
  {
    /* d lq_rev/d ls_r = e2/sigr^2 - 3 ; d ls/d o3 = 1 - tanh^2(o3/2) */
    double th = tanh(0.5 * cr.o[3]);
    go_r[3] = cl * (e2 / (sigr * sigr) - 3.0) * (1.0 - th * th);
  }
  double gfr[12];
  or_mlp_backward(W, &cr, go_r, grad, gfr);
  /* features at r' -> r': bond vectors (+I for prev, -I for next) and the
   * interpolated field gradient (d g_d / d r'_d = hi - lo) */
  double dg[3], gtmp[3];
  or_field_gradient(s, w_t, rp, gtmp, dg);
  for (int d = 0; d < 3; ++d) {
    if (i > 0) g_rp[d] += gfr[d];
    if (i + 1 < s->N) g_rp[d] -= gfr[3 + d];
    g_rp[d] += gfr[6 + d] * dg[d];
  }
  /* r' = r + mu(x) + sigma(x) xi: to the forward network outputs, plus the
   * -lq_fwd = +3 ls term */
  double go_f[4];
  for (int d = 0; d < 3; ++d) go_f[d] = g_rp[d];
  {
    double th = tanh(0.5 * cf.o[3]);
    double dls = 0.0;
    for (int d = 0; d < 3; ++d) dls += g_rp[d] * sig * xi[d];
    dls += cl * 3.0;
    go_f[3] = dls * (1.0 - th * th);
  }
  double gf[12];
  or_mlp_backward(W, &cf, go_f, grad, gf);
  return J;
}

/* Set order of one chain for one sweep: bit 0 of the fourth word of the move
 * draw of the chain's first particle picks odd->even (1) or even->odd (0); the
 * 24 bits that make the acceptance uniform are the word's top bits, so the set
 * order is independent of every uniform the moves use. */
static uint32_t or_first_set(const or_system* s, uint64_t chain, uint32_t sweep) {
  if (s->set_order != 0) return 0u;
  uint32_t w[4];
  or_draw(s, OR_PURPOSE_MOVE, chain * s->N, sweep, w);
  return w[3] & 1u;
}

void or_sweep(const or_system* s, float* x, float* y, float* z,
              const double* wA, const double* wB, uint32_t sweep,
              uint64_t c0, uint64_t c1,
              double* margin, uint8_t* accepted, or_sweep_stats* st) {
  or_sweep_trial(s, x, y, z, wA, wB, sweep, c0, c1, margin, accepted, NULL, st);
}

void or_sweep_trial(const or_system* s, float* x, float* y, float* z,
                    const double* wA, const double* wB, uint32_t sweep,
                    uint64_t c0, uint64_t c1,
                    double* margin, uint8_t* accepted, float* trial, or_sweep_stats* st) {
  const uint32_t N = s->N;
  uint64_t acc = 0, ties = 0;
  long long i0 = (long long)c0, i1 = (long long)c1;
#pragma omp parallel for schedule(static) reduction(+ : acc, ties)
  for (long long cc = i0; cc < i1; ++cc) {
    uint64_t chain = (uint64_t)cc;
    if (s->set_order == 2) {
      for (uint32_t j = 0; j < or_length(s, chain); ++j) {
        uint64_t a1 = 0, t1 = 0;
        or_move_attempt(s, x, y, z, wA, wB, sweep, chain, j, margin, accepted, trial,
                        s->chosen, &a1, &t1);
        acc += a1;
        ties += t1;
      }
      continue;
    }
    if (s->topo && s->arch) {
      /* sets of the molecule's architecture in this sweep's order; within a
       * set the particles are independent, so their order does not matter */
      const uint32_t a = s->arch[chain];
      const uint32_t n_sets = s->topo_nsets[a];
      uint32_t order[8];
      or_set_order(s, chain, sweep, n_sets, order);
      for (uint32_t k = 0; k < n_sets; ++k)
        for (uint32_t i = 0; i < N; ++i) {
          if (s->topo_set[(uint64_t)a * N + i] != order[k]) continue;
          uint64_t a1 = 0, t1 = 0;
          if (s->move == 1)
            or_move_smc(s, x, y, z, wA, wB, sweep, chain, i, margin, accepted, trial, &a1, &t1);
          else
            or_move_uniform(s, x, y, z, wA, wB, sweep, chain, i, margin, accepted, trial, &a1, &t1);
          acc += a1;
          ties += t1;
        }
      continue;
    }
    uint32_t first = or_first_set(s, chain, sweep);
    for (uint32_t k = 0; k < 2; ++k) {
      uint32_t set = first ^ k;
      for (uint32_t i = set; i < N; i += 2) {
        uint64_t a1 = 0, t1 = 0;
        if (s->move == 1)
          or_move_smc(s, x, y, z, wA, wB, sweep, chain, i, margin, accepted, trial, &a1, &t1);
        else if (s->move == 2)
          or_move_learned(s, x, y, z, wA, wB, sweep, chain, i, margin, accepted, trial, &a1, &t1);
        else
          or_move_uniform(s, x, y, z, wA, wB, sweep, chain, i, margin, accepted, trial, &a1, &t1);
        acc += a1;
        ties += t1;
      }
    }
  }
  if (st) {
    uint64_t att = 0;
    for (uint64_t k = c0; k < c1; ++k) att += or_length(s, k);
    st->attempted += att;
    st->accepted += acc;
    st->near_ties += ties;
  }
}

/* One SCMF cycle in the order of Sec. 2.2 as run by the library: the fields of
 * the current configuration are frozen for the MC step, then the occupation
 * numbers and the fields are recomputed from the new configuration. */
void or_cycle(const or_system* s, float* x, float* y, float* z,
              uint32_t* nA, uint32_t* nB, double* wA, double* wB,
              uint32_t sweep, int round_mode, or_sweep_stats* st) {
  or_sweep(s, x, y, z, wA, wB, sweep, 0, s->n_chains, NULL, NULL, st);
  or_histogram(s, x, y, z, nA, nB);
  or_fields(s, nA, nB, wA, wB, round_mode);
}

/* ------------------------------------------------------------------------- */
/* a5: observables.                                                             */
/*   E_b  = sum_bonds (k0/2) |b|^2               (Eq. h-bond, V-harmonic)       */
/*   E_nb = rho_0 dL^3 / N * sum_c [ kappaN/2 (phiA+phiB-1)^2                    */
/*                                   - chiN/4 (phiA-phiB)^2 ]   (Eq. discrete-ham, */
/*          K_fluc + K^0 with the A-B pair counted once)                         */
/* ------------------------------------------------------------------------- */
void or_observables(const or_system* s, const float* x, const float* y, const float* z,
                    const uint32_t* nA, const uint32_t* nB, or_obs* out) {
  const uint32_t N = s->N;
  double Eb = 0.0, Re2 = 0.0, b2 = 0.0;
  double n_bonds = 0.0;
  for (uint64_t k = 0; k < s->n_chains; ++k) {
    uint64_t m0 = k * N;
    if (s->topo && s->arch) {
      /* every bond once: from the particle with the smaller index */
      uint32_t partners[256];
      for (uint32_t i = 0; i < or_length(s, k); ++i) {
        const uint32_t np = or_partners(s, k, i, partners);
        for (uint32_t b = 0; b < np; ++b) {
          const uint32_t j = partners[b];
          if (j <= i) continue;
          double dx = (double)x[m0 + j] - (double)x[m0 + i];
          double dy = (double)y[m0 + j] - (double)y[m0 + i];
          double dz = (double)z[m0 + j] - (double)z[m0 + i];
          double bb = dx * dx + dy * dy + dz * dz;
          b2 += bb;
          Eb += s->K_b * bb;
          n_bonds += 1.0;
        }
      }
    }
    for (uint32_t i = 0; i + 1 < N && !(s->topo && s->arch); ++i) {
      double dx = (double)x[m0 + i + 1] - (double)x[m0 + i];
      double dy = (double)y[m0 + i + 1] - (double)y[m0 + i];
      double dz = (double)z[m0 + i + 1] - (double)z[m0 + i];
      double bb = dx * dx + dy * dy + dz * dz;
      b2 += bb;
      Eb += s->K_b * bb;
    }
    const uint32_t last = or_length(s, k) - 1u;   /* the molecule's last particle */
    double ex = (double)x[m0 + last] - (double)x[m0];
    double ey = (double)y[m0 + last] - (double)y[m0];
    double ez = (double)z[m0 + last] - (double)z[m0];
    Re2 += ex * ex + ey * ey + ez * ez;
  }
  const uint64_t cells = (uint64_t)s->grid[0] * s->grid[1] * s->grid[2];
  double K = 0.0, Eext = 0.0;
  for (uint64_t c = 0; c < cells; ++c) {
    double phiA = (double)nA[c] / s->rho_cell;
    double phiB = (double)nB[c] / s->rho_cell;
    double fl = phiA + phiB - 1.0;
    double df = phiA - phiB;
    if (s->hamiltonian == 1)
      K += 0.5 * s->kappaN * fl * fl + s->chiN * phiA * phiB;
    else
      K += 0.5 * s->kappaN * fl * fl - 0.25 * s->chiN * df * df;
    if (s->ext) Eext += (double)nA[c] * s->ext[c] + (double)nB[c] * s->ext[cells + c];
  }
  out->E_b = Eb;
  out->E_nb = s->rho_cell / (double)N * K;
  out->E_ext = Eext;
  out->Re2 = Re2 / (double)s->n_chains;
  if (!(s->topo && s->arch)) n_bonds = (double)s->n_chains * (double)(N > 1 ? N - 1 : 0);
  out->b2 = n_bonds > 0.0 ? b2 / n_bonds : 0.0;
}

/* Composition structure factor on the collocation grid (the radial S(q) of
 * Sec. 5.6 is the shell average of this quantity).  Direct DFT. */
void or_structure_factor(const or_system* s, const uint32_t* nA, const uint32_t* nB,
                         const int32_t* m, size_t k, double* out) {
  const double M = or_particles(s);
  for (size_t q = 0; q < k; ++q) {
    double re = 0.0, im = 0.0;
    for (uint32_t cz = 0; cz < s->grid[2]; ++cz)
      for (uint32_t cy = 0; cy < s->grid[1]; ++cy)
        for (uint32_t cx = 0; cx < s->grid[0]; ++cx) {
          uint64_t c = ((uint64_t)cz * s->grid[1] + cy) * s->grid[0] + cx;
          double dn = (double)nA[c] - (double)nB[c];
          if (dn == 0.0) continue;
          double ph = 2.0 * M_PI * ((double)m[3 * q] * cx / s->grid[0] +
                                    (double)m[3 * q + 1] * cy / s->grid[1] +
                                    (double)m[3 * q + 2] * cz / s->grid[2]);
          re += dn * cos(ph);
          im -= dn * sin(ph);
        }
    out[q] = (re * re + im * im) / M;
  }
}
