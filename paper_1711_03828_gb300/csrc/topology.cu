// topology.cu -- the SET Monte-Carlo step for molecules of any architecture
// (arXiv:1711.03828, Sec. 3.1.2, second scheme, with the molecular-architecture
// array of Sec. 3.2.1), and the bond sums of the observables for them.
//
// Architecture array (Sec. 3.2.1, Fig. polyarch): per architecture a block of
// N, then one word per particle, (index of its first bond word << 8) | type
// (0xFFFFFF: no bonds), the bond words holding (signed 27-bit partner offset
// << 5) | (bond type << 1) | last.  A molecule has the system's N <= 64
// particle slots; its architecture (mol_arch) fills the first n <= N of them,
// the others are absent (never moved or counted).
// The array is checked and re-encoded on the host when it is set: per
// particle one 32-bit word with its number of partners, its first three
// partners, its type, its set and the number of sets (L1-resident: 256 bytes
// per architecture), and a 64-bit mask of all its partners that the kernel
// reads only for a particle with more than three; no list of dependent loads
// is walked on the device.
//
// Independent sets: generated on the host when the architectures are set
// (particles in index order take the smallest set index that none of their
// earlier bond partners holds) and kept per architecture; a molecule visits
// its sets in a random order per sweep: with two sets the linear-chain rule
// (bit 0 of the acceptance word of particle 0's move draw puts set 1 first),
// with more an inside-out Fisher-Yates shuffle driven by the 16-bit halves of
// one Philox draw (purpose 6, counter = molecule, sweep).
//
// Work decomposition.  A warp owns a tile of G = floor(64/N) whole molecules;
// lane l draws for tile particles l and l + 32 (coalesced 4-byte loads for any
// N); the next tile's positions and architectures are loaded during the
// current.  Draws, trial positions, cells and both field values are computed
// first and recorded, with the positions, in a per-warp shared-memory record.
// Step k of the tile then moves every particle whose set its molecule visits
// k-th: those particles are listed (ballot + prefix count) and taken one per
// lane, so every lane is busy whatever the sizes and orders of the sets, and a
// mover reads its bond partners from the record wherever they sit.  Bond
// energy change of r -> r + d with partners q: K_b (2 d.U + k d.d),
// U = sum_q (r - r_q).  256 threads, 3 blocks per SM (80 registers, 28 KB of
// shared memory per block).
#include <algorithm>

#include "kernels.h"
#include "draws.cuh"

namespace soma {

namespace {

constexpr uint32_t TOPO_NO_BONDS = 0xFFFFFFu;
constexpr uint32_t PURPOSE_SETS = 6;
constexpr int TOPO_TILE = 64;
constexpr int TOPO_WARPS = 8;
constexpr int TOPO_MAX_SETS = 8;

// Visiting step of every set of one molecule, 4 bits per set (nibble s = the
// step at which set s moves).
__device__ __forceinline__ uint32_t set_steps(uint32_t n_sets, bool random, uint32_t first_bit,
                                              uint64_t mol, uint32_t sweep, uint32_t ctr3,
                                              const Geom& g) {
  if (n_sets < 2) return 0u;
  if (!random) {
    uint32_t s = 0;
#pragma unroll
    for (uint32_t k = 1; k < TOPO_MAX_SETS; ++k)
      if (k < n_sets) s |= k << (4u * k);
    return s;
  }
  if (n_sets == 2) return first_bit ? 0x01u : 0x10u;
  const uint64_t gm = mol + g.chain_base;
  const uint4 r = philox_rk(make_uint4((uint32_t)gm, (uint32_t)(gm >> 32), sweep, ctr3), g);
  const uint32_t w[4] = {r.x, r.y, r.z, r.w};
  uint32_t order = 0;  // nibble k: the set visited at step k
#pragma unroll
  for (uint32_t k = 1; k < TOPO_MAX_SETS; ++k) {
    if (k >= n_sets) break;
    const uint32_t h = (w[(k - 1u) >> 1] >> (16u * ((k - 1u) & 1u))) & 0xFFFFu;
    const uint32_t j = (h * (k + 1u)) >> 16;
    const uint32_t oj = (order >> (4u * j)) & 15u;
    order = (order & ~(15u << (4u * k))) | (oj << (4u * k));
    order = (order & ~(15u << (4u * j))) | (k << (4u * j));
  }
  uint32_t steps = 0;
#pragma unroll
  for (uint32_t k = 0; k < TOPO_MAX_SETS; ++k)
    if (k < n_sets) steps |= k << (4u * ((order >> (4u * k)) & 15u));
  return steps;
}

// Per-particle word of the architecture table: bits 0-5 number of partners,
// 6-11 / 12-17 / 18-23 the first three partners (index in the molecule),
// bit 24 type (1 = B), 25-27 set, 28-31 number of sets of the architecture.
__device__ __forceinline__ uint32_t pw_degree(uint32_t w) { return w & 63u; }
__device__ __forceinline__ uint32_t pw_partner(uint32_t w, int k) { return (w >> (6 + 6 * k)) & 63u; }
__device__ __forceinline__ bool pw_is_B(uint32_t w) { return (w >> 24) & 1u; }
__device__ __forceinline__ uint32_t pw_set(uint32_t w) { return (w >> 25) & 7u; }
__device__ __forceinline__ uint32_t pw_sets(uint32_t w) { return w >> 28; }

// Shared-memory record of one warp's tile, one 16-byte entry per particle and
// array (a mover reads each with one 128-bit access), entry q at slot
// rec(q) = q + q/8: a quarter warp's 128-bit accesses are conflict-free when
// its eight entries fall in distinct 16-byte bank groups, and the movers of
// one set of a chain (every second particle) do once each run of eight
// entries is shifted by one slot.  P = current position and
// final cell, T = trial position and acceptance threshold (smart Monte Carlo:
// the three normals and ln u), Q = table word, trial cell, molecule start |
// architecture << 8, type; W (smart Monte Carlo only) = omega and field force
// at the current cell; and the list of this step's movers.
template <bool SMC>
struct TopoTile {
  static constexpr int REC = TOPO_TILE + TOPO_TILE / 8;
  static __device__ __forceinline__ uint32_t rec(uint32_t q) { return q + (q >> 3); }
  float4 P[REC];
  float4 T[REC];
  uint4 Q[REC];
  float4 W[SMC ? REC : 1];
  uint8_t movers[TOPO_TILE];
};

// IDX: particle index type (32-bit when M < 2^32: Philox counter word 1 = 0).
// MULTI: n_t particle types (type table, one field and one count plane per
// type; FP32 fields); else the two types A, B of the packed grid.
// SMC: the smart Monte Carlo move (Sec. 2.2) in place of the uniform one.  Its
// trial position depends on the force of the particle's partners, which may
// have moved in an earlier step of the tile, so only the draws are made up
// front (three Box-Muller normals and ln u from the one move draw, purpose 1,
// as for linear chains); the mover computes the
// force U of its partners from the record, the field and field force at its
// cell and at the trial cell from the per-type table, the trial position
// r + A F + sqrt(2A) xi and the acceptance min(1, exp(-dE) T(r'->r)/T(r->r')).
template <typename WT, typename IDX, bool MULTI, bool SMC>
__global__ void __launch_bounds__(256, 3) sweep_topology_kernel(const TopoArgs t) {
  __shared__ TopoTile<SMC> tiles[TOPO_WARPS];
  const SweepArgs& p = t.s;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  TopoTile<SMC>& S = tiles[wib];
  const IDX nwarps = (IDX)gridDim.x * TOPO_WARPS;
  const IDX n_tiles = (IDX)p.n_tiles;
  const IDX n_mol = (IDX)p.g.n_chains;
  const unsigned long long s64 = *p.d_sweep;
  const uint32_t sweep = (uint32_t)s64;
  uint32_t* __restrict__ nacc = MULTI ? (((s64 + 1ull) & 1ull) ? t.nt1 : t.nt0)
                                      : (((s64 + 1ull) & 1ull) ? p.n1 : p.n0);
  const WT* __restrict__ wA = static_cast<const WT*>(p.wA);
  const WT* __restrict__ wB = static_cast<const WT*>(p.wB);
  const uint32_t N = p.g.N, G = p.G;
  const uint32_t ctr3 = (PURPOSE_MOVE << 24) | (p.g.replica & 0xFFFFFFu);
  const bool random = p.set_order_random != 0;
  const uint32_t below = (1u << lane) - 1u;

  // Tile-invariant slot data, one register per slot: molecule in the tile
  // (bits 0-7) and position in the molecule (bits 8-15).  Slot j of lane l is
  // tile particle l + 32 j.
  uint32_t gc[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const uint32_t tl = (uint32_t)lane + 32u * (uint32_t)j;
    const uint32_t g = tl / N;
    gc[j] = g | (tl - g * N) << 8;
  }
  auto tile_rows = [&](IDX tile) {
    const IDX rem = n_mol - tile * G;
    return (rem < (IDX)G ? (uint32_t)rem : G) * N;
  };

  // positions, architectures (a0 | a1 << 8) and table words of the next
  // tile, loaded while the current one is processed (the field gathers of
  // a tile then wait on nothing but its own draws)
  float px[2] = {0.f, 0.f}, py[2] = {0.f, 0.f}, pz[2] = {0.f, 0.f};
  uint32_t pa = 0u, ppw[2] = {0u, 0u};
  auto prefetch = [&](IDX tile) {
    if (tile >= n_tiles) return;
    const uint32_t rows = tile_rows(tile);
    pa = 0u;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint32_t tl = (uint32_t)lane + 32u * (uint32_t)j;
      ppw[j] = 0u;
      if (tl >= rows) continue;
      const IDX m = tile * (G * N) + tl;
      px[j] = __ldcs(p.x + m);
      py[j] = __ldcs(p.y + m);
      pz[j] = __ldcs(p.z + m);
      const uint32_t aj = __ldg(t.mol_arch + (tile * G + (gc[j] & 0xFFu)));
      pa |= aj << (8 * j);
      ppw[j] = __ldg(t.ptab + aj * TOPO_TILE + (gc[j] >> 8));
    }
  };
  IDX tile = (IDX)blockIdx.x * TOPO_WARPS + wib;
  prefetch(tile);

  unsigned my_acc = 0;
  for (; tile < n_tiles; tile += nwarps) {
    const IDX chain0 = tile * G;
    const uint32_t nmono = tile_rows(tile);
    const IDX base = chain0 * N;
    const float x[2] = {px[0], px[1]}, y[2] = {py[0], py[1]}, z[2] = {pz[0], pz[1]};
    const uint32_t a2 = pa;
    const uint32_t pw2[2] = {ppw[0], ppw[1]};
    prefetch(tile + nwarps);

    // Draws, trial positions, cells and field changes of the natural slots,
    // recorded in the tile record.
    uint32_t own[2], step[2], ty[2], n_steps = 0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint32_t tl = (uint32_t)lane + 32u * (uint32_t)j;
      const bool valid = tl < nmono;
      const uint32_t ci = gc[j] >> 8;
      const uint32_t a = (a2 >> (8 * j)) & 0xFFu;
      const IDX m = base + tl;
      const uint32_t pw = pw2[j];
      const bool present = pw_sets(pw) != 0u;   // false: empty slot or absent particle
      const IDX mc = m + (IDX)p.g.id_base;
      const uint32_t hi = sizeof(IDX) > 4 ? (uint32_t)((uint64_t)mc >> 32) : 0u;
      const uint4 r = philox_rk(make_uint4((uint32_t)mc, hi, sweep, ctr3), p.g);
      const uint32_t co = cell_of(p.g, x[j], y[j], z[j]);
      // type: the architecture's type byte (n_t types) or the A/B bit
      const uint32_t type = MULTI ? (present ? __ldg(t.ttab + a * TOPO_TILE + ci) : 0u)
                                  : (uint32_t)pw_is_B(pw);
      S.P[S.rec(tl)] = make_float4(x[j], y[j], z[j], __uint_as_float(co));
      if (SMC) {
        float gx, gy, gz;
        smc_normals(r, gx, gy, gz);
        S.T[S.rec(tl)] = make_float4(gx, gy, gz, log_uniform_open(spare_uniform_word(r)));
        S.Q[S.rec(tl)] = make_uint4(pw, 0u, (gc[j] & 0xFFu) * N | a << 8, type);
        // the table entry of the current cell, gathered here for all slots at
        // once rather than inside the mover's dependent chain
        S.W[S.rec(tl)] = present ? __ldg(p.smc_tab + (size_t)type * p.g.cells + co)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        const float xn = __fmaf_rn(p.a, uniform_sym(r.x), x[j]);
        const float yn = __fmaf_rn(p.a, uniform_sym(r.y), y[j]);
        const float zn = __fmaf_rn(p.a, uniform_sym(r.z), z[j]);
        const uint32_t cn = cell_of(p.g, xn, yn, zn);
        // the field change, gathered for every slot (an absent or empty
        // slot's cells are in the grid, its value unused): no wait on the
        // table word
        float dEf;
        if (MULTI) {
          const float* wt = t.wt + (size_t)type * p.g.cells;
          dEf = __ldg(wt + cn) - __ldg(wt + co);
        } else {
          const WT* wt = type ? wB : wA;
          dEf = load_w<WT>(wt, cn) - load_w<WT>(wt, co);
        }
        S.T[S.rec(tl)] = make_float4(xn, yn, zn, -log_uniform_open(r.w) - dEf);
        S.Q[S.rec(tl)] = make_uint4(pw, cn, (gc[j] & 0xFFu) * N | a << 8, type);
      }
      ty[j] = type;
      own[j] = (valid && ci == 0u)
                   ? set_steps(pw_sets(pw), random, r.w & 1u, (uint64_t)(chain0 + (gc[j] & 0xFFu)),
                               sweep, (PURPOSE_SETS << 24) | (p.g.replica & 0xFFFFFFu), p.g)
                   : 0u;
      step[j] = pw;   // resolved below, once every slot's own steps exist
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint32_t first = (gc[j] & 0xFFu) * N;   // tile index of the molecule's particle 0
      const uint32_t v0 = __shfl_sync(FULL, own[0], (int)(first & 31u));
      const uint32_t v1 = __shfl_sync(FULL, own[1], (int)(first & 31u));
      const uint32_t pw = step[j];
      const uint32_t ns = pw_sets(pw);             // 0 for an empty slot
      step[j] = (ns ? (((first >> 5) ? v1 : v0) >> (4u * pw_set(pw))) & 15u : 15u) |
                ty[j] << 4;
      n_steps = max(n_steps, ns);
    }
    n_steps = __reduce_max_sync(FULL, n_steps);
    __syncwarp();

    // Step k: the particles whose set moves k-th are listed and taken one per
    // lane (all lanes busy whatever the sets' sizes and orders).
    for (uint32_t k = 0; k < n_steps; ++k) {
      const bool m0 = (step[0] & 15u) == k, m1 = (step[1] & 15u) == k;
      const uint32_t b0 = __ballot_sync(FULL, m0), b1 = __ballot_sync(FULL, m1);
      const uint32_t c0 = __popc(b0);
      if (m0) S.movers[__popc(b0 & below)] = (uint8_t)lane;
      if (m1) S.movers[c0 + __popc(b1 & below)] = (uint8_t)(32 + lane);
      __syncwarp();
      const uint32_t count = c0 + __popc(b1);
      for (uint32_t r = (uint32_t)lane; r < count; r += 32u) {
        const uint32_t q = S.movers[r];
        const uint4 Qq = S.Q[S.rec(q)];
        const float4 Pq = S.P[S.rec(q)];
        const uint32_t pw = Qq.x, mol0 = Qq.z & 0xFFu;
        const uint32_t deg = pw_degree(pw);
        float ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          if ((uint32_t)b < deg) {
            const float4 Pn = S.P[S.rec(mol0 + pw_partner(pw, b))];
            ux += Pq.x - Pn.x;
            uy += Pq.y - Pn.y;
            uz += Pq.z - Pn.z;
          }
        }
        if (deg > 3u) {   // the partners after the third, from the full mask
          uint64_t mk = __ldg(t.pmask + (Qq.z >> 8) * TOPO_TILE + (q - mol0));
          mk &= mk - 1ull;
          mk &= mk - 1ull;
          mk &= mk - 1ull;
          for (; mk; mk &= mk - 1ull) {
            const float4 Pn = S.P[S.rec(mol0 + (uint32_t)__ffsll((long long)mk) - 1u)];
            ux += Pq.x - Pn.x;
            uy += Pq.y - Pn.y;
            uz += Pq.z - Pn.z;
          }
        }
        const float4 Tq = S.T[S.rec(q)];
        if (SMC) {
          // bonded force -2 K_b U plus the field force of the particle's type
          const float4* __restrict__ tab = p.smc_tab + (size_t)Qq.w * p.g.cells;
          const float A = p.smc_A, K2 = 2.f * p.K_b, k = (float)deg;
          const float4 Wq = S.W[S.rec(q)];
          const float w_old = Wq.x, fox = Wq.y, foy = Wq.z, foz = Wq.w;
          float fnx, fny, fnz;
          const float Fx = fmaf(-K2, ux, fox), Fy = fmaf(-K2, uy, foy), Fz = fmaf(-K2, uz, foz);
          const float tx = __fadd_rn(Pq.x, fmaf(p.smc_s2A, Tq.x, A * Fx));
          const float ty = __fadd_rn(Pq.y, fmaf(p.smc_s2A, Tq.y, A * Fy));
          const float tz = __fadd_rn(Pq.z, fmaf(p.smc_s2A, Tq.z, A * Fz));
          const uint32_t cn = cell_of(p.g, tx, ty, tz);
          const float w_new = smc_field(tab, cn, fnx, fny, fnz);
          const float dx = tx - Pq.x, dy = ty - Pq.y, dz = tz - Pq.z;
          // bonded energy change d.(2U + k d); the force at r' uses U' = U + k d
          const float du = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
          const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          const float dE = fmaf(p.K_b, fmaf(2.f, du, k * dd), w_new - w_old);
          const float Gx = fmaf(-K2, fmaf(k, dx, ux), fnx), Gy = fmaf(-K2, fmaf(k, dy, uy), fny),
                      Gz = fmaf(-K2, fmaf(k, dz, uz), fnz);
          const float ax = dx - A * Fx, ay = dy - A * Fy, az = dz - A * Fz;     // forward residual
          const float bx = -dx - A * Gx, by = -dy - A * Gy, bz = -dz - A * Gz;  // reverse residual
          const float fwd = fmaf(ax, ax, fmaf(ay, ay, az * az));
          const float rev = fmaf(bx, bx, fmaf(by, by, bz * bz));
          const float log_alpha = fmaf(fwd - rev, p.smc_inv4A, -dE);
          if (log_alpha >= 0.f || Tq.w < log_alpha) {
            S.P[S.rec(q)] = make_float4(tx, ty, tz, __uint_as_float(cn));
            ++my_acc;
          }
        } else {
          const float dx = Tq.x - Pq.x, dy = Tq.y - Pq.y, dz = Tq.z - Pq.z;
          const float du = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
          const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (p.K_b * fmaf(2.f, du, (float)deg * dd) <= Tq.w) {
            S.P[S.rec(q)] = make_float4(Tq.x, Tq.y, Tq.z, __uint_as_float(Qq.y));
            ++my_acc;
          }
        }
      }
      __syncwarp();
    }

#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint32_t tl = (uint32_t)lane + 32u * (uint32_t)j;
      if (tl >= nmono) continue;
      const IDX m = base + tl;
      const float4 Pf = S.P[S.rec(tl)];
      if ((step[j] & 15u) == 15u) continue;   // an absent slot: kept, not counted
      __stcs(p.x + m, Pf.x);
      __stcs(p.y + m, Pf.y);
      __stcs(p.z + m, Pf.z);
      if (MULTI)
        atomicAdd(nacc + (size_t)(step[j] >> 4) * p.g.cells + __float_as_uint(Pf.w), 1u);
      else
        atomicAdd(nacc + __float_as_uint(Pf.w), (step[j] >> 4) ? 0x10000u : 1u);
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_acc += __shfl_xor_sync(FULL, my_acc, o);
  if (lane == 0 && my_acc) atomicAdd(p.acc, (unsigned long long)my_acc);
}

template <bool SMC>
const void* topology_kernel_ptr_of(int grid_dtype, bool big, bool types) {
  // the smart Monte Carlo move reads the FP32 table, whatever the field storage
  if (types || SMC) grid_dtype = 0;
  if (types)   // FP32 fields only
    return big ? (const void*)sweep_topology_kernel<float, uint64_t, true, SMC>
               : (const void*)sweep_topology_kernel<float, uint32_t, true, SMC>;
  if (big) {
    switch (grid_dtype) {
      case 1: return (const void*)sweep_topology_kernel<__nv_bfloat16, uint64_t, false, SMC>;
      case 2: return (const void*)sweep_topology_kernel<__half, uint64_t, false, SMC>;
      default: return (const void*)sweep_topology_kernel<float, uint64_t, false, SMC>;
    }
  }
  switch (grid_dtype) {
    case 1: return (const void*)sweep_topology_kernel<__nv_bfloat16, uint32_t, false, SMC>;
    case 2: return (const void*)sweep_topology_kernel<__half, uint32_t, false, SMC>;
    default: return (const void*)sweep_topology_kernel<float, uint32_t, false, SMC>;
  }
}

const void* topology_kernel_ptr(int grid_dtype, bool big, bool types, bool smc) {
  return smc ? topology_kernel_ptr_of<true>(grid_dtype, big, types)
             : topology_kernel_ptr_of<false>(grid_dtype, big, types);
}

// Sum over bonds of |r_i - r_j|^2 (each bond once, from its lower index), FP64.
__global__ void __launch_bounds__(256) topology_bonds_kernel(
    const Geom g, const float* __restrict__ x, const float* __restrict__ y,
    const float* __restrict__ z, const uint64_t* __restrict__ pmask,
    const uint8_t* __restrict__ mol_arch, const uint8_t* __restrict__ alen,
    double* __restrict__ part) {
  __shared__ double sh[2 * 32];
  double v = 0.0, re = 0.0;
  const uint64_t M = g.n_chains * g.N;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += stride) {
    const uint64_t mol = m / g.N;
    const uint32_t i = (uint32_t)(m - mol * g.N);
    const uint32_t a = __ldg(mol_arch + mol);
    const uint64_t pm = __ldg(pmask + a * TOPO_TILE + i);
    if (i == 0u) {   // end to end: particle 0 to the architecture's last particle
      const uint64_t e = m + (uint64_t)__ldg(alen + a) - 1u;
      const double dx = (double)x[e] - (double)x[m];
      const double dy = (double)y[e] - (double)y[m];
      const double dz = (double)z[e] - (double)z[m];
      re += dx * dx + dy * dy + dz * dz;
    }
    // partners above i
    for (uint64_t mk = i < 63u ? pm >> (i + 1u) : 0ull; mk; mk &= mk - 1ull) {
      const uint64_t q = m + (uint64_t)__ffsll((long long)mk);
      const double dx = (double)x[q] - (double)x[m];
      const double dy = (double)y[q] - (double)y[m];
      const double dz = (double)z[q] - (double)z[m];
      v += dx * dx + dy * dy + dz * dz;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    v += __shfl_xor_sync(FULL, v, o);
    re += __shfl_xor_sync(FULL, re, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5] = v;
    sh[32 + (threadIdx.x >> 5)] = re;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, r = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      s += sh[k];
      r += sh[32 + k];
    }
    part[2 * blockIdx.x] = s;
    part[2 * blockIdx.x + 1] = r;
  }
}

__global__ void topology_bonds_final_kernel(const double* __restrict__ part, int nb,
                                            double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s = 0.0, r = 0.0;
  for (int k = 0; k < nb; ++k) {
    s += part[2 * k];
    r += part[2 * k + 1];
  }
  out[0] = s;
  out[1] = r;
}

}  // namespace

std::string topology_tables(const uint32_t* w, uint64_t n_words, const uint32_t* start,
                            uint32_t n_arch, uint32_t N, TopologyTables* T, uint32_t n_types) {
  char msg[256];
  if (N > (uint32_t)TOPO_TILE) return "architectures take N <= 64";
  T->pmask.assign((size_t)n_arch * TOPO_TILE, 0);
  T->ptab.assign((size_t)n_arch * TOPO_TILE, 0);
  T->ttab.assign((size_t)n_arch * TOPO_TILE, 0);
  T->max_type = 0;
  T->nsets.assign(n_arch, 0);
  std::vector<uint8_t> set_of(TOPO_TILE);
  T->seq.assign(n_arch, 0);
  T->bonds.assign(n_arch, 0);
  T->len.assign(n_arch, 0);
  // absent slots: no partners, no sets (table word 0), type byte 0xFF
  std::fill(T->ttab.begin(), T->ttab.end(), (uint8_t)0xFF);
  for (uint32_t a = 0; a < n_arch; ++a) {
    const uint64_t s = start[a];
    if (s >= n_words) {
      snprintf(msg, sizeof msg, "architecture %u: block at word %llu runs past the %llu words", a,
               (unsigned long long)s, (unsigned long long)n_words);
      return msg;
    }
    const uint32_t n_a = w[s];   // particles of this architecture, the first n_a slots
    if (n_a < 1 || n_a > N) {
      snprintf(msg, sizeof msg, "architecture %u has %u particles (1..%u, the system's N)", a, n_a,
               N);
      return msg;
    }
    if (s + 1u + n_a > n_words) {
      snprintf(msg, sizeof msg, "architecture %u: block at word %llu runs past the %llu words", a,
               (unsigned long long)s, (unsigned long long)n_words);
      return msg;
    }
    T->len[a] = (uint8_t)n_a;
    uint64_t partners[TOPO_TILE] = {0};  // bit j of partners[i]: i and j are bonded
    for (uint32_t i = 0; i < n_a; ++i) {
      const uint32_t mw = w[s + 1u + i];
      const uint32_t type = mw & 0xFFu;
      if (type >= n_types) {
        snprintf(msg, sizeof msg, "architecture %u particle %u: type %u (the system has %u types)",
                 a, i, type, n_types);
        return msg;
      }
      if (type == 1u) T->seq[a] |= 1ull << i;
      T->ttab[(size_t)a * TOPO_TILE + i] = (uint8_t)type;
      T->max_type = std::max(T->max_type, type);
      const uint32_t off = mw >> 8;
      if (off == TOPO_NO_BONDS) continue;
      for (uint64_t b = off;; ++b) {
        if (b >= n_words) {
          snprintf(msg, sizeof msg, "architecture %u particle %u: bond list runs past the array",
                   a, i);
          return msg;
        }
        const uint32_t bw = w[b];
        if ((bw >> 1) & 15u) {
          snprintf(msg, sizeof msg, "architecture %u particle %u: bond type %u (harmonic 0 only)",
                   a, i, (bw >> 1) & 15u);
          return msg;
        }
        const int64_t j = (int64_t)i + ((int32_t)bw >> 5);
        if (j < 0 || j >= (int64_t)n_a || j == (int64_t)i) {
          snprintf(msg, sizeof msg, "architecture %u particle %u: partner %lld outside the molecule",
                   a, i, (long long)j);
          return msg;
        }
        if (partners[i] >> j & 1ull) {
          snprintf(msg, sizeof msg, "architecture %u particle %u: partner %lld listed twice", a, i,
                   (long long)j);
          return msg;
        }
        partners[i] |= 1ull << j;
        if (bw & 1u) break;
      }
    }
    uint32_t n_sets = 0;
    for (uint32_t i = 0; i < n_a; ++i) {
      for (uint32_t j = 0; j < n_a; ++j)
        if ((partners[i] >> j & 1ull) != (partners[j] >> i & 1ull)) {
          snprintf(msg, sizeof msg, "architecture %u: bond %u-%u listed on one side only", a, i, j);
          return msg;
        }
      if (i + 1u < 64u) T->bonds[a] += (uint32_t)__builtin_popcountll(partners[i] >> (i + 1u));
      uint32_t taken = 0;
      for (uint32_t j = 0; j < i; ++j)
        if (partners[i] >> j & 1ull) taken |= 1u << set_of[j];
      uint32_t c = 0;
      while (taken >> c & 1u) ++c;
      if (c >= (uint32_t)TOPO_MAX_SETS) {
        snprintf(msg, sizeof msg, "architecture %u needs more than %d independent sets", a,
                 TOPO_MAX_SETS);
        return msg;
      }
      set_of[i] = (uint8_t)c;
      n_sets = std::max(n_sets, c + 1u);
    }
    T->nsets[a] = (uint8_t)n_sets;
    for (uint32_t i = 0; i < n_a; ++i) {
      T->pmask[(size_t)a * TOPO_TILE + i] = partners[i];
      // degree, first three partners, type, set, sets (see pw_* above)
      uint32_t w = (uint32_t)__builtin_popcountll(partners[i]);
      uint64_t mk = partners[i];
      for (int b = 0; b < 3 && mk; ++b, mk &= mk - 1ull)
        w |= (uint32_t)__builtin_ctzll(mk) << (6 + 6 * b);
      w |= (uint32_t)(T->seq[a] >> i & 1ull) << 24 | (uint32_t)set_of[i] << 25 | n_sets << 28;
      T->ptab[(size_t)a * TOPO_TILE + i] = w;
    }
  }
  return std::string();
}

int topology_grid(int grid_dtype, bool big, int sm_count, uint64_t n_tiles, bool types, bool smc) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm,
                                                topology_kernel_ptr(grid_dtype, big, types, smc),
                                                TOPO_WARPS * 32, 0);
  if (per_sm < 1) per_sm = 1;
  const uint64_t need = (n_tiles + TOPO_WARPS - 1) / TOPO_WARPS;
  const uint64_t cap = (uint64_t)sm_count * (uint64_t)per_sm;
  return (int)std::max<uint64_t>(1, std::min(need, cap));
}

cudaError_t launch_sweep_topology(const TopoArgs& a, int grid, int grid_dtype, bool big,
                                  cudaStream_t st, bool types, bool smc) {
  void* args[] = {const_cast<TopoArgs*>(&a)};
  return cudaLaunchKernel(topology_kernel_ptr(grid_dtype, big, types, smc), dim3(grid),
                          dim3(TOPO_WARPS * 32), args, 0, st);
}

cudaError_t launch_topology_bonds(const Geom& g, const float* x, const float* y, const float* z,
                                  const uint64_t* pmask, const uint8_t* mol_arch,
                                  const uint8_t* alen, double* part, double* out,
                                  cudaStream_t st) {
  const uint64_t M = g.n_chains * g.N;
  uint64_t nb = (M + 255) / 256;
  if (nb > OBS_BLOCKS) nb = OBS_BLOCKS;
  topology_bonds_kernel<<<(unsigned)nb, 256, 0, st>>>(g, x, y, z, pmask, mol_arch, alen, part);
  topology_bonds_final_kernel<<<1, 32, 0, st>>>(part, (int)nb, out);
  return cudaGetLastError();
}

}  // namespace soma
