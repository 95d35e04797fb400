// topology.cu -- the SET Monte-Carlo step for molecules of any architecture
// (arXiv:1711.03828, Sec. 3.1.2, second scheme, with the molecular-architecture
// array of Sec. 3.2.1), and the bond sums of the observables for them.
//
// Architecture array (Sec. 3.2.1, Fig. polyarch): per architecture a block of
// N, then one word per particle, (index of its first bond word << 8) | type
// (0xFFFFFF: no bonds), the bond words holding (signed 27-bit partner offset
// << 5) | (bond type << 1) | last.  Every molecule of a system has the
// system's N <= 64 particles; mol_arch gives each molecule's architecture.
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
// lane l holds tile particles l and l + 32 (coalesced 4-byte loads for any N).
// The tile's positions are staged in shared memory, where a moving particle
// reads its bond partners (any partner in its molecule, wherever its lane).
// Draws, trial positions, cells and both field values are computed before
// the sets; then step k of the tile moves every particle whose set is visited
// k-th in its molecule, with a __syncwarp between steps.  Bond energy change of
// r -> r + d with partners q: K_b (2 d.U + k d.d), U = sum_q (r - r_q).
#include <algorithm>

#include "kernels.h"

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
  const uint4 r = philox_rk(make_uint4((uint32_t)mol, (uint32_t)(mol >> 32), sweep, ctr3), g);
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

template <typename WT>
__global__ void __launch_bounds__(256) sweep_topology_kernel(const TopoArgs t) {
  __shared__ float sh[TOPO_WARPS][3][TOPO_TILE];
  const SweepArgs& p = t.s;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* sx = sh[wib][0];
  float* sy = sh[wib][1];
  float* sz = sh[wib][2];
  const uint64_t nwarps = (uint64_t)gridDim.x * TOPO_WARPS;
  const unsigned long long s64 = *p.d_sweep;
  const uint32_t sweep = (uint32_t)s64;
  uint32_t* __restrict__ nacc = ((s64 + 1ull) & 1ull) ? p.n1 : p.n0;
  const WT* __restrict__ wA = static_cast<const WT*>(p.wA);
  const WT* __restrict__ wB = static_cast<const WT*>(p.wB);
  const uint32_t N = p.g.N;
  const uint32_t ctr3 = (PURPOSE_MOVE << 24) | (p.g.replica & 0xFFFFFFu);
  const uint32_t ctr3s = (PURPOSE_SETS << 24) | (p.g.replica & 0xFFFFFFu);
  const bool random = p.set_order_random != 0;

  // Tile-invariant slot data: tile index, molecule in the tile, position in
  // the molecule, and (lane, slot) holding the molecule's particle 0.
  uint32_t tl[2], gm[2], ci[2], src_lane[2], src_slot[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    tl[j] = (uint32_t)lane + 32u * (uint32_t)j;
    gm[j] = tl[j] / N;
    ci[j] = tl[j] - gm[j] * N;
    const uint32_t first = gm[j] * N;
    src_lane[j] = first & 31u;
    src_slot[j] = first >> 5;
  }

  unsigned my_acc = 0;
  for (uint64_t tile = (uint64_t)blockIdx.x * TOPO_WARPS + wib; tile < p.n_tiles; tile += nwarps) {
    const uint64_t chain0 = tile * p.G;
    const uint64_t rem = p.g.n_chains - chain0;
    const uint32_t nmono = (rem < p.G ? (uint32_t)rem : p.G) * N;
    const uint64_t base = chain0 * N;

    float x[2], y[2], z[2], xn[2], yn[2], zn[2], lnu[2], dEf[2];
    uint32_t co[2], cn[2], boff[2], inc[2], set_of[2], own[2], n_sets[2];
    bool valid[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      valid[j] = tl[j] < nmono;
      const uint64_t m = base + tl[j];
      x[j] = valid[j] ? __ldcs(p.x + m) : 0.f;
      y[j] = valid[j] ? __ldcs(p.y + m) : 0.f;
      z[j] = valid[j] ? __ldcs(p.z + m) : 0.f;
      sx[tl[j]] = x[j];
      sy[tl[j]] = y[j];
      sz[tl[j]] = z[j];
      const uint64_t mol = chain0 + gm[j];
      const uint32_t a = valid[j] ? __ldg(t.mol_arch + mol) : 0u;
      const uint32_t mw = __ldg(t.words + __ldg(t.start + a) + 1u + ci[j]);
      const bool isB = (mw & 0xFFu) != 0u;
      boff[j] = mw >> 8;
      inc[j] = isB ? 0x10000u : 1u;
      set_of[j] = __ldg(t.sets + a * TOPO_TILE + ci[j]);
      n_sets[j] = valid[j] ? __ldg(t.nsets + a) : 0u;
      const uint4 r = philox_rk(make_uint4((uint32_t)m, (uint32_t)(m >> 32), sweep, ctr3), p.g);
      xn[j] = __fadd_rn(x[j], __fmul_rn(p.a, uniform_sym(r.x)));
      yn[j] = __fadd_rn(y[j], __fmul_rn(p.a, uniform_sym(r.y)));
      zn[j] = __fadd_rn(z[j], __fmul_rn(p.a, uniform_sym(r.z)));
      lnu[j] = log_uniform_open(r.w);
      co[j] = cell_of(p.g, x[j], y[j], z[j]);
      cn[j] = cell_of(p.g, xn[j], yn[j], zn[j]);
      const WT* wt = isB ? wB : wA;
      dEf[j] = valid[j] ? load_w<WT>(wt, cn[j]) - load_w<WT>(wt, co[j]) : 0.f;
      own[j] = (valid[j] && ci[j] == 0u)
                   ? set_steps(n_sets[j], random, r.w & 1u, mol, sweep, ctr3s, p.g) : 0u;
    }
    uint32_t step[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint32_t v0 = __shfl_sync(FULL, own[0], (int)src_lane[j]);
      const uint32_t v1 = __shfl_sync(FULL, own[1], (int)src_lane[j]);
      step[j] = ((src_slot[j] ? v1 : v0) >> (4u * set_of[j])) & 15u;
    }
    const uint32_t n_steps = __reduce_max_sync(FULL, max(n_sets[0], n_sets[1]));
    __syncwarp();

    for (uint32_t k = 0; k < n_steps; ++k) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (!valid[j] || step[j] != k) continue;
        float ux = 0.f, uy = 0.f, uz = 0.f, nb = 0.f;
        if (boff[j] != TOPO_NO_BONDS) {
          const int mol0 = (int)(gm[j] * N) + (int)ci[j];
          // a validated list has at most N - 1 < 64 entries
          for (uint32_t b = boff[j], e = boff[j] + TOPO_TILE; b < e; ++b) {
            const uint32_t w = __ldg(t.words + b);
            const uint32_t q = (uint32_t)(mol0 + ((int32_t)w >> 5));
            ux += x[j] - sx[q];
            uy += y[j] - sy[q];
            uz += z[j] - sz[q];
            nb += 1.f;
            if (w & 1u) break;
          }
        }
        const float dx = xn[j] - x[j], dy = yn[j] - y[j], dz = zn[j] - z[j];
        const float du = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
        const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float dE = fmaf(p.K_b, fmaf(2.f, du, nb * dd), dEf[j]);
        if (dE <= -lnu[j]) {
          x[j] = xn[j];
          y[j] = yn[j];
          z[j] = zn[j];
          co[j] = cn[j];
          sx[tl[j]] = x[j];
          sy[tl[j]] = y[j];
          sz[tl[j]] = z[j];
          ++my_acc;
        }
      }
      __syncwarp();
    }

#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (!valid[j]) continue;
      const uint64_t m = base + tl[j];
      __stcs(p.x + m, x[j]);
      __stcs(p.y + m, y[j]);
      __stcs(p.z + m, z[j]);
      atomicAdd(nacc + co[j], inc[j]);
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_acc += __shfl_xor_sync(FULL, my_acc, o);
  if (lane == 0 && my_acc) atomicAdd(p.acc, (unsigned long long)my_acc);
}

const void* topology_kernel_ptr(int grid_dtype) {
  switch (grid_dtype) {
    case 1: return (const void*)sweep_topology_kernel<__nv_bfloat16>;
    case 2: return (const void*)sweep_topology_kernel<__half>;
    default: return (const void*)sweep_topology_kernel<float>;
  }
}

// Sum over bonds of |r_i - r_j|^2 (each bond once, from its lower index), FP64.
__global__ void __launch_bounds__(256) topology_bonds_kernel(
    const Geom g, const float* __restrict__ x, const float* __restrict__ y,
    const float* __restrict__ z, const uint32_t* __restrict__ words,
    const uint32_t* __restrict__ start, const uint8_t* __restrict__ mol_arch,
    double* __restrict__ part) {
  __shared__ double sh[32];
  double v = 0.0;
  const uint64_t M = g.n_chains * g.N;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += stride) {
    const uint64_t mol = m / g.N;
    const uint32_t i = (uint32_t)(m - mol * g.N);
    const uint32_t mw = __ldg(words + __ldg(start + __ldg(mol_arch + mol)) + 1u + i);
    const uint32_t b0 = mw >> 8;
    if (b0 == TOPO_NO_BONDS) continue;
    for (uint32_t b = b0, e = b0 + TOPO_TILE; b < e; ++b) {
      const uint32_t w = __ldg(words + b);
      const int32_t off = (int32_t)w >> 5;
      if (off > 0) {
        const uint64_t q = m + (uint64_t)off;
        const double dx = (double)x[q] - (double)x[m];
        const double dy = (double)y[q] - (double)y[m];
        const double dz = (double)z[q] - (double)z[m];
        v += dx * dx + dy * dy + dz * dz;
      }
      if (w & 1u) break;
    }
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    part[blockIdx.x] = s;
  }
}

__global__ void topology_bonds_final_kernel(const double* __restrict__ part, int nb,
                                            double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int k = 0; k < nb; ++k) s += part[k];
  out[0] = s;
}

}  // namespace

std::string topology_tables(const uint32_t* w, uint64_t n_words, const uint32_t* start,
                            uint32_t n_arch, uint32_t N, TopologyTables* T) {
  char msg[256];
  if (N > (uint32_t)TOPO_TILE) return "architectures take N <= 64";
  T->sets.assign((size_t)n_arch * TOPO_TILE, 0);
  T->nsets.assign(n_arch, 0);
  T->seq.assign(n_arch, 0);
  T->bonds.assign(n_arch, 0);
  for (uint32_t a = 0; a < n_arch; ++a) {
    const uint64_t s = start[a];
    if (s >= n_words || s + 1u + N > n_words) {
      snprintf(msg, sizeof msg, "architecture %u: block at word %llu runs past the %llu words", a,
               (unsigned long long)s, (unsigned long long)n_words);
      return msg;
    }
    if (w[s] != N) {
      snprintf(msg, sizeof msg, "architecture %u has %u particles, the system %u", a, w[s], N);
      return msg;
    }
    uint64_t partners[TOPO_TILE] = {0};  // bit j of partners[i]: i and j are bonded
    for (uint32_t i = 0; i < N; ++i) {
      const uint32_t mw = w[s + 1u + i];
      const uint32_t type = mw & 0xFFu;
      if (type > 1u) {
        snprintf(msg, sizeof msg, "architecture %u particle %u: type %u (0 A, 1 B only)", a, i, type);
        return msg;
      }
      if (type) T->seq[a] |= 1ull << i;
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
        if (j < 0 || j >= (int64_t)N || j == (int64_t)i) {
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
    for (uint32_t i = 0; i < N; ++i) {
      for (uint32_t j = 0; j < N; ++j)
        if ((partners[i] >> j & 1ull) != (partners[j] >> i & 1ull)) {
          snprintf(msg, sizeof msg, "architecture %u: bond %u-%u listed on one side only", a, i, j);
          return msg;
        }
      if (i + 1u < 64u) T->bonds[a] += (uint32_t)__builtin_popcountll(partners[i] >> (i + 1u));
      uint32_t taken = 0;
      for (uint32_t j = 0; j < i; ++j)
        if (partners[i] >> j & 1ull) taken |= 1u << T->sets[(size_t)a * TOPO_TILE + j];
      uint32_t c = 0;
      while (taken >> c & 1u) ++c;
      if (c >= (uint32_t)TOPO_MAX_SETS) {
        snprintf(msg, sizeof msg, "architecture %u needs more than %d independent sets", a,
                 TOPO_MAX_SETS);
        return msg;
      }
      T->sets[(size_t)a * TOPO_TILE + i] = (uint8_t)c;
      n_sets = std::max(n_sets, c + 1u);
    }
    T->nsets[a] = (uint8_t)n_sets;
  }
  return std::string();
}

int topology_grid(int grid_dtype, int sm_count, uint64_t n_tiles) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, topology_kernel_ptr(grid_dtype),
                                                TOPO_WARPS * 32, 0);
  if (per_sm < 1) per_sm = 1;
  const uint64_t need = (n_tiles + TOPO_WARPS - 1) / TOPO_WARPS;
  const uint64_t cap = (uint64_t)sm_count * (uint64_t)per_sm;
  return (int)std::max<uint64_t>(1, std::min(need, cap));
}

cudaError_t launch_sweep_topology(const TopoArgs& a, int grid, int grid_dtype, cudaStream_t st) {
  void* args[] = {const_cast<TopoArgs*>(&a)};
  return cudaLaunchKernel(topology_kernel_ptr(grid_dtype), dim3(grid), dim3(TOPO_WARPS * 32), args,
                          0, st);
}

cudaError_t launch_topology_bonds(const Geom& g, const float* x, const float* y, const float* z,
                                  const uint32_t* words, const uint32_t* start,
                                  const uint8_t* mol_arch, double* part, double* out,
                                  cudaStream_t st) {
  const uint64_t M = g.n_chains * g.N;
  uint64_t nb = (M + 255) / 256;
  if (nb > OBS_BLOCKS) nb = OBS_BLOCKS;
  topology_bonds_kernel<<<(unsigned)nb, 256, 0, st>>>(g, x, y, z, words, start, mol_arch, part);
  topology_bonds_final_kernel<<<1, 32, 0, st>>>(part, (int)nb, out);
  return cudaGetLastError();
}

}  // namespace soma
