// sweep.cu -- the Monte-Carlo step of the SCMF cycle (arXiv:1711.03828,
// Sec. 2.2 and the SET iteration of Sec. 3.1.2) on sm_103a.
//
// Work decomposition.  A 32-lane warp owns a tile of G whole chains laid out
// contiguously (G*N <= 64Q particles).  Lane l holds the 2Q consecutive
// particles 2Ql .. 2Ql+2Q-1 of the tile in registers, so each lane owns as
// many even as odd chain positions and BOTH independent sets keep all lanes
// busy (the paper's SET scheme leaves half its threads idle per set for a
// linear chain).  Bond partners in a neighbouring lane are exchanged with
// warp shuffles; no shared memory and no inter-warp synchronisation.
//
// Per particle: one Philox4x32-10 draw (counter = particle, sweep) gives the
// three displacement uniforms and the acceptance uniform; the set order of a
// chain is bit 0 of the acceptance word of its first particle.  The trial
// position r + a v is rounded once to the stored FP32 precision (a fused
// multiply-add, round-to-nearest).  The two field values omega_t(c) and
// omega_t(c') are gathered from the L2-resident omega planes before the set
// loop since c' does not depend on the neighbours.  After both sets the final
// cells are added to the packed occupation grid n[(s+1)&1] with 32-bit
// atomics (the occupation count of the next field update, fused).
//
// Streams: positions are loaded and stored with evict-first hints so the
// 28 MB grid and the omega planes stay in L2.
#include "kernels.h"
#include "pair_body.cuh"

namespace soma {

template <int S>
__device__ __forceinline__ void load_slots(const float* __restrict__ p, float (&v)[S]) {
  if constexpr (S == 2) {
    const float2 t = __ldcs(reinterpret_cast<const float2*>(p));
    v[0] = t.x;
    v[1] = t.y;
  } else {
#pragma unroll
    for (int k = 0; k < S / 4; ++k) {
      const float4 t = __ldcs(reinterpret_cast<const float4*>(p) + k);
      v[4 * k] = t.x;
      v[4 * k + 1] = t.y;
      v[4 * k + 2] = t.z;
      v[4 * k + 3] = t.w;
    }
  }
}

template <int S>
__device__ __forceinline__ void store_slots(float* __restrict__ p, const float (&v)[S]) {
  if constexpr (S == 2) {
    __stcs(reinterpret_cast<float2*>(p), make_float2(v[0], v[1]));
  } else {
#pragma unroll
    for (int k = 0; k < S / 4; ++k)
      __stcs(reinterpret_cast<float4*>(p) + k,
             make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
  }
}

__device__ __forceinline__ float dist2(float ax, float ay, float az, float bx, float by, float bz) {
  const float dx = ax - bx, dy = ay - by, dz = az - bz;
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

template <int Q, bool VEC, typename WT>
__global__ void __launch_bounds__(256) sweep_uniform_kernel(const SweepArgs p) {
  constexpr int S = 2 * Q;
  const int lane = threadIdx.x & 31;
  const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned long long s64 = *p.d_sweep;
  const uint32_t sweep = (uint32_t)s64;
  uint32_t* __restrict__ nacc = ((s64 + 1ull) & 1ull) ? p.n1 : p.n0;
  const WT* __restrict__ wA = static_cast<const WT*>(p.wA);
  const WT* __restrict__ wB = static_cast<const WT*>(p.wB);
  const uint32_t N = p.g.N, N_A = p.g.N_A;
  const uint32_t ctr3 = (PURPOSE_MOVE << 24) | (p.g.replica & 0xFFFFFFu);
  const uint32_t li0 = (uint32_t)lane * S;

  // Tile-invariant slot metadata: chain-local index, chain within the tile,
  // and (lane, slot) of that chain's first particle.
  uint32_t ci[S], src_lane[S], src_slot[S];
  {
    uint32_t g = li0 / N, i = li0 - g * N;
#pragma unroll
    for (int j = 0; j < S; ++j) {
      ci[j] = i;
      const uint32_t first = g * N;
      src_lane[j] = (first / S) & 31u;
      src_slot[j] = first % S;
      if (++i == N) { i = 0; ++g; }
    }
  }

  unsigned my_acc = 0;
  for (uint64_t tile = warp0; tile < p.n_tiles; tile += nwarps) {
    const uint64_t chain0 = tile * p.G;
    const uint64_t rem = p.g.n_chains - chain0;
    const uint32_t nmono = (rem < p.G ? (uint32_t)rem : p.G) * N;
    const uint64_t base = chain0 * N + li0;
    const bool full = li0 + S <= nmono;

    float x[S], y[S], z[S];
    if (VEC && full) {
      load_slots<S>(p.x + base, x);
      load_slots<S>(p.y + base, y);
      load_slots<S>(p.z + base, z);
    } else {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const bool ok = li0 + j < nmono;
        x[j] = ok ? __ldcs(p.x + base + j) : 0.f;
        y[j] = ok ? __ldcs(p.y + base + j) : 0.f;
        z[j] = ok ? __ldcs(p.z + base + j) : 0.f;
      }
    }

    // Draws, trial positions, cells and the field change of every slot.
    float xn[S], yn[S], zn[S], lnu[S], dEf[S];
    uint32_t co[S], cn[S];
    uint32_t lowbits = 0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const uint64_t m = base + j + p.g.id_base;
      const uint4 r = philox_rk(make_uint4((uint32_t)m, (uint32_t)(m >> 32), sweep, ctr3), p.g);
      xn[j] = __fmaf_rn(p.a, uniform_sym(r.x), x[j]);
      yn[j] = __fmaf_rn(p.a, uniform_sym(r.y), y[j]);
      zn[j] = __fmaf_rn(p.a, uniform_sym(r.z), z[j]);
      lnu[j] = log_uniform_open(r.w);
      lowbits |= (r.w & 1u) << j;
      co[j] = cell_of(p.g, x[j], y[j], z[j]);
      cn[j] = cell_of(p.g, xn[j], yn[j], zn[j]);
      const WT* wt = (ci[j] < N_A) ? wA : wB;
      dEf[j] = (li0 + j < nmono) ? load_w<WT>(wt, cn[j]) - load_w<WT>(wt, co[j]) : 0.f;
    }

    // Set of each slot in this sweep: 0 moves first.
    uint32_t phase[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      uint32_t b = 0;
      if (p.set_order_random) b = (__shfl_sync(FULL, lowbits, src_lane[j]) >> src_slot[j]) & 1u;
      phase[j] = (ci[j] & 1u) ^ b;
    }

#pragma unroll
    for (uint32_t ph = 0; ph < 2; ++ph) {
      const float pxl = __shfl_up_sync(FULL, x[S - 1], 1);
      const float pyl = __shfl_up_sync(FULL, y[S - 1], 1);
      const float pzl = __shfl_up_sync(FULL, z[S - 1], 1);
      const float nxl = __shfl_down_sync(FULL, x[0], 1);
      const float nyl = __shfl_down_sync(FULL, y[0], 1);
      const float nzl = __shfl_down_sync(FULL, z[0], 1);
#pragma unroll
      for (int j = 0; j < S; ++j) {
        if (li0 + j >= nmono || phase[j] != ph) continue;
        const float qx = (j > 0) ? x[j - 1] : pxl;
        const float qy = (j > 0) ? y[j - 1] : pyl;
        const float qz = (j > 0) ? z[j - 1] : pzl;
        const float rx = (j < S - 1) ? x[j + 1] : nxl;
        const float ry = (j < S - 1) ? y[j + 1] : nyl;
        const float rz = (j < S - 1) ? z[j + 1] : nzl;
        float e = 0.f;
        if (ci[j] > 0)
          e += dist2(xn[j], yn[j], zn[j], qx, qy, qz) - dist2(x[j], y[j], z[j], qx, qy, qz);
        if (ci[j] + 1 < N)
          e += dist2(xn[j], yn[j], zn[j], rx, ry, rz) - dist2(x[j], y[j], z[j], rx, ry, rz);
        const float dE = fmaf(p.K_b, e, dEf[j]);
        if (dE <= 0.f || lnu[j] < -dE) {
          x[j] = xn[j];
          y[j] = yn[j];
          z[j] = zn[j];
          co[j] = cn[j];
          ++my_acc;
        }
      }
    }

    if (VEC && full) {
      store_slots<S>(p.x + base, x);
      store_slots<S>(p.y + base, y);
      store_slots<S>(p.z + base, z);
    } else {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        if (li0 + j < nmono) {
          __stcs(p.x + base + j, x[j]);
          __stcs(p.y + base + j, y[j]);
          __stcs(p.z + base + j, z[j]);
        }
      }
    }

    // Occupation count of the final cells; consecutive slots in one cell are
    // merged into a single atomic (A adds 1, B adds 1<<16).
    uint32_t carry = 0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if (li0 + j >= nmono) continue;
      const uint32_t v = carry + ((ci[j] < N_A) ? 1u : 0x10000u);
      if (j + 1 < S && li0 + j + 1 < nmono && co[j + 1] == co[j]) {
        carry = v;
      } else {
        atomicAdd(nacc + co[j], v);
        carry = 0;
      }
    }
  }

#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_acc += __shfl_xor_sync(FULL, my_acc, o);
  if (lane == 0 && my_acc) atomicAdd(p.acc, (unsigned long long)my_acc);
}

// Even N <= 64: the paired tile body of pair_body.cuh over one system.  One
// block of 24 warps per SM owns a contiguous range of tiles (spatially
// ordered chains); its warps take the range's tiles in order from a
// shared-memory counter, so they work on neighbouring tiles (field values
// repeat in L1) and all finish within a tile of each other.  With three
// blocks of a third of the range each, the warp scheduler's preference for
// the oldest warps finished the first block well before the third, and the
// SM ran its last sixth at a third or two thirds of its warps.  The next
// tile's positions are loaded while the current one is processed.  IDX is the
// index type: 32-bit when M < 2^32 (Philox counter word 1 = 0).
// MIXED: a mixture of linear architectures (the type sequence of each chain
// is read per tile); otherwise every chain is the diblock of N_A A particles.
template <typename WT, typename IDX, bool MIXED>
__global__ void __launch_bounds__(768, 1) sweep_pair_kernel(const SweepArgs p) {
  __shared__ uint32_t s_next;
  const int lane = threadIdx.x & 31;
  const uint32_t n_tiles_all = (uint32_t)p.n_tiles;
  const uint32_t chunk = (n_tiles_all + gridDim.x - 1) / gridDim.x;
  const uint32_t t_begin = blockIdx.x * chunk;
  const uint32_t t_end = min(t_begin + chunk, n_tiles_all);
  if (threadIdx.x == 0) s_next = 0u;
  __syncthreads();
  auto claim = [&]() -> uint32_t {
    uint32_t t = 0u;
    if (lane == 0) t = atomicAdd(&s_next, 1u);
    return t_begin + __shfl_sync(FULL, t, 0);
  };
  const unsigned long long s64 = *p.d_sweep;
  const uint32_t sweep = (uint32_t)s64;
  uint32_t* __restrict__ nacc = ((s64 + 1ull) & 1ull) ? p.n1 : p.n0;
  const uint32_t ctr3 = (PURPOSE_MOVE << 24) | (p.g.replica & 0xFFFFFFu);
  PairLane<WT> L;
  L.init(lane, p.g.N, p.g.N_A, p.wA, p.wB);
  const uint32_t TN = p.G * p.g.N;
  const uint32_t full_tiles = (uint32_t)p.full_tiles;
  auto lane_ok = [&](uint32_t t) { return t < full_tiles || L.li0 < p.last_rows; };
  const bool wide = p.g.nx > 1 && p.g.ny > 1 && p.g.nz > 1;

  float2 px = make_float2(0.f, 0.f), py = px, pz = px;
  auto load_pos = [&](uint32_t t) {
    if (t < t_end && lane_ok(t)) {
      const IDX b = (IDX)t * TN + L.li0;
      px = __ldcs(reinterpret_cast<const float2*>(p.x + b));
      py = __ldcs(reinterpret_cast<const float2*>(p.y + b));
      pz = __ldcs(reinterpret_cast<const float2*>(p.z + b));
    }
  };
  uint32_t tile = claim();
  load_pos(tile);
  unsigned my_acc = 0;
  while (tile < t_end) {
    const bool valid = lane_ok(tile);
    const IDX base = (IDX)tile * TN + L.li0;
    const float x0 = px.x, x1 = px.y, y0 = py.x, y1 = py.y, z0 = pz.x, z1 = pz.y;
    const uint32_t next_tile = claim();
    load_pos(next_tile);
    PairLane<WT> Lt = L;
    if (MIXED) {
      const uint64_t chain = (uint64_t)tile * p.G + L.lane_chain;
      const uint64_t seq = chain < p.g.n_chains ? __ldg(p.seq + __ldg(p.arch + chain)) : 0ull;
      Lt.set_types((seq >> L.ci0) & 1ull, (seq >> (L.ci0 + 1u)) & 1ull, p.wA, p.wB);
    }
    const IDX cbase = base + (IDX)p.g.id_base;
    if (tile < full_tiles && wide)
      my_acc += pair_tile<WT, IDX, false, true>(p.g, p.g, Lt, p.x, p.y, p.z, nacc, base, cbase, true,
                                                sweep, ctr3, p.set_order_random, p.a, p.K_b, x0, x1,
                                                y0, y1, z0, z1);
    else if (tile < full_tiles)
      my_acc += pair_tile<WT, IDX, false, false>(p.g, p.g, Lt, p.x, p.y, p.z, nacc, base, cbase, true,
                                                 sweep, ctr3, p.set_order_random, p.a, p.K_b, x0,
                                                 x1, y0, y1, z0, z1);
    else
      my_acc += pair_tile<WT, IDX, true, false>(p.g, p.g, Lt, p.x, p.y, p.z, nacc, base, cbase, valid,
                                                sweep, ctr3, p.set_order_random, p.a, p.K_b, x0, x1,
                                                y0, y1, z0, z1);
    tile = next_tile;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_acc += __shfl_xor_sync(FULL, my_acc, o);
  if (lane == 0 && my_acc) atomicAdd(p.acc, (unsigned long long)my_acc);
}

template <int Q, bool VEC>
static const void* pick_kernel(int grid_dtype) {
  switch (grid_dtype) {
    case 1: return (const void*)sweep_uniform_kernel<Q, VEC, __nv_bfloat16>;
    case 2: return (const void*)sweep_uniform_kernel<Q, VEC, __half>;
    default: return (const void*)sweep_uniform_kernel<Q, VEC, float>;
  }
}

static const void* sweep_kernel_ptr(int Q, bool vec, int grid_dtype, bool pair, bool big,
                                    int move, bool mixed) {
  if (move == 1) return smc_kernel_ptr(Q, pair && !big, grid_dtype);
  if (move == 2) return learned_kernel_ptr(Q, grid_dtype);
  if (pair) {
    if (big) {
      switch (grid_dtype) {
        case 1: return (const void*)sweep_pair_kernel<__nv_bfloat16, uint64_t, false>;
        case 2: return (const void*)sweep_pair_kernel<__half, uint64_t, false>;
        default: return (const void*)sweep_pair_kernel<float, uint64_t, false>;
      }
    }
    if (mixed) {
      switch (grid_dtype) {
        case 1: return (const void*)sweep_pair_kernel<__nv_bfloat16, uint32_t, true>;
        case 2: return (const void*)sweep_pair_kernel<__half, uint32_t, true>;
        default: return (const void*)sweep_pair_kernel<float, uint32_t, true>;
      }
    }
    switch (grid_dtype) {
      case 1: return (const void*)sweep_pair_kernel<__nv_bfloat16, uint32_t, false>;
      case 2: return (const void*)sweep_pair_kernel<__half, uint32_t, false>;
      default: return (const void*)sweep_pair_kernel<float, uint32_t, false>;
    }
  }
  if (Q == 1) return vec ? pick_kernel<1, true>(grid_dtype) : pick_kernel<1, false>(grid_dtype);
  if (Q == 2) return vec ? pick_kernel<2, true>(grid_dtype) : pick_kernel<2, false>(grid_dtype);
  return vec ? pick_kernel<4, true>(grid_dtype) : pick_kernel<4, false>(grid_dtype);
}

SweepShape sweep_shape(uint64_t n_chains, uint32_t N, int sm_count, int grid_dtype, int move,
                       bool learned_fp32, bool learned_umma, bool molecule) {
  SweepShape s;
  s.move = move;
  s.learned_tc = false;
  s.learned_umma = false;
  s.molecule = false;
  s.smem = 0;
  s.Q = (N <= 64) ? 1 : (N <= 128 ? 2 : 4);
  s.G = (uint32_t)(64 * s.Q) / N;
  s.n_tiles = (n_chains + s.G - 1) / s.G;
  const uint32_t S = 2u * (uint32_t)s.Q;
  const uint32_t align = S < 4u ? S : 4u;
  s.vec = ((uint64_t)s.G * N) % align == 0;
  s.pair = (s.Q == 1) && (N % 2 == 0);
  s.big = n_chains * N >= (1ull << 32) || s.n_tiles >= (1ull << 31);
  // the paired uniform and smart Monte Carlo kernels: one block of 24 warps per SM
  s.block = ((move == 0 && s.pair) || (move == 1 && s.pair && !s.big)) ? 768 : 256;
  const void* fn = sweep_kernel_ptr(s.Q, s.vec, grid_dtype, s.pair, s.big, s.move, false);
  if (move == 2 && s.pair && !s.big && !learned_fp32) {
    s.learned_tc = true;
    s.learned_umma = learned_umma;
    s.block = 128;
    fn = learned_tc_kernel_ptr(grid_dtype, s.learned_umma);
  }
  if (molecule && move == 0) {
    s.molecule = true;
    s.block = MOL_BLOCK;
    fn = molecule_kernel_ptr(N, grid_dtype, &s.smem, true);
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, s.block, s.smem);
  if (per_sm < 1) per_sm = 1;
  const uint64_t warps_per_block = (uint64_t)s.block / 32;
  const uint64_t need = s.molecule ? (n_chains + s.block - 1) / s.block
                                   : (s.n_tiles + warps_per_block - 1) / warps_per_block;
  const uint64_t cap = (uint64_t)sm_count * (uint64_t)per_sm;
  s.grid = (int)(need < cap ? need : cap);
  if (s.grid < 1) s.grid = 1;
  return s;
}

cudaError_t launch_sweep_uniform(const SweepArgs& a, const SweepShape& s, int grid_dtype,
                                 cudaStream_t st) {
  size_t smem = 0;
  const void* fn = s.molecule ? molecule_kernel_ptr(a.g.N, grid_dtype, &smem, false)
                              : sweep_kernel_ptr(s.Q, s.vec, grid_dtype, s.pair, s.big, s.move,
                                                 a.seq != nullptr);
  void* args[] = {const_cast<SweepArgs*>(&a)};
  return cudaLaunchKernel(fn, dim3(s.grid), dim3(s.block), args, smem, st);
}

}  // namespace soma
