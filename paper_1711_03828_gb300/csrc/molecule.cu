// molecule.cu -- the molecule-parallel iteration (Sec. 3.1.2, first scheme).
//
// One thread per chain: the chain's N attempts of one MC step run one after
// another, each on a particle of the chain chosen at random, so every particle
// is attempted once per step on average and a move always sees the current
// positions of its bonded partners.  Attempt j of chain k draws Philox purpose
// 3 with id k*N + j: words 0-2 give the uniform displacement, the top 24 bits
// of word 3 the acceptance uniform and its low byte the particle,
// ((word3 & 0xFF) * N) >> 8.  A block stages its 128 chains in shared memory
// (coalesced in and out) when they fit (N <= 64), then counts the final cells
// while writing them back.  Molecules of any architecture (the architecture
// array of Sec. 3.2.1, re-encoded per particle as for the SET kernel of
// topology.cu) take the same body with their bond partners and types from
// the per-particle table words.
#include "kernels.h"

namespace soma {

constexpr uint32_t PURPOSE_ATTEMPT = 3;

// Table word of the architecture path (see topology.cu): bits 0-5 number of
// partners, 6-23 the first three partners, bit 24 type.
__device__ __forceinline__ uint32_t mol_partner(uint32_t w, int k) { return (w >> (6 + 6 * k)) & 63u; }

// TOPO: molecules of any architecture (t holds the tables); else linear chains
// (the diblock, or a mixture through p.seq / p.arch).
// MULTI (with TOPO): n_t particle types, the type from the type table, one
// FP32 field plane and one count plane per type.
template <typename WT, bool STAGE, bool TOPO, bool MULTI = false>
__device__ __forceinline__ void molecule_body(const SweepArgs& p, const TopoArgs& tp) {
  extern __shared__ float sm[];
  const uint32_t N = p.g.N, N_A = p.g.N_A;
  const uint32_t t = threadIdx.x;
  const unsigned long long s64 = *p.d_sweep;
  const uint32_t sweep = (uint32_t)s64;
  uint32_t* __restrict__ nacc = MULTI ? (((s64 + 1ull) & 1ull) ? tp.nt1 : tp.nt0)
                                      : (((s64 + 1ull) & 1ull) ? p.n1 : p.n0);
  const uint32_t ctr3 = (PURPOSE_ATTEMPT << 24) | (p.g.replica & 0xFFFFFFu);
  const WT* __restrict__ wA = static_cast<const WT*>(p.wA);
  const WT* __restrict__ wB = static_cast<const WT*>(p.wB);
  const float a = p.a, K1 = p.K_b, K2 = 2.f * p.K_b;
  const uint64_t n_blocks = (p.g.n_chains + MOL_BLOCK - 1) / MOL_BLOCK;
  unsigned my_acc = 0;
  for (uint64_t cb = blockIdx.x; cb < n_blocks; cb += gridDim.x) {
    const uint64_t chain0 = cb * MOL_BLOCK;
    const uint64_t rem = p.g.n_chains - chain0;
    const uint32_t nch = rem < (uint64_t)MOL_BLOCK ? (uint32_t)rem : (uint32_t)MOL_BLOCK;
    const uint32_t cnt = nch * N;       // particles of this block
    const uint64_t m0 = chain0 * N;
    float* sx = sm;
    float* sy = sm + MOL_BLOCK * N;
    float* sz = sm + 2 * MOL_BLOCK * N;
    if (STAGE) {
      for (uint32_t q = t; q < cnt; q += MOL_BLOCK) {
        sx[q] = __ldcs(p.x + m0 + q);
        sy[q] = __ldcs(p.y + m0 + q);
        sz[q] = __ldcs(p.z + m0 + q);
      }
      __syncthreads();
    }
    if (t < nch) {
      const uint64_t chain = chain0 + t;
      // type sequence of this chain (bit i set: particle i is B)
      const uint64_t seq = p.seq ? __ldg(p.seq + __ldg(p.arch + chain)) : 0ull;
      const uint32_t arch_k = TOPO ? (uint32_t)__ldg(tp.mol_arch + chain) : 0u;
      const uint32_t* tab = TOPO ? tp.ptab + arch_k * 64u : nullptr;
      // particles of the molecule: its architecture's (the slots past them
      // are absent), else N; it makes that many attempts on its own particles
      const uint32_t len = TOPO ? (uint32_t)__ldg(tp.alen + arch_k) : N;
      float* X = STAGE ? sx + t * N : p.x + chain * N;
      float* Y = STAGE ? sy + t * N : p.y + chain * N;
      float* Z = STAGE ? sz + t * N : p.z + chain * N;
      // linear chains: the next attempt's draw (independent of this attempt's
      // outcome) is computed while this attempt's field gathers are in flight;
      // for architectures that measured slower (more registers in the longer
      // partner loop), so they draw in turn
      const uint64_t id0 = chain * N + p.g.id_base;
      uint4 rnext = make_uint4(0u, 0u, 0u, 0u);
      if (!TOPO)
        rnext = philox_rk(make_uint4((uint32_t)id0, (uint32_t)(id0 >> 32), sweep, ctr3), p.g);
      for (uint32_t j = 0; j < len; ++j) {
        uint4 r;
        if (!TOPO) {
          r = rnext;
          const uint64_t idn = id0 + j + 1u;
          rnext = philox_rk(make_uint4((uint32_t)idn, (uint32_t)(idn >> 32), sweep, ctr3), p.g);
        } else {
          const uint64_t id = id0 + j;
          r = philox_rk(make_uint4((uint32_t)id, (uint32_t)(id >> 32), sweep, ctr3), p.g);
        }
        const uint32_t i = ((r.w & 0xFFu) * len) >> 8;
        const float xo = X[i], yo = Y[i], zo = Z[i];
        const float xn = __fmaf_rn(a, uniform_sym(r.x), xo);
        const float yn = __fmaf_rn(a, uniform_sym(r.y), yo);
        const float zn = __fmaf_rn(a, uniform_sym(r.z), zo);
        float dEf;
        if (MULTI) {
          const uint32_t ty = __ldg(tp.ttab + (uint32_t)__ldg(tp.mol_arch + chain) * 64u + i);
          const float* w = tp.wt + (size_t)ty * p.g.cells;
          dEf = __ldg(w + cell_of(p.g, xn, yn, zn)) - __ldg(w + cell_of(p.g, xo, yo, zo));
        } else {
          const bool isB = TOPO ? ((__ldg(tab + i) >> 24) & 1u) != 0
                                : (p.seq ? ((seq >> i) & 1ull) != 0 : i >= N_A);
          const WT* w = isB ? wB : wA;
          dEf = load_w<WT>(w, cell_of(p.g, xn, yn, zn)) - load_w<WT>(w, cell_of(p.g, xo, yo, zo));
        }
        // U = sum over bonded partners of (r - n), k partners
        float ux = 0.f, uy = 0.f, uz = 0.f, k = 0.f;
        if (TOPO) {
          const uint32_t pw = __ldg(tab + i);
          const uint32_t deg = pw & 63u;
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            if ((uint32_t)b < deg) {
              const uint32_t n = mol_partner(pw, b);
              ux += xo - X[n];
              uy += yo - Y[n];
              uz += zo - Z[n];
            }
          }
          if (deg > 3u) {   // the partners after the third, from the full mask
            uint64_t mk = __ldg(tp.pmask + (uint32_t)__ldg(tp.mol_arch + chain) * 64u + i);
            mk &= mk - 1ull;
            mk &= mk - 1ull;
            mk &= mk - 1ull;
            for (; mk; mk &= mk - 1ull) {
              const uint32_t n = (uint32_t)__ffsll((long long)mk) - 1u;
              ux += xo - X[n];
              uy += yo - Y[n];
              uz += zo - Z[n];
            }
          }
          k = (float)deg;
        } else {
          if (i > 0) { ux += xo - X[i - 1]; uy += yo - Y[i - 1]; uz += zo - Z[i - 1]; k += 1.f; }
          if (i + 1 < N) { ux += xo - X[i + 1]; uy += yo - Y[i + 1]; uz += zo - Z[i + 1]; k += 1.f; }
        }
        const float dx = xn - xo, dy = yn - yo, dz = zn - zo;
        const float du = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
        const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float dE = fmaf(k * K1, dd, fmaf(K2, du, dEf));
        if (dE <= -log_uniform_open(r.w)) {
          X[i] = xn;
          Y[i] = yn;
          Z[i] = zn;
          ++my_acc;
        }
      }
    }
    __syncthreads();
    // write back (staged) and count the final cells
    uint32_t ci = t % N;
    const uint32_t step = MOL_BLOCK % N;
    for (uint32_t q = t; q < cnt; q += MOL_BLOCK) {
      float x, y, z;
      if (STAGE) {
        x = sx[q]; y = sy[q]; z = sz[q];
        __stcs(p.x + m0 + q, x);
        __stcs(p.y + m0 + q, y);
        __stcs(p.z + m0 + q, z);
      } else {
        x = p.x[m0 + q]; y = p.y[m0 + q]; z = p.z[m0 + q];
      }
      if (TOPO && ci >= (uint32_t)__ldg(tp.alen + __ldg(tp.mol_arch + chain0 + q / N))) {
        // an absent slot: written back unchanged, not counted
      } else if (MULTI) {
        const uint32_t ty = __ldg(tp.ttab + (uint32_t)__ldg(tp.mol_arch + chain0 + q / N) * 64u + ci);
        atomicAdd(nacc + (size_t)ty * p.g.cells + cell_of(p.g, x, y, z), 1u);
      } else {
        bool isB;
        if (TOPO)
          isB = ((__ldg(tp.ptab + (uint32_t)__ldg(tp.mol_arch + chain0 + q / N) * 64u + ci) >> 24) &
                 1u) != 0;
        else
          isB = p.seq ? ((__ldg(p.seq + __ldg(p.arch + chain0 + q / N)) >> ci) & 1ull) != 0
                      : ci >= N_A;
        atomicAdd(nacc + cell_of(p.g, x, y, z), isB ? 0x10000u : 1u);
      }
      ci += step;
      if (ci >= N) ci -= N;
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_acc += __shfl_xor_sync(FULL, my_acc, o);
  if ((t & 31u) == 0 && my_acc) atomicAdd(p.acc, (unsigned long long)my_acc);
}

template <typename WT, bool STAGE>
__global__ void __launch_bounds__(MOL_BLOCK) sweep_molecule_kernel(const SweepArgs p) {
  molecule_body<WT, STAGE, false>(p, TopoArgs{});
}

template <typename WT, bool MULTI>
__global__ void __launch_bounds__(MOL_BLOCK) sweep_molecule_topology_kernel(const TopoArgs t) {
  molecule_body<WT, true, true, MULTI>(t.s, t);
}

static const void* molecule_topology_ptr(int grid_dtype, bool types = false) {
  if (types) return (const void*)sweep_molecule_topology_kernel<float, true>;   // FP32 fields
  switch (grid_dtype) {
    case 1: return (const void*)sweep_molecule_topology_kernel<__nv_bfloat16, false>;
    case 2: return (const void*)sweep_molecule_topology_kernel<__half, false>;
    default: return (const void*)sweep_molecule_topology_kernel<float, false>;
  }
}

int molecule_topology_grid(uint32_t N, int grid_dtype, int sm_count, uint64_t n_chains) {
  const void* fn = molecule_topology_ptr(grid_dtype);
  const size_t smem = (size_t)3 * MOL_BLOCK * N * sizeof(float);
  if (smem > 48 * 1024) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(molecule_topology_ptr(0, true), cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, MOL_BLOCK, smem);
  if (per_sm < 1) per_sm = 1;
  const uint64_t need = (n_chains + MOL_BLOCK - 1) / MOL_BLOCK;
  const uint64_t cap = (uint64_t)sm_count * (uint64_t)per_sm;
  return (int)(need < cap ? need : cap);
}

cudaError_t launch_molecule_topology(const TopoArgs& a, int grid, int grid_dtype, cudaStream_t st,
                                     bool types) {
  void* args[] = {const_cast<TopoArgs*>(&a)};
  const size_t smem = (size_t)3 * MOL_BLOCK * a.s.g.N * sizeof(float);
  return cudaLaunchKernel(molecule_topology_ptr(grid_dtype, types), dim3(grid), dim3(MOL_BLOCK),
                          args, smem, st);
}

template <bool STAGE>
static const void* pick_molecule(int grid_dtype) {
  switch (grid_dtype) {
    case 1: return (const void*)sweep_molecule_kernel<__nv_bfloat16, STAGE>;
    case 2: return (const void*)sweep_molecule_kernel<__half, STAGE>;
    default: return (const void*)sweep_molecule_kernel<float, STAGE>;
  }
}

const void* molecule_kernel_ptr(uint32_t N, int grid_dtype, size_t* smem, bool prepare) {
  const bool stage = N <= 64;
  *smem = stage ? (size_t)3 * MOL_BLOCK * N * sizeof(float) : 0;
  const void* fn = stage ? pick_molecule<true>(grid_dtype) : pick_molecule<false>(grid_dtype);
  if (prepare && *smem > 48 * 1024)
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
  return fn;
}

}  // namespace soma
