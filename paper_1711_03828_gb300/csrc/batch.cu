// batch.cu -- many independent SCMF systems advanced by one sweep launch and
// one field launch per cycle.
//
// The paper tunes one parallel region at a time and runs one system per MPI
// rank (Sec. 3.1, 3.2.2).  Here a batch of independent systems (different
// sizes, chain lengths, compositions, chiN, replicas of one seed) shares a
// single persistent launch: the tiles of all systems are cut into work items
// of contiguous tiles of one system; block j takes items j, j + grid, ... and
// its warps walk an item's tiles with the same tile body as the single-system
// kernel (pair_body.cuh), so every system evolves bit-identically to the same
// system run alone.  The host lays the items out either as fixed-length items
// of each system in turn or as one equal contiguous range of the concatenated
// tiles per block, cut at system boundaries (piece r of block j at item
// r * grid + j, padded with empty items).  Launch shape (block size, blocks
// per SM, split) is picked by an autotuner that times the candidates during
// the run.
#include "kernels.h"
#include "pair_body.cuh"

namespace soma {

template <typename WT>
__global__ void __launch_bounds__(256, 3) sweep_batch_kernel(const BatchArgs p) {
  const int lane = threadIdx.x & 31;
  const uint32_t warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const unsigned long long s64 = *p.d_sweep;
  const uint32_t sweep = (uint32_t)s64;
  const bool odd = ((s64 + 1ull) & 1ull) != 0;

  uint32_t cur = 0xFFFFFFFFu;
  BatchSys S;
  PairLane<WT> L;
  uint32_t* nacc = nullptr;
  uint32_t ctr3 = 0, TN = 0;
  unsigned my_acc = 0;

  for (uint32_t item = blockIdx.x; item < p.n_items; item += gridDim.x) {
    const BatchItem it = p.items[item];
    if (it.sys != cur) {
      if (cur != 0xFFFFFFFFu) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_acc += __shfl_xor_sync(FULL, my_acc, o);
        if (lane == 0 && my_acc) atomicAdd(S.counters + 1, (unsigned long long)my_acc);
        my_acc = 0;
      }
      cur = it.sys;
      S = p.sys[cur];
      L.init(lane, S.g.N, S.g.N_A, S.wA, S.wB);
      nacc = odd ? S.n1 : S.n0;
      ctr3 = (PURPOSE_MOVE << 24) | (S.g.replica & 0xFFFFFFu);
      TN = S.G * S.g.N;
    }
    auto lane_ok = [&](uint32_t t) { return t < S.full_tiles || L.li0 < S.last_rows; };
    const uint32_t t0 = it.t0 + warp;
    float2 px = make_float2(0.f, 0.f), py = px, pz = px;
    if (t0 < it.t1 && lane_ok(t0)) {
      const uint32_t b0 = t0 * TN + L.li0;
      px = __ldcs(reinterpret_cast<const float2*>(S.x + b0));
      py = __ldcs(reinterpret_cast<const float2*>(S.y + b0));
      pz = __ldcs(reinterpret_cast<const float2*>(S.z + b0));
    }
    for (uint32_t tile = t0; tile < it.t1; tile += nwarps) {
      const bool valid = lane_ok(tile);
      const uint32_t base = tile * TN + L.li0;
      const float x0 = px.x, x1 = px.y, y0 = py.x, y1 = py.y, z0 = pz.x, z1 = pz.y;
      const uint32_t nt = tile + nwarps;
      if (nt < it.t1 && lane_ok(nt)) {
        const uint32_t bn = nt * TN + L.li0;
        px = __ldcs(reinterpret_cast<const float2*>(S.x + bn));
        py = __ldcs(reinterpret_cast<const float2*>(S.y + bn));
        pz = __ldcs(reinterpret_cast<const float2*>(S.z + bn));
      }
      if (tile < S.full_tiles)
        my_acc += pair_tile<WT, uint32_t, false, false>(S.g, p.keys, L, S.x, S.y, S.z, nacc, base, base,
                                                 true, sweep, ctr3, S.set_order_random, S.a, S.K_b, x0,
                                                 x1, y0, y1, z0, z1);
      else
        my_acc += pair_tile<WT, uint32_t, true, false>(S.g, p.keys, L, S.x, S.y, S.z, nacc, base, base,
                                                valid, sweep, ctr3, S.set_order_random, S.a, S.K_b, x0,
                                                x1, y0, y1, z0, z1);
    }
  }
  if (cur != 0xFFFFFFFFu) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_acc += __shfl_xor_sync(FULL, my_acc, o);
    if (lane == 0 && my_acc) atomicAdd(S.counters + 1, (unsigned long long)my_acc);
  }
}

// Field update of every system: one thread per cell of the concatenated grids;
// the system of a cell is found by binary search over the grid offsets held in
// shared memory.  The last block to finish advances every system's counter.
template <typename WT>
__global__ void __launch_bounds__(256) fields_batch_kernel(const BatchArgs p, uint32_t total_cells,
                                                           unsigned* arrive, unsigned* err) {
  extern __shared__ uint32_t cell_begin[];  // n_sys + 1 entries
  for (uint32_t k = threadIdx.x; k <= p.n_sys; k += blockDim.x)
    cell_begin[k] = k < p.n_sys ? p.sys[k].cell_begin : total_cells;
  __syncthreads();
  const unsigned long long s = *p.d_sweep;
  const bool rd1 = ((s + 1ull) & 1ull) != 0;
  unsigned bad = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < total_cells; c += stride) {
    uint32_t lo = 0, hi = p.n_sys;  // cell_begin[lo] <= c < cell_begin[hi]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (cell_begin[mid] <= c) lo = mid; else hi = mid;
    }
    const BatchSys* S = p.sys + lo;
    const uint32_t local = c - cell_begin[lo];
    const uint32_t* nr = rd1 ? S->n1 : S->n0;
    uint32_t* nc = rd1 ? S->n0 : S->n1;
    const uint32_t v = nr[local];
    nc[local] = 0u;
    const uint32_t a = v & 0xFFFFu, b = v >> 16;
    const float phiA = (float)a * S->inv_rho;
    const float phiB = (float)b * S->inv_rho;
    const float comp = S->kappa0 * (phiA + phiB - 1.f);
    float wa, wb;
    if (S->hamiltonian) {
      wa = fmaf(2.f * S->half_chi0, phiB, comp);
      wb = fmaf(2.f * S->half_chi0, phiA, comp);
    } else {
      const float d = S->half_chi0 * (phiA - phiB);
      wa = comp - d;
      wb = comp + d;
    }
    static_cast<WT*>(const_cast<void*>(S->wA))[local] = store_cvt<WT>(wa);
    static_cast<WT*>(const_cast<void*>(S->wB))[local] = store_cvt<WT>(wb);
    bad |= (a >= 0xC000u) | (b >= 0xC000u);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, ERR_OVERFLOW);
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(arrive, 1u);
    if (done == gridDim.x - 1) {
      *arrive = 0u;
      for (uint32_t k = 0; k < p.n_sys; ++k) p.sys[k].counters[0] = s + 1ull;
    }
  }
}

cudaError_t launch_sweep_batch(const BatchArgs& a, int grid, int block, int grid_dtype,
                               cudaStream_t st) {
  switch (grid_dtype) {
    case 1: sweep_batch_kernel<__nv_bfloat16><<<grid, block, 0, st>>>(a); break;
    case 2: sweep_batch_kernel<__half><<<grid, block, 0, st>>>(a); break;
    default: sweep_batch_kernel<float><<<grid, block, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_fields_batch(const BatchArgs& a, uint32_t total_cells, unsigned* arrive,
                                unsigned* err, int grid_dtype, int sm_count, cudaStream_t st) {
  uint64_t blocks = ((uint64_t)total_cells + 255) / 256;
  const uint64_t cap = (uint64_t)sm_count * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  const size_t sh = sizeof(uint32_t) * (a.n_sys + 1);
  switch (grid_dtype) {
    case 1: fields_batch_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, sh, st>>>(a, total_cells, arrive, err); break;
    case 2: fields_batch_kernel<__half><<<(unsigned)blocks, 256, sh, st>>>(a, total_cells, arrive, err); break;
    default: fields_batch_kernel<float><<<(unsigned)blocks, 256, sh, st>>>(a, total_cells, arrive, err); break;
  }
  return cudaGetLastError();
}

int batch_kernel_blocks_per_sm(int block, int grid_dtype) {
  const void* fn = grid_dtype == 1 ? (const void*)sweep_batch_kernel<__nv_bfloat16>
                 : grid_dtype == 2 ? (const void*)sweep_batch_kernel<__half>
                                   : (const void*)sweep_batch_kernel<float>;
  cudaFuncAttributes attr;
  if (cudaFuncGetAttributes(&attr, fn) != cudaSuccess || block > attr.maxThreadsPerBlock) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, 0) != cudaSuccess) return 0;
  return n;
}

}  // namespace soma
