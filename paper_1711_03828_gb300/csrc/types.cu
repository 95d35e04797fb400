// types.cu -- n_t particle types (arXiv:1711.03828, Sec. 2.1: Eq.
// density-characteristics, hamil-comp, hamil-pair and omega-fields for n_t
// types): occupation numbers per type, the field update and the non-bonded
// energy.
//
// With n_t types (2..8, set by soma_set_types; the particle types are the type
// bytes of the architecture array) the occupation numbers are one 32-bit plane
// per type, double buffered like the packed A | B grid of the two-type path:
// the sweep of step s counts into planes (s+1)&1 while the fields of planes s&1
// are in use.  The fields per cell, in FP32:
//   K^0: omega_i = kappa_0 (sum_k phi_k - 1) - sum_{k != i} chi_0ik/2 (phi_i - phi_k)
//   K^1: omega_i = kappa_0 (sum_k phi_k - 1) + sum_{k != i} chi_0ik phi_k
// with chi_0ik = chi_ik N / N and every pair of types counted once in the
// energy (as for two types).
#include "kernels.h"

namespace soma {

namespace {

// One thread per cell: reads the planes being read, clears the planes the
// next sweep counts into, writes every type's field; after a sweep the last
// block to finish advances the device sweep counter (as fields_kernel does).
__global__ void __launch_bounds__(256) fields_types_kernel(const TypesArgs p, unsigned* arrive) {
  const unsigned long long s = *p.d_sweep;
  const int rd = p.after_sweep ? (int)((s + 1ull) & 1ull) : (int)(s & 1ull);
  const uint32_t* __restrict__ nr = rd ? p.n1 : p.n0;
  uint32_t* __restrict__ nc = rd ? p.n0 : p.n1;
  const uint32_t cells = p.g.cells, T = p.n_types;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += stride) {
    float phi[TYPES_MAX];
    float total = 0.f;
#pragma unroll
    for (uint32_t t = 0; t < TYPES_MAX; ++t) {
      phi[t] = 0.f;
      if (t < T) {
        phi[t] = (float)nr[(size_t)t * cells + c] * p.inv_rho;
        nc[(size_t)t * cells + c] = 0u;
        total += phi[t];
      }
    }
    const float comp = p.kappa0 * (total - 1.f);
#pragma unroll
    for (uint32_t i = 0; i < TYPES_MAX; ++i) {
      if (i >= T) break;
      float v = comp;
#pragma unroll
      for (uint32_t k = 0; k < TYPES_MAX; ++k) {
        if (k >= T || k == i) continue;
        const float chi0 = p.chi0[i * TYPES_MAX + k];
        v = p.hamiltonian ? fmaf(chi0, phi[k], v) : fmaf(-0.5f * chi0, phi[i] - phi[k], v);
      }
      p.w[(size_t)i * cells + c] = v;
    }
  }
  if (p.after_sweep) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned done = atomicAdd(arrive, 1u);
      if (done == gridDim.x - 1) {
        *arrive = 0u;
        *p.d_sweep = s + 1ull;
      }
    }
  }
}

// Occupation numbers per type of the current positions (types from the
// architecture table of each molecule).
__global__ void __launch_bounds__(256) histogram_types_kernel(
    const Geom g, const float* __restrict__ x, const float* __restrict__ y,
    const float* __restrict__ z, const uint8_t* __restrict__ ttab,
    const uint8_t* __restrict__ mol_arch, uint32_t* __restrict__ n) {
  const uint64_t M = g.n_chains * g.N;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += stride) {
    const uint64_t mol = m / g.N;
    const uint32_t i = (uint32_t)(m - mol * g.N);
    const uint32_t t = __ldg(ttab + (uint32_t)__ldg(mol_arch + mol) * 64u + i);
    if (t == 0xFFu) continue;   // an absent slot
    atomicAdd(n + (size_t)t * g.cells + cell_of(g, x[m], y[m], z[m]), 1u);
  }
}

// Per block: the sum over cells of the energy per cell (without rho dL^3/N)
// and the largest total count, FP64.
__global__ void __launch_bounds__(256) obs_types_kernel(const TypesArgs p, double kappaN,
                                                        const uint32_t* __restrict__ n,
                                                        double* __restrict__ part) {
  __shared__ double sk[32], sm[32];
  const uint32_t cells = p.g.cells, T = p.n_types;
  const double inv_rho = p.inv_rho_f64;
  double K = 0.0, mx = 0.0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += stride) {
    double phi[TYPES_MAX], total = 0.0, cnt = 0.0;
    for (uint32_t t = 0; t < T; ++t) {
      const double v = (double)n[(size_t)t * cells + c];
      cnt += v;
      phi[t] = v * inv_rho;
      total += phi[t];
    }
    const double fl = total - 1.0;
    double k = 0.5 * kappaN * fl * fl;
    for (uint32_t i = 0; i < T; ++i)
      for (uint32_t j = i + 1; j < T; ++j) {
        const double chi = p.chiN[i * TYPES_MAX + j];
        k += p.hamiltonian ? chi * phi[i] * phi[j]
                           : -0.25 * chi * (phi[i] - phi[j]) * (phi[i] - phi[j]);
      }
    K += k;
    mx = fmax(mx, cnt);
  }
  for (int o = 16; o > 0; o >>= 1) {
    K += __shfl_xor_sync(FULL, K, o);
    mx = fmax(mx, __shfl_xor_sync(FULL, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    sk[threadIdx.x >> 5] = K;
    sm[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += sk[w];
      b = fmax(b, sm[w]);
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

__global__ void obs_types_final_kernel(const double* __restrict__ part, int nb,
                                       double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < nb; ++k) {
    a += part[2 * k];
    b = fmax(b, part[2 * k + 1]);
  }
  out[2] = a;
  out[3] = b;
  out[4] = 0.0;
}

// Packs the counts of types i and j into one grid, n_i | n_j << 16, for the
// composition structure factor; a count that does not fit 16 bits sets the
// overflow bit of the error word.
__global__ void __launch_bounds__(256) pack_pair_kernel(const uint32_t* __restrict__ n,
                                                        uint32_t cells, uint32_t ti, uint32_t tj,
                                                        uint32_t* __restrict__ out,
                                                        unsigned* __restrict__ err) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += stride) {
    const uint32_t a = n[(size_t)ti * cells + c], b = n[(size_t)tj * cells + c];
    if ((a | b) >> 16) atomicOr(err, ERR_OVERFLOW);
    out[c] = (a & 0xFFFFu) | (b << 16);
  }
}

}  // namespace

cudaError_t launch_pack_type_pair(const uint32_t* n, uint32_t cells, uint32_t ti, uint32_t tj,
                                  uint32_t* out, unsigned* err, int sm_count, cudaStream_t st) {
  uint64_t blocks = ((uint64_t)cells + 255) / 256;
  const uint64_t cap = (uint64_t)sm_count * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  pack_pair_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, cells, ti, tj, out, err);
  return cudaGetLastError();
}

cudaError_t launch_fields_types(const TypesArgs& a, unsigned* arrive, int sm_count,
                                cudaStream_t st) {
  uint64_t blocks = ((uint64_t)a.g.cells + 255) / 256;
  const uint64_t cap = (uint64_t)sm_count * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  fields_types_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, arrive);
  return cudaGetLastError();
}

cudaError_t launch_histogram_types(const Geom& g, const float* x, const float* y, const float* z,
                                   const uint8_t* ttab, const uint8_t* mol_arch, uint32_t* n,
                                   int sm_count, cudaStream_t st) {
  const uint64_t M = g.n_chains * g.N;
  uint64_t blocks = (M + 255) / 256;
  const uint64_t cap = (uint64_t)sm_count * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  histogram_types_kernel<<<(unsigned)blocks, 256, 0, st>>>(g, x, y, z, ttab, mol_arch, n);
  return cudaGetLastError();
}

cudaError_t launch_observables_types(const TypesArgs& a, double kappaN, const uint32_t* n,
                                     double* part, double* out, cudaStream_t st) {
  uint64_t nb = ((uint64_t)a.g.cells + 255) / 256;
  if (nb > OBS_BLOCKS) nb = OBS_BLOCKS;
  obs_types_kernel<<<(unsigned)nb, 256, 0, st>>>(a, kappaN, n, part);
  obs_types_final_kernel<<<1, 32, 0, st>>>(part, (int)nb, out);
  return cudaGetLastError();
}

}  // namespace soma
