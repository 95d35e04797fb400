// grid.cu -- grid-side kernels of libsoma: the occupation count, the field
// update, the initial configuration and the FP64 observables.
//   - occupation numbers n_t(c): Eq. (density-characteristics), Sec. 3.1.1;
//   - fields omega_A/B: Eq. (omega-fields), option K^0;
//   - initial chains: Sec. 2.1 (Gaussian bonds, b0 = sqrt(3/k0));
//   - energies: Eq. (h-bond), (V-harmonic), (discrete-ham); S(q): Sec. 5.6.
#include "kernels.h"
#include "draws.cuh"

namespace soma {

// ---------------------------------------------------------------------------
// Occupation count of a whole configuration (used outside the sweep, whose
// epilogue counts on its own).  One thread per particle.
__global__ void histogram_kernel(const Geom g, const float* __restrict__ x,
                                 const float* __restrict__ y, const float* __restrict__ z,
                                 uint32_t* __restrict__ n, const uint64_t* __restrict__ seq,
                                 const uint8_t* __restrict__ arch,
                                 const uint8_t* __restrict__ alen) {
  const uint64_t M = g.n_chains * g.N;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += stride) {
    const uint64_t chain = m / g.N;
    const uint32_t i = (uint32_t)(m - chain * g.N);
    if (alen && i >= alen[arch[chain]]) continue;   // an absent slot
    const bool isB = seq ? ((seq[arch[chain]] >> i) & 1ull) != 0 : i >= g.N_A;
    atomicAdd(n + cell_of(g, x[m], y[m], z[m]), isB ? 0x10000u : 1u);
  }
}

cudaError_t launch_histogram(const Geom& g, const float* x, const float* y, const float* z,
                             uint32_t* n, int sm_count, cudaStream_t st, const uint64_t* seq,
                             const uint8_t* arch, const uint8_t* alen) {
  const uint64_t M = g.n_chains * g.N;
  uint64_t blocks = (M + 255) / 256;
  const uint64_t cap = (uint64_t)sm_count * 8;
  if (blocks > cap) blocks = cap;
  histogram_kernel<<<(unsigned)blocks, 256, 0, st>>>(g, x, y, z, n, seq, arch, alen);
  return cudaGetLastError();
}

// Range check of positions given by the caller: flag = 1 if any value is not
// finite or has |v| >= lim (the supported range of the cell fold).
// p starts 16-byte aligned (every position plane is 256-byte aligned): four
// coordinates per 16-byte load, the last n mod 4 one by one.
__global__ void __launch_bounds__(256) range_check_kernel(const float* __restrict__ p, uint64_t n,
                                                          float lim, unsigned* flag) {
  unsigned bad = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t n4 = n / 4;
  const float4* __restrict__ q = reinterpret_cast<const float4*>(p);
  for (uint64_t i = tid; i < n4; i += stride) {
    const float4 v = __ldg(q + i);
    bad |= !(fabsf(v.x) < lim) | !(fabsf(v.y) < lim) | !(fabsf(v.z) < lim) | !(fabsf(v.w) < lim);
  }
  for (uint64_t i = 4 * n4 + tid; i < n; i += stride) bad |= !(fabsf(p[i]) < lim);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1u);
}

cudaError_t launch_range_check(const float* p, uint64_t n, float lim, unsigned* flag, int sm_count,
                               cudaStream_t st) {
  uint64_t blocks = (n / 4 + 255) / 256;
  const uint64_t cap = (uint64_t)sm_count * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  range_check_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, n, lim, flag);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Field update: omega from the packed counts of one buffer, while the other
// buffer is cleared for the next sweep's count.  The last block to finish
// (arrival counter, no waiting) advances the sweep counter, so every block
// read the same counter value.
template <typename WT>
__global__ void __launch_bounds__(256) fields_kernel(const FieldArgs p, unsigned* arrive) {
  const unsigned long long s = *p.d_sweep;
  const int rd = p.after_sweep ? (int)((s + 1ull) & 1ull) : (int)(s & 1ull);
  const uint32_t* __restrict__ nr = rd ? p.n1 : p.n0;
  uint32_t* __restrict__ nc = rd ? p.n0 : p.n1;
  WT* __restrict__ wA = static_cast<WT*>(p.wA);
  WT* __restrict__ wB = static_cast<WT*>(p.wB);
  unsigned bad = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < p.g.cells; c += stride) {
    const uint32_t v = nr[c];
    nc[c] = 0u;
    const uint32_t a = v & 0xFFFFu, b = v >> 16;
    const float phiA = (float)a * p.inv_rho;
    const float phiB = (float)b * p.inv_rho;
    const float comp = p.kappa0 * (phiA + phiB - 1.f);
    float wa, wb;
    if (p.hamiltonian) {          // K^1: + chi_0 phi_k of the other type
      wa = fmaf(2.f * p.half_chi0, phiB, comp);
      wb = fmaf(2.f * p.half_chi0, phiA, comp);
    } else {                      // K^0: -/+ chi_0/2 (phi_A - phi_B)
      const float d = p.half_chi0 * (phiA - phiB);
      wa = comp - d;
      wb = comp + d;
    }
    if (p.ext) {
      wa += p.ext[c];
      wb += p.ext[p.g.cells + c];
    }
    if (p.forbidden && p.forbidden[c]) wa = wb = __int_as_float(0x7F800000);   // +inf
    wA[c] = store_cvt<WT>(wa);
    wB[c] = store_cvt<WT>(wb);
    bad |= (a >= 0xC000u) | (b >= 0xC000u);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(p.err, ERR_OVERFLOW);
  if (p.after_sweep && threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(arrive, 1u);
    if (done == gridDim.x - 1) {
      *arrive = 0u;
      *p.d_sweep = s + 1ull;
    }
  }
}

cudaError_t launch_fields(const FieldArgs& a, unsigned* arrive, int grid_dtype, int sm_count,
                          cudaStream_t st) {
  uint64_t blocks = ((uint64_t)a.g.cells + 255) / 256;
  const uint64_t cap = (uint64_t)sm_count * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  switch (grid_dtype) {
    case 1: fields_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, st>>>(a, arrive); break;
    case 2: fields_kernel<__half><<<(unsigned)blocks, 256, 0, st>>>(a, arrive); break;
    default: fields_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(a, arrive); break;
  }
  return cudaGetLastError();
}

template <typename WT>
__global__ void convert_kernel(const WT* __restrict__ w, float* __restrict__ dst, uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    dst[i] = load_w<WT>(w, (uint32_t)i);
}

cudaError_t launch_convert_fields(const void* w, int grid_dtype, float* dst, uint64_t n,
                                  cudaStream_t st) {
  const unsigned blocks = 1024;
  switch (grid_dtype) {
    case 1: convert_kernel<<<blocks, 256, 0, st>>>((const __nv_bfloat16*)w, dst, n); break;
    case 2: convert_kernel<<<blocks, 256, 0, st>>>((const __half*)w, dst, n); break;
    default: convert_kernel<<<blocks, 256, 0, st>>>((const float*)w, dst, n); break;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Initial configuration, one thread per chain, FP64 with explicit rounding
// (no contraction) so the arithmetic is the textbook one: first particle
// uniform in the box, then N-1 bond vectors with components sigma * z, z from
// the Box-Muller transform of two open uniforms.
__global__ void init_kernel(const Geom g, float* __restrict__ x, float* __restrict__ y,
                            float* __restrict__ z, double sigma) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint32_t ctr3 = (PURPOSE_INIT << 24) | (g.replica & 0xFFFFFFu);
  const double two_pi = 6.283185307179586;  // 2*pi rounded to FP64
  for (uint64_t chain = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; chain < g.n_chains;
       chain += stride) {
    const uint64_t gc = chain + g.chain_base;   // the chain's index in the whole system
    const uint32_t lo = (uint32_t)gc, hi = (uint32_t)(gc >> 32);
    uint4 w = philox4x32_10(make_uint4(lo, hi, 0u, ctr3), g.key0, g.key1);
    double r[3] = {__dmul_rn(uniform_open_f64(w.x), (double)g.nx),
                   __dmul_rn(uniform_open_f64(w.y), (double)g.ny),
                   __dmul_rn(uniform_open_f64(w.z), (double)g.nz)};
    const uint64_t m0 = chain * g.N;
    x[m0] = (float)r[0];
    y[m0] = (float)r[1];
    z[m0] = (float)r[2];
    uint32_t cached = 0xFFFFFFFFu;
    for (uint32_t i = 0; i + 1 < g.N; ++i) {
      for (int d = 0; d < 3; ++d) {
        const uint32_t j = 3u * i + (uint32_t)d;
        const uint32_t call = 1u + j / 4u;
        if (call != cached) {
          w = philox4x32_10(make_uint4(lo, hi, call, ctr3), g.key0, g.key1);
          cached = call;
        }
        const uint32_t pr = (j % 4u) / 2u;
        const double u1 = uniform_open_f64(pr ? w.z : w.x);
        const double u2 = uniform_open_f64(pr ? w.w : w.y);
        const double rad = sqrt(__dmul_rn(-2.0, log(u1)));
        const double th = __dmul_rn(two_pi, u2);
        const double gz = (j % 2u == 0u) ? __dmul_rn(rad, cos(th)) : __dmul_rn(rad, sin(th));
        r[d] = __dadd_rn(r[d], __dmul_rn(sigma, gz));
      }
      x[m0 + i + 1] = (float)r[0];
      y[m0 + i + 1] = (float)r[1];
      z[m0 + i + 1] = (float)r[2];
    }
  }
}

cudaError_t launch_init(const Geom& g, float* x, float* y, float* z, double sigma, int sm_count,
                        cudaStream_t st) {
  uint64_t blocks = (g.n_chains + 127) / 128;
  const uint64_t cap = (uint64_t)sm_count * 16;
  if (blocks > cap) blocks = cap;
  init_kernel<<<(unsigned)blocks, 128, 0, st>>>(g, x, y, z, sigma);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Spatial labelling of chains at initialisation: key = Morton code of the
// 8^3-cell block of the chain's first particle, packed above the old label so
// all keys are distinct and the sorted order is unique; a bitonic network
// sorts them; a gather moves whole chains to their new labels.
constexpr uint32_t SORT_BLOCK_SHIFT = 3;  // 8-cell blocks

__global__ void chain_key_kernel(const Geom g, const float* __restrict__ x,
                                 const float* __restrict__ y, const float* __restrict__ z,
                                 uint64_t* __restrict__ keys, uint64_t n_pad) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_pad; k += stride) {
    if (k >= g.n_chains) {
      keys[k] = ~0ull;
      continue;
    }
    const uint64_t m = k * g.N;
    const uint32_t b[3] = {
        fold_axis(g, 0, x[m], (uint32_t)g.nx) >> SORT_BLOCK_SHIFT,
        fold_axis(g, 1, y[m], (uint32_t)g.ny) >> SORT_BLOCK_SHIFT,
        fold_axis(g, 2, z[m], (uint32_t)g.nz) >> SORT_BLOCK_SHIFT};
    uint64_t key = 0;
    for (int bit = 0; bit < 10; ++bit)
      for (int d = 0; d < 3; ++d) key |= (uint64_t)((b[d] >> bit) & 1u) << (3 * bit + d);
    keys[k] = (key << 32) | k;
  }
}

__global__ void bitonic_step_kernel(uint64_t* __restrict__ a, uint64_t n, uint64_t j, uint64_t k) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t l = i ^ j;
    if (l <= i) continue;
    const uint64_t u = a[i], v = a[l];
    const bool up = (i & k) == 0;
    if ((u > v) == up) {
      a[i] = v;
      a[l] = u;
    }
  }
}

__global__ void chain_gather_kernel(const Geom g, const uint64_t* __restrict__ keys,
                                    const float* __restrict__ src, float* __restrict__ dst,
                                    uint64_t src_plane, uint64_t dst_plane) {
  const uint64_t M = g.n_chains * g.N;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += stride) {
    const uint64_t j = m / g.N, i = m - j * g.N;
    const uint64_t old = keys[j] & 0xFFFFFFFFull;
    const uint64_t from = old * g.N + i;
#pragma unroll
    for (int d = 0; d < 3; ++d) dst[d * dst_plane + m] = src[d * src_plane + from];
  }
}

cudaError_t launch_sort_chains(const Geom& g, const float* src, uint64_t src_plane, float* dst,
                               uint64_t dst_plane, uint64_t* keys, uint64_t n_pad, int sm_count,
                               cudaStream_t st) {
  const unsigned blocks = (unsigned)sm_count * 8;
  chain_key_kernel<<<blocks, 256, 0, st>>>(g, src, src + src_plane, src + 2 * src_plane, keys,
                                           n_pad);
  for (uint64_t k = 2; k <= n_pad; k <<= 1)
    for (uint64_t j = k >> 1; j > 0; j >>= 1)
      bitonic_step_kernel<<<blocks, 256, 0, st>>>(keys, n_pad, j, k);
  chain_gather_kernel<<<blocks, 256, 0, st>>>(g, keys, src, dst, src_plane, dst_plane);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 block reduction in a fixed order (deterministic for a fixed launch).
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* sh /* K*32 */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(FULL, v[k], o);
  if (lane == 0)
    for (int k = 0; k < K; ++k) sh[k * 32 + wid] = v[k];
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < K; ++k) {
      double t = lane < nw ? sh[k * 32 + lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
      v[k] = t;
    }
  }
}

__global__ void __launch_bounds__(256) chain_obs_kernel(const Geom g, const float* __restrict__ x,
                                                        const float* __restrict__ y,
                                                        const float* __restrict__ z,
                                                        double* __restrict__ part) {
  __shared__ double sh[2 * 32];
  const uint64_t M = g.n_chains * g.N;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double v[2] = {0.0, 0.0};
  for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += stride) {
    const uint32_t i = (uint32_t)(m % g.N);
    const double x0 = x[m], y0 = y[m], z0 = z[m];
    if (i + 1 < g.N) {
      const double dx = (double)x[m + 1] - x0, dy = (double)y[m + 1] - y0,
                   dz = (double)z[m + 1] - z0;
      v[0] += dx * dx + dy * dy + dz * dz;
    }
    if (i == 0) {
      const uint64_t e = m + g.N - 1;
      const double dx = (double)x[e] - x0, dy = (double)y[e] - y0, dz = (double)z[e] - z0;
      v[1] += dx * dx + dy * dy + dz * dz;
    }
  }
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x * 2 + 0] = v[0];
    part[blockIdx.x * 2 + 1] = v[1];
  }
}

__global__ void __launch_bounds__(256) grid_obs_kernel(const Geom g, const uint32_t* __restrict__ n,
                                                       double inv_rho, double kappaN, double chiN,
                                                       int hamiltonian, const float* __restrict__ ext,
                                                       double* __restrict__ part) {
  __shared__ double sh[2 * 32];
  double v[2] = {0.0, 0.0}, e_ext = 0.0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < g.cells; c += stride) {
    const uint32_t w = n[c];
    const double a = (double)(w & 0xFFFFu), b = (double)(w >> 16);
    const double phiA = a * inv_rho, phiB = b * inv_rho;
    const double fl = phiA + phiB - 1.0, df = phiA - phiB;
    v[0] += hamiltonian ? 0.5 * kappaN * fl * fl + chiN * phiA * phiB
                        : 0.5 * kappaN * fl * fl - 0.25 * chiN * df * df;
    if (ext) e_ext += a * (double)ext[c] + b * (double)ext[g.cells + c];
    v[1] = fmax(v[1], a + b);
  }
  // the max is folded by a second pass over the per-warp maxima
  double mx = v[1];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL, mx, o));
  __shared__ double shm[32];
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mx;
  double s1[2] = {v[0], e_ext};
  block_sum<2>(s1, sh);
  if (threadIdx.x == 0) {
    double m2 = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m2 = fmax(m2, shm[k]);
    part[2 * OBS_BLOCKS + blockIdx.x * 3 + 0] = s1[0];
    part[2 * OBS_BLOCKS + blockIdx.x * 3 + 1] = m2;
    part[2 * OBS_BLOCKS + blockIdx.x * 3 + 2] = s1[1];
  }
}

__global__ void obs_final_kernel(const double* __restrict__ part, int nb_chain, int nb_grid,
                                 double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double b2 = 0.0, re2 = 0.0, k = 0.0, mx = 0.0, ee = 0.0;
  for (int i = 0; i < nb_chain; ++i) {
    b2 += part[2 * i];
    re2 += part[2 * i + 1];
  }
  for (int i = 0; i < nb_grid; ++i) {
    k += part[2 * OBS_BLOCKS + 3 * i];
    mx = fmax(mx, part[2 * OBS_BLOCKS + 3 * i + 1]);
    ee += part[2 * OBS_BLOCKS + 3 * i + 2];
  }
  out[0] = b2;
  out[1] = re2;
  out[2] = k;
  out[3] = mx;
  out[4] = ee;
}

cudaError_t launch_observables(const Geom& g, const float* x, const float* y, const float* z,
                               const uint32_t* n, double inv_rho, double kappaN, double chiN,
                               int hamiltonian, const float* ext, double* part, double* out,
                               cudaStream_t st) {
  const uint64_t M = g.n_chains * g.N;
  uint64_t nb1 = (M + 255) / 256;
  if (nb1 > OBS_BLOCKS) nb1 = OBS_BLOCKS;
  uint64_t nb2 = ((uint64_t)g.cells + 255) / 256;
  if (nb2 > OBS_BLOCKS) nb2 = OBS_BLOCKS;
  chain_obs_kernel<<<(unsigned)nb1, 256, 0, st>>>(g, x, y, z, part);
  grid_obs_kernel<<<(unsigned)nb2, 256, 0, st>>>(g, n, inv_rho, kappaN, chiN, hamiltonian, ext,
                                                 part);
  obs_final_kernel<<<1, 32, 0, st>>>(part, (int)nb1, (int)nb2, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// S(q) = |sum_c dn(c) e^{-i q.c}|^2 / M with e^{-i q.c} the product of three
// per-axis twiddles (FP64, prepared on the host with exact argument reduction).
__global__ void __launch_bounds__(256) sq_kernel(const Geom g, const uint32_t* __restrict__ n,
                                                 const double* __restrict__ tw, int k,
                                                 double* __restrict__ part) {
  __shared__ double sh[2 * SQ_MAX * 32];
  double acc[2 * SQ_MAX];
#pragma unroll
  for (int q = 0; q < 2 * SQ_MAX; ++q) acc[q] = 0.0;
  const int T = g.nx + g.ny + g.nz;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < g.cells; c += stride) {
    const uint32_t w = n[c];
    const double dn = (double)(w & 0xFFFFu) - (double)(w >> 16);
    if (dn == 0.0) continue;
    const uint32_t cx = c % (uint32_t)g.nx;
    const uint32_t cy = (c / (uint32_t)g.nx) % (uint32_t)g.ny;
    const uint32_t cz = c / ((uint32_t)g.nx * (uint32_t)g.ny);
#pragma unroll
    for (int q = 0; q < SQ_MAX; ++q) {
      if (q >= k) break;
      const double* t = tw + (size_t)q * T * 2;
      const double ax = t[2 * cx], bx = t[2 * cx + 1];
      const double ay = t[2 * (g.nx + cy)], by = t[2 * (g.nx + cy) + 1];
      const double az = t[2 * (g.nx + g.ny + cz)], bz = t[2 * (g.nx + g.ny + cz) + 1];
      // (ax + i bx)(ay + i by)(az + i bz)
      const double pr = ax * ay - bx * by, pi = ax * by + bx * ay;
      const double rr = pr * az - pi * bz, ri = pr * bz + pi * az;
      acc[2 * q] += dn * rr;
      acc[2 * q + 1] += dn * ri;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < 2 * k; ++q) {
    double t = acc[q];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    if (lane == 0) sh[q * 32 + wid] = t;
  }
  __syncthreads();
  if (threadIdx.x < 2 * k) {
    double t = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += sh[threadIdx.x * 32 + w2];
    part[blockIdx.x * 2 * SQ_MAX + threadIdx.x] = t;
  }
}

__global__ void sq_final_kernel(const double* __restrict__ part, int nb, int k, double invM,
                                double* __restrict__ out) {
  const int q = threadIdx.x;
  if (q >= k) return;
  double re = 0.0, im = 0.0;
  for (int b = 0; b < nb; ++b) {
    re += part[b * 2 * SQ_MAX + 2 * q];
    im += part[b * 2 * SQ_MAX + 2 * q + 1];
  }
  out[q] = (re * re + im * im) * invM;
}

cudaError_t launch_structure_factor(const Geom& g, const uint32_t* n, const double* tw, int k,
                                    double* part, double* out, cudaStream_t st) {
  uint64_t nb = ((uint64_t)g.cells + 255) / 256;
  if (nb > SQ_BLOCKS) nb = SQ_BLOCKS;
  sq_kernel<<<(unsigned)nb, 256, 0, st>>>(g, n, tw, k, part);
  const double invM = 1.0 / (double)g.particles;
  sq_final_kernel<<<1, SQ_MAX, 0, st>>>(part, (int)nb, k, invM, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void philox_kernel(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key,
                              uint32_t* __restrict__ out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint4 r = philox4x32_10(c, key[2 * i], key[2 * i + 1]);
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n,
                          cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctr, key, out, n);
  return cudaGetLastError();
}

// What a smart Monte Carlo move makes of its draw (four words): the three
// normals and ln u of the spare 24 bits, by the sweeps' own device functions.
__global__ void smc_draws_kernel(const uint32_t* __restrict__ w, float* __restrict__ out,
                                 size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint4 r = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
    float gx, gy, gz;
    smc_normals(r, gx, gy, gz);
    out[4 * i] = gx;
    out[4 * i + 1] = gy;
    out[4 * i + 2] = gz;
    out[4 * i + 3] = log_uniform_open(spare_uniform_word(r));
  }
}

cudaError_t launch_smc_draws(const uint32_t* words, float* out, size_t n, int sm_count,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + 255) / 256;
  const size_t cap = (size_t)8 * (size_t)(sm_count > 0 ? sm_count : 1);
  smc_draws_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, st>>>(words, out, n);
  return cudaGetLastError();
}

}  // namespace soma
