// common.cuh -- device-side building blocks of libsoma (sm_103a).
//
// Philox4x32-10 counter RNG (Salmon, Moraes, Dror, Shaw, SC'11), the uniform
// maps, the periodic cell fold and the kernel argument blocks.  Nothing here
// is shared with the CPU oracle; both sides implement the generator from its
// published definition.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace soma {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint32_t PURPOSE_INIT = 0, PURPOSE_MOVE = 1, PURPOSE_MOVE2 = 2, PURPOSE_TRAIN = 5;

// Philox4x32-10: ten rounds of two 32x32->64 products (counter words 0 and 2
// times the round multipliers) whose high halves are xored with counter words
// 1 and 3 and the round key, with the key advanced by the Weyl constants
// between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Symmetric uniform (2k+1)/2^24 - 1 of the top 24 bits k of r: never 0, and
// exact in FP32: k*2^-23 + (2^-24 - 1) is representable, and the fused
// multiply-add rounds the exact value once.
__device__ __forceinline__ float uniform_sym(uint32_t r) {
  return fmaf(__uint2float_rn(r >> 8), 1.1920928955078125e-7f, -0.99999994039535522461f);
}

// ln of the open uniform (k + 1/2)/2^24.
__device__ __forceinline__ float log_uniform_open(uint32_t r) {
  return __logf(fmaf(__uint2float_rn(r >> 8), 5.9604644775390625e-8f, 2.98023223876953125e-8f));
}

// ln of the open uniform u = (k + 1/2)/2^24, accurate to about one FP32 ulp of
// the result for every k: below 1/2 u itself is exact in FP32; above, 1 - u =
// (2^24 - k - 1/2)/2^24 is exact instead and log1p is used.
__device__ __forceinline__ float log_uniform_open_accurate(uint32_t r) {
  const uint32_t k = r >> 8;
  if (k < (1u << 23)) return logf(fmaf(__uint2float_rn(k), 5.9604644775390625e-8f,
                                       2.98023223876953125e-8f));
  const float one_minus_u = fmaf(__uint2float_rn((1u << 24) - k), 5.9604644775390625e-8f,
                                 -2.98023223876953125e-8f);
  return log1pf(-one_minus_u);
}

// cos and sin of 2 pi u for the open uniform u = (k + 1/2)/2^24: with the exact
// symmetric uniform v = 2u - 1, 2 pi u = pi v + pi, so cos = -cospi(v) and
// sin = -sinpi(v), evaluated without rounding the phase.
__device__ __forceinline__ void sincos_2pi_uniform(uint32_t r, float* s, float* c) {
  float sv, cv;
  sincospif(uniform_sym(r), &sv, &cv);
  *s = -sv;
  *c = -cv;
}

// Open uniform in FP64 (init path): (k + 1/2)/2^24, exact.
__device__ __forceinline__ double uniform_open_f64(uint32_t r) {
  return ((double)(r >> 8) + 0.5) * 5.9604644775390625e-8;
}

// Cell of one coordinate: floor(x) folded into [0, n) by an exact
// multiply-high division (Granlund & Montgomery 1994, Thm. 4.2, for 31-bit
// numerators): with l = ceil(log2 n) and m = floor(2^(31+l)/n) + 1,
// floor(c/n) = umulhi(c, m) >> (l-1) for every 0 <= c < 2^31.  c = floor(x) +
// bias, bias = n*floor(2^30/n), so every |x| < 2^30 is folded exactly.  The
// final unsigned min keeps the index inside the grid for any input (and makes
// an axis with n = 1, which has m = 0, always fold to 0).
__device__ __forceinline__ uint32_t fold_cell(float x, uint32_t n, uint32_t m, uint32_t sh,
                                              uint32_t bias) {
  const uint32_t c = (uint32_t)__float2int_rd(x) + bias;
  const uint32_t q = __umulhi(c, m) >> sh;
  return min(c - q * n, n - 1u);
}

template <typename WT> __device__ __forceinline__ float load_w(const WT* p, uint32_t i);
template <> __device__ __forceinline__ float load_w<float>(const float* p, uint32_t i) {
  return __ldg(p + i);
}
template <> __device__ __forceinline__ float load_w<__nv_bfloat16>(const __nv_bfloat16* p, uint32_t i) {
  return __bfloat162float(__ldg(p + i));
}
template <> __device__ __forceinline__ float load_w<__half>(const __half* p, uint32_t i) {
  return __half2float(__ldg(p + i));
}

template <typename WT> __device__ __forceinline__ WT store_cvt(float v);
template <> __device__ __forceinline__ float store_cvt<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 store_cvt<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half store_cvt<__half>(float v) { return __float2half_rn(v); }

// Geometry and Philox key shared by every kernel of one system.
struct Geom {
  uint64_t n_chains;
  uint32_t N, N_A;
  int nx, ny, nz;
  uint32_t fold_m[3];     // multiply-high magic per axis (0 for n = 1)
  uint32_t fold_sh[3];    // ceil(log2 n) - 1 per axis
  uint32_t fold_bias[3];  // n * floor(2^30/n) per axis
  uint32_t cells;
  uint32_t key0, key1;
  uint32_t rk0[10], rk1[10];  // Philox round keys: key + r * (Weyl constant)
  uint32_t replica;
};

__device__ __forceinline__ uint32_t cell_of(const Geom& g, float x, float y, float z) {
  const uint32_t cx = fold_cell(x, (uint32_t)g.nx, g.fold_m[0], g.fold_sh[0], g.fold_bias[0]);
  const uint32_t cy = fold_cell(y, (uint32_t)g.ny, g.fold_m[1], g.fold_sh[1], g.fold_bias[1]);
  const uint32_t cz = fold_cell(z, (uint32_t)g.nz, g.fold_m[2], g.fold_sh[2], g.fold_bias[2]);
  return (cz * (uint32_t)g.ny + cy) * (uint32_t)g.nx + cx;
}

// Philox4x32-10 with the round keys taken from the kernel parameters (the
// key schedule is the same for every thread, so it is computed once on the
// host and read from the constant bank).
__device__ __forceinline__ uint4 philox_rk(uint4 c, const Geom& g) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ g.rk0[r], (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ g.rk1[r], (uint32_t)p0);
  }
  return c;
}

struct SweepArgs {
  Geom g;
  float* x;
  float* y;
  float* z;
  const void* wA;           // omega_A plane, storage type WT
  const void* wB;           // omega_B plane
  uint32_t* n0;             // occupation buffers; the sweep of step s adds into
  uint32_t* n1;             // n[(s+1)&1]
  unsigned long long* acc;  // accepted-move counter
  const unsigned long long* d_sweep;
  float a;                  // maximal displacement (dL), FP32
  float K_b;                // k0/2 in kT/dL^2
  uint32_t G;               // chains per warp tile
  uint64_t n_tiles;
  uint64_t full_tiles;      // tiles holding G chains
  uint32_t last_rows;       // particles in the last, partial tile (0: none)
  int set_order_random;
  // smart Monte Carlo: A = a^2/6, sqrt(2A), 1/(4A)
  float smc_A, smc_s2A, smc_inv4A;
  float learned_sigma0;     // a/sqrt(3): scale of the learned proposal
};

// Training of the learned proposal: one expected-squared-jump sample per thread.
struct TrainArgs {
  Geom g;
  const float* x;
  const float* y;
  const float* z;
  const void* wA;
  const void* wB;
  const float* w;            // FP32 parameters (1604)
  float* grad;               // accumulated dJ/dW (1604)
  float* J;                  // per-sample objective (optional)
  float* log_alpha;          // per-sample log acceptance (optional)
  const uint32_t* samples;   // (chain, i) pairs, or NULL: drawn with Philox (purpose 5)
  const float* xi;           // 3 normals per sample when samples are given
  uint32_t n;                // samples
  uint32_t step;             // training step (counter word of the drawn samples)
  float sigma0, K_b;
};

struct FieldArgs {
  Geom g;
  uint32_t* n0;             // occupation buffers (packed A | B<<16)
  uint32_t* n1;
  void* wA;                 // omega_A plane, storage type WT
  void* wB;                 // omega_B plane
  unsigned long long* d_sweep;
  unsigned int* err;        // sticky error bits
  float inv_rho;            // 1/(rho_0 dL^3)
  float kappa0;             // kappaN/N
  float half_chi0;          // chiN/(2N)
  int after_sweep;          // 1: read n[(s+1)&1], clear n[s&1], then s += 1
                            // 0: read n[s&1], clear n[(s+1)&1]
};

// One system of a batch (device table entry).
struct BatchSys {
  Geom g;                          // geometry and cell fold of this system
  float* x;
  float* y;
  float* z;
  const void* wA;
  const void* wB;
  uint32_t* n0;
  uint32_t* n1;
  unsigned long long* counters;    // [0] sweep counter, [1] accepted moves
  float a, K_b;
  uint32_t G, full_tiles, last_rows;
  uint32_t cell_begin;             // offset of this grid in the concatenated cells
  float inv_rho, kappa0, half_chi0;
  int set_order_random;
};

struct BatchItem {
  uint32_t sys, t0, t1;            // tiles [t0, t1) of system sys
};

struct BatchArgs {
  const BatchSys* sys;
  uint32_t n_sys;
  const BatchItem* items;
  uint32_t n_items;
  Geom keys;                       // Philox round keys (one seed for the batch)
  const unsigned long long* d_sweep;  // every member's counter has this value
};

constexpr unsigned ERR_OVERFLOW = 1u;
constexpr unsigned ERR_TIMEOUT = 2u;

}  // namespace soma
