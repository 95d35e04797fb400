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

// Open uniform in FP64 (init path): (k + 1/2)/2^24, exact.
__device__ __forceinline__ double uniform_open_f64(uint32_t r) {
  return ((double)(r >> 8) + 0.5) * 5.9604644775390625e-8;
}

// Cell of one coordinate: floor(x) folded into [0, n), exact for |x| < 2^18
// (the supported position range, in units of dL).
//  - floor: adding 1.5*2^23 with rounding toward -inf leaves floor(x) +
//    1.5*2^23 exactly (|x| < 2^22), whose bit pattern is 0x4B400000 + floor(x);
//  - c = floor(x) + bias with bias = n*ceil(2^18/n), so 0 <= c < 2^19 + n
//    (the bit pattern times s = 1 plus b = bias - 0x4B400000, mod 2^32);
//  - c mod n = c - n*umulhi(c, m), m = ceil(2^32/n): with e = m*n - 2^32 < n,
//    umulhi(c, m) = floor(c/n + c*e/(n*2^32)) = floor(c/n) whenever c*e < 2^32,
//    which holds for c < 2^19 + n and n <= 4096 (Granlund & Montgomery 1994,
//    Sec. 4, with the shift folded into m).
// An axis with n = 1 has s = b = m = 0 and always folds to 0.  Everything runs
// on the FMA pipe (one FADD, three IMAD).  Outside the supported range the
// result is not the cell; callers clamp it so that memory stays in bounds.
__device__ __forceinline__ uint32_t fold_raw(float x, uint32_t n, uint32_t m, uint32_t s,
                                             uint32_t b) {
  const uint32_t c = __float_as_uint(__fadd_rd(x, 12582912.0f)) * s + b;
  return c - __umulhi(c, m) * n;
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
  uint32_t fold_m[3];     // ceil(2^32/n) per axis (0 for n = 1)
  uint32_t fold_s[3];     // 1 (0 for n = 1)
  uint32_t fold_b[3];     // n*ceil(2^18/n) - 0x4B400000 mod 2^32 (0 for n = 1)
  uint32_t cells;
  uint32_t key0, key1;
  uint32_t rk0[10], rk1[10];  // Philox round keys: key + r * (Weyl constant)
  uint32_t replica;
  // One shard of a larger system (chains distributed over ranks, Sec. 3.1.1):
  // its chain k is chain chain_base + k of the whole system, and every draw
  // is keyed on the whole system's chain and particle indices (id_base =
  // chain_base * N), so that the shards together draw what one handle holding
  // every chain draws.  Both 0 for a system held whole.  A sharded system has
  // fewer than 2^32 particles, so 32-bit counters stay exact.
  uint64_t chain_base, id_base;
  // Particles the occupation numbers count: n_chains * N, less the absent
  // slots of molecules with fewer particles than N; for a shard, those of the
  // whole system (its grid holds the whole system's counts).
  uint64_t particles;
};

// Per-axis cell, clamped into [0, n) (exact inside the supported range).
// The clamp already sends an n = 1 axis to 0, so the bias is added without
// the multiplier s (an integer add instead of a multiply-add).
__device__ __forceinline__ uint32_t fold_axis(const Geom& g, int k, float x, uint32_t n) {
  const uint32_t c = __float_as_uint(__fadd_rd(x, 12582912.0f)) + g.fold_b[k];
  return min(c - __umulhi(c, g.fold_m[k]) * n, n - 1u);
}

// Linear cell index (x fastest), clamped into the grid as a whole: one min
// instead of one per axis.
__device__ __forceinline__ uint32_t cell_of(const Geom& g, float x, float y, float z) {
  const uint32_t cx = fold_raw(x, (uint32_t)g.nx, g.fold_m[0], g.fold_s[0], g.fold_b[0]);
  const uint32_t cy = fold_raw(y, (uint32_t)g.ny, g.fold_m[1], g.fold_s[1], g.fold_b[1]);
  const uint32_t cz = fold_raw(z, (uint32_t)g.nz, g.fold_m[2], g.fold_s[2], g.fold_b[2]);
  return min((cz * (uint32_t)g.ny + cy) * (uint32_t)g.nx + cx, g.cells - 1u);
}

// Cell of the floor bits fb = bits of __fadd_rd(x, 1.5*2^23) per axis (the
// first step of fold_raw done by the caller).  WIDE: every axis has at least
// two cells, so the bias is added without the multiplier s (an integer add on
// the ALU instead of a multiply-add on the FMA pipe); otherwise as fold_raw.
template <bool WIDE>
__device__ __forceinline__ uint32_t cell_of_floor_bits(const Geom& g, uint32_t fbx, uint32_t fby,
                                                       uint32_t fbz) {
  uint32_t c[3];
  const uint32_t fb[3] = {fbx, fby, fbz};
  const uint32_t n[3] = {(uint32_t)g.nx, (uint32_t)g.ny, (uint32_t)g.nz};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint32_t b = WIDE ? fb[k] + g.fold_b[k] : fb[k] * g.fold_s[k] + g.fold_b[k];
    c[k] = b - __umulhi(b, g.fold_m[k]) * n[k];
  }
  return min((c[2] * n[1] + c[1]) * n[0] + c[0], g.cells - 1u);
}

// Two FP32 values in one 64-bit register pair for the packed FP32x2
// instructions of sm_100 and later: each half is rounded exactly as the
// scalar instruction with the same rounding mode rounds it.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_add_rm(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_fma_rn(unsigned long long a, unsigned long long b,
                                                        unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
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
  const float4* smc_tab;    // smart Monte Carlo: omega and field force per cell, A then B
  unsigned* err;            // sticky error bits (a bounded wait that gave up)
  const uint64_t* seq;      // mixture of linear architectures: bit i of seq[a] set =
  const uint8_t* arch;      // particle i of architecture a is B; arch[chain] (or NULL)
};

// Smart Monte Carlo: omega and the field force (minus the central difference
// of omega along each axis) of cell c, one 16-byte entry of the table plane
// of the particle's type.
__device__ __forceinline__ float smc_field(const float4* __restrict__ tab, uint32_t c, float& fx,
                                           float& fy, float& fz) {
  const float4 q = __ldg(tab + c);
  fx = q.y;
  fy = q.z;
  fz = q.w;
  return q.x;
}

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
  int hamiltonian;          // 0: K^0_inter, 1: K^1_inter
  const float* ext;         // external potential, A cells then B cells (or NULL)
  const uint8_t* forbidden; // cells no particle may enter (or NULL)
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
  int hamiltonian;                 // 0: K^0_inter, 1: K^1_inter
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
