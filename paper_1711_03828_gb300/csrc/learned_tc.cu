// learned_tc.cu -- the learned proposal for even N <= 64 with the network on
// the tensor cores.
//
// In the paired layout (pair_body.cuh) every lane moves exactly one particle
// per SET phase, so each phase evaluates the network on one feature row per
// lane: 32 rows per warp, 128 rows per 4-warp block.  Two evaluators of the
// 12 -> 32 -> 32 -> 4 network (BF16 operands, FP32 accumulation):
//   WarpNet   (default) warp-level mma.sync m16n8k16 with the weights held as
//             register fragments: every warp walks its own tiles;
//   UmmaNet   5th-generation tensor cores: the block's 128 rows are one
//             M = 128 tile; one thread issues tcgen05.mma per layer (K = 16
//             for layer 1 with the bias folded in as a constant-1 feature,
//             2 x K = 16 for layers 2 and 3, N = 32 / 32 / 16), operands in
//             shared memory in the K-major core-matrix layout (8 rows x 16
//             bytes per core matrix), the accumulator in 32 TMEM columns,
//             completion through tcgen05.commit on an mbarrier, results read
//             back with tcgen05.ld (each warp its 32 TMEM lanes).  Each
//             tile needs twelve dependent products (two SET phases, forward
//             and reverse network, three layers) and the block's warps must
//             meet for each, so this evaluator is the slower one here.
// The move itself (normals, features, reverse density, acceptance) is the one
// of learned.cu and is shared by both.
#include "kernels.h"
#include "pair_body.cuh"
#include "draws.cuh"

namespace soma {

constexpr int TC_W1 = 0, TC_B1 = 384, TC_W2 = 416, TC_B2 = 1440, TC_W3 = 1472, TC_B3 = 1600;

struct MlpFrag {
  uint32_t w1[4][2];     // layer 1, n-tile x (k 0-7 | k 8-15)
  uint32_t w2[2][4][2];  // layer 2, k-step x n-tile
  uint32_t w3[2][2];     // layer 3, k-step
  float b1[4][2], b2[4][2], b3[2];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat16 l = __float2bfloat16_rn(lo), h = __float2bfloat16_rn(hi);
  return (uint32_t)__bfloat16_as_ushort(l) | ((uint32_t)__bfloat16_as_ushort(h) << 16);
}

__device__ __forceinline__ uint32_t relu_pack(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

__device__ __forceinline__ void mma16816(float d[4], const uint32_t a[4], const uint32_t b[2],
                                         const float c[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%10,%11,%12,%13};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "f"(c[0]), "f"(c[1]),
        "f"(c[2]), "f"(c[3]));
}

__device__ __forceinline__ float wv(const __nv_bfloat16* W, int idx) { return __bfloat162float(W[idx]); }

// Fragments of this lane: g = lane/4 (row / output column group), c = lane%4.
__device__ __forceinline__ void mlp_load(MlpFrag& R, const __nv_bfloat16* __restrict__ W, int lane) {
  const int g = lane >> 2, c = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int j = 8 * nt + g;  // output unit (column of B)
    const int k0 = 2 * c, k1 = 2 * c + 8;
    R.w1[nt][0] = pack_bf16(wv(W, TC_W1 + 12 * j + k0), wv(W, TC_W1 + 12 * j + k0 + 1));
    R.w1[nt][1] = (k1 < 12) ? pack_bf16(wv(W, TC_W1 + 12 * j + k1), wv(W, TC_W1 + 12 * j + k1 + 1)) : 0u;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const int kk = 16 * ks + 2 * c;
      R.w2[ks][nt][0] = pack_bf16(wv(W, TC_W2 + 32 * j + kk), wv(W, TC_W2 + 32 * j + kk + 1));
      R.w2[ks][nt][1] = pack_bf16(wv(W, TC_W2 + 32 * j + kk + 8), wv(W, TC_W2 + 32 * j + kk + 9));
    }
    R.b1[nt][0] = wv(W, TC_B1 + 8 * nt + 2 * c);
    R.b1[nt][1] = wv(W, TC_B1 + 8 * nt + 2 * c + 1);
    R.b2[nt][0] = wv(W, TC_B2 + 8 * nt + 2 * c);
    R.b2[nt][1] = wv(W, TC_B2 + 8 * nt + 2 * c + 1);
  }
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    const int kk = 16 * ks + 2 * c;
    R.w3[ks][0] = g < 4 ? pack_bf16(wv(W, TC_W3 + 32 * g + kk), wv(W, TC_W3 + 32 * g + kk + 1)) : 0u;
    R.w3[ks][1] = g < 4 ? pack_bf16(wv(W, TC_W3 + 32 * g + kk + 8), wv(W, TC_W3 + 32 * g + kk + 9)) : 0u;
  }
  R.b3[0] = c < 2 ? wv(W, TC_B3 + 2 * c) : 0.f;
  R.b3[1] = c < 2 ? wv(W, TC_B3 + 2 * c + 1) : 0.f;
}

// Network outputs for this lane's feature vector f; every lane of the warp
// takes part.  sf: this warp's [32][16] BF16 staging rows; so: [32][4] floats.
__device__ __forceinline__ void mlp_warp(const MlpFrag& R, __nv_bfloat16* sf, float* so,
                                         const float f[12], float o[4], int lane) {
  const int g = lane >> 2, c = lane & 3;
  uint4 lo4, hi4;
  lo4.x = pack_bf16(f[0], f[1]);
  lo4.y = pack_bf16(f[2], f[3]);
  lo4.z = pack_bf16(f[4], f[5]);
  lo4.w = pack_bf16(f[6], f[7]);
  hi4.x = pack_bf16(f[8], f[9]);
  hi4.y = pack_bf16(f[10], f[11]);
  hi4.z = 0u;
  hi4.w = 0u;
  reinterpret_cast<uint4*>(sf + 16 * lane)[0] = lo4;
  reinterpret_cast<uint4*>(sf + 16 * lane)[1] = hi4;
  __syncwarp();
  uint32_t a1[2][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int row = 16 * mt + (lane & 15), col = (lane >> 4) * 8;
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(sf + 16 * row + col);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a1[mt][0]), "=r"(a1[mt][1]), "=r"(a1[mt][2]), "=r"(a1[mt][3])
                 : "r"(addr));
  }
  // layer 1 -> ReLU -> layer 2 operands
  uint32_t a2[2][2][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    float d[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const float cb[4] = {R.b1[nt][0], R.b1[nt][1], R.b1[nt][0], R.b1[nt][1]};
      mma16816(d[nt], a1[mt], R.w1[nt], cb);
    }
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      a2[mt][ks][0] = relu_pack(d[2 * ks][0], d[2 * ks][1]);
      a2[mt][ks][1] = relu_pack(d[2 * ks][2], d[2 * ks][3]);
      a2[mt][ks][2] = relu_pack(d[2 * ks + 1][0], d[2 * ks + 1][1]);
      a2[mt][ks][3] = relu_pack(d[2 * ks + 1][2], d[2 * ks + 1][3]);
    }
  }
  // layer 2 -> ReLU -> layer 3 -> outputs
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    float d[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const float cb[4] = {R.b2[nt][0], R.b2[nt][1], R.b2[nt][0], R.b2[nt][1]};
      mma16816(d[nt], a2[mt][0], R.w2[0][nt], cb);
      mma16816(d[nt], a2[mt][1], R.w2[1][nt], d[nt]);
    }
    uint32_t a3[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      a3[ks][0] = relu_pack(d[2 * ks][0], d[2 * ks][1]);
      a3[ks][1] = relu_pack(d[2 * ks][2], d[2 * ks][3]);
      a3[ks][2] = relu_pack(d[2 * ks + 1][0], d[2 * ks + 1][1]);
      a3[ks][3] = relu_pack(d[2 * ks + 1][2], d[2 * ks + 1][3]);
    }
    float e[4];
    const float cb[4] = {R.b3[0], R.b3[1], R.b3[0], R.b3[1]};
    mma16816(e, a3[0], R.w3[0], cb);
    mma16816(e, a3[1], R.w3[1], e);
    if (c < 2) {
      so[4 * (16 * mt + g) + 2 * c] = e[0];
      so[4 * (16 * mt + g) + 2 * c + 1] = e[1];
      so[4 * (16 * mt + g + 8) + 2 * c] = e[2];
      so[4 * (16 * mt + g + 8) + 2 * c + 1] = e[3];
    }
  }
  __syncwarp();
  const float4 r = reinterpret_cast<const float4*>(so)[lane];
  o[0] = r.x;
  o[1] = r.y;
  o[2] = r.z;
  o[3] = r.w;
  __syncwarp();
}

// The mma.sync evaluator: one warp, its own 32 rows.
struct WarpNet {
  const MlpFrag* R;
  __nv_bfloat16* sf;
  float* so;
  int lane;
  __device__ __forceinline__ void eval(const float f[12], float o[4]) { mlp_warp(*R, sf, so, f, o, lane); }
};

// ---------------------------------------------------------------------------
// The tcgen05 evaluator.
constexpr uint32_t UMMA_TMEM_COLS = 32;
// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t umma_idesc(uint32_t M, uint32_t N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
// shared-memory matrix descriptor, no swizzle: start, leading-dimension (K)
// and stride-dimension (M/N) byte offsets, all >> 4; bits 46-48 = 0b001
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void umma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(bar) : "memory");
}
// Bounded wait for the given phase parity of an mbarrier.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          uint32_t limit = (1u << 22)) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile("{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, P;\n}\n" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t v[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
               "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                 "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                 "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
                 "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
                 "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
                 "=r"(v[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t v[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Byte offset of element (r, k) of a K-major BF16 operand with K = 16 * kc
// columns: core matrices of 8 rows x 8 elements (128 bytes), adjacent along K
// 128 bytes apart (leading offset), 8-row groups 128 * 2 kc bytes apart.
__host__ __device__ constexpr uint32_t cm_off(uint32_t r, uint32_t k, uint32_t kcores) {
  return (r >> 3) * (128u * kcores) + (k >> 3) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

// Shared memory of one block of the tcgen05 kernel.
struct UmmaSmem {
  __align__(1024) unsigned char x[128 * 16 * 2];   // features, 128 x 16 (2 K cores)
  __align__(1024) unsigned char h[128 * 32 * 2];   // hidden layer, 128 x 32 (4 K cores)
  __align__(1024) unsigned char w1[32 * 16 * 2];   // W1 | b1 as N x K = 32 x 16
  __align__(1024) unsigned char w2[32 * 32 * 2];   // W2, 32 x 32
  __align__(1024) unsigned char w3[16 * 32 * 2];   // W3 padded to 16 rows, 16 x 32
  float b2[32];
  float b3[4];
  __align__(8) unsigned long long bar;
  uint32_t tmem_base;
};

// The block's 128 threads evaluate together; thread t owns row t.  ok turns
// false (block-wide at the next synchronisation) when a wait for the tensor
// cores gives up; from then on nothing is issued and the outputs are zeros.
struct UmmaNet {
  UmmaSmem* sm;
  uint32_t tmem;     // accumulator columns of this block
  uint32_t bar;      // mbarrier address
  uint32_t phase;    // parity of the next completion
  uint32_t t;        // row
  uint32_t lane_off; // this warp's TMEM lane quarter (<< 16)
  bool ok;

  // Make this thread's shared-memory rows visible to the tensor cores and
  // agree block-wide on the error state.
  __device__ __forceinline__ void sync() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    const int bad = __syncthreads_or(!ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = !bad;
  }
  __device__ __forceinline__ void wait() {
    bool done = ok && mbar_wait(bar, phase);
    done = __all_sync(FULL, done);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = ok && done;
  }
  // relu(v + b) of 32 accumulator columns as BF16 into this thread's row of h
  __device__ __forceinline__ void store_hidden(const uint32_t v[32], const float* b) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint4 q;
      uint32_t* w = &q.x;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = 8 * c + 2 * e;
        w[e] = relu_pack(__uint_as_float(v[k]) + (b ? b[k] : 0.f),
                         __uint_as_float(v[k + 1]) + (b ? b[k + 1] : 0.f));
      }
      *reinterpret_cast<uint4*>(sm->h + cm_off(t, 8 * c, 4)) = q;
    }
  }
  __device__ __forceinline__ void eval(const float f[12], float o[4]) {
    uint4 lo, hi;
    lo.x = pack_bf16(f[0], f[1]);
    lo.y = pack_bf16(f[2], f[3]);
    lo.z = pack_bf16(f[4], f[5]);
    lo.w = pack_bf16(f[6], f[7]);
    hi.x = pack_bf16(f[8], f[9]);
    hi.y = pack_bf16(f[10], f[11]);
    hi.z = pack_bf16(1.f, 0.f);   // constant feature 12 carries b1
    hi.w = 0u;
    *reinterpret_cast<uint4*>(sm->x + cm_off(t, 0, 2)) = lo;
    *reinterpret_cast<uint4*>(sm->x + cm_off(t, 8, 2)) = hi;
    const uint32_t xa = (uint32_t)__cvta_generic_to_shared(sm->x);
    const uint32_t ha = (uint32_t)__cvta_generic_to_shared(sm->h);
    const uint32_t w1a = (uint32_t)__cvta_generic_to_shared(sm->w1);
    const uint32_t w2a = (uint32_t)__cvta_generic_to_shared(sm->w2);
    const uint32_t w3a = (uint32_t)__cvta_generic_to_shared(sm->w3);
    uint32_t v[32];
    // layer 1: [128 x 16] x [16 x 32]
    sync();
    if (ok && t == 0) {
      umma_f16(tmem, umma_sdesc(xa, 128, 256), umma_sdesc(w1a, 128, 256), umma_idesc(128, 32), 0);
      umma_commit(bar);
    }
    wait();
    if (ok) tmem_ld32(tmem + lane_off, v);
    else
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = 0u;
    store_hidden(v, nullptr);
    // layer 2: [128 x 32] x [32 x 32] as two K = 16 steps
    sync();
    if (ok && t == 0) {
      umma_f16(tmem, umma_sdesc(ha, 128, 512), umma_sdesc(w2a, 128, 512), umma_idesc(128, 32), 0);
      umma_f16(tmem, umma_sdesc(ha + 256, 128, 512), umma_sdesc(w2a + 256, 128, 512),
               umma_idesc(128, 32), 1);
      umma_commit(bar);
    }
    wait();
    if (ok) tmem_ld32(tmem + lane_off, v);
    else
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = 0u;
    store_hidden(v, sm->b2);
    // layer 3: [128 x 32] x [32 x 16] (outputs 0-3 used)
    sync();
    if (ok && t == 0) {
      umma_f16(tmem, umma_sdesc(ha, 128, 512), umma_sdesc(w3a, 128, 512), umma_idesc(128, 16), 0);
      umma_f16(tmem, umma_sdesc(ha + 256, 128, 512), umma_sdesc(w3a + 256, 128, 512),
               umma_idesc(128, 16), 1);
      umma_commit(bar);
    }
    wait();
    uint32_t u[4] = {0u, 0u, 0u, 0u};
    if (ok) tmem_ld4(tmem + lane_off, u);
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = __uint_as_float(u[j]) + sm->b3[j];
  }
};

// Interpolated field gradient at (x,y,z) and omega of its cell (as learned.cu).
template <typename WT>
__device__ __forceinline__ float grad_at(const Geom& g, const WT* w, float x, float y, float z,
                                         float gr[3], uint32_t* cell) {
  const uint32_t cx = fold_axis(g, 0, x, (uint32_t)g.nx);
  const uint32_t cy = fold_axis(g, 1, y, (uint32_t)g.ny);
  const uint32_t cz = fold_axis(g, 2, z, (uint32_t)g.nz);
  const uint32_t nx = g.nx, ny = g.ny, nz = g.nz;
  const uint32_t c = (cz * ny + cy) * nx + cx;
  const uint32_t xm = cx == 0 ? nx - 1 : cx - 1, xp = cx + 1 == nx ? 0 : cx + 1;
  const uint32_t ym = cy == 0 ? ny - 1 : cy - 1, yp = cy + 1 == ny ? 0 : cy + 1;
  const uint32_t zm = cz == 0 ? nz - 1 : cz - 1, zp = cz + 1 == nz ? 0 : cz + 1;
  const float w0 = load_w<WT>(w, c);
  const float lo0 = w0 - load_w<WT>(w, (cz * ny + cy) * nx + xm);
  const float lo1 = w0 - load_w<WT>(w, (cz * ny + ym) * nx + cx);
  const float lo2 = w0 - load_w<WT>(w, (zm * ny + cy) * nx + cx);
  const float hi0 = load_w<WT>(w, (cz * ny + cy) * nx + xp) - w0;
  const float hi1 = load_w<WT>(w, (cz * ny + yp) * nx + cx) - w0;
  const float hi2 = load_w<WT>(w, (zp * ny + cy) * nx + cx) - w0;
  gr[0] = fmaf(x - floorf(x), hi0 - lo0, lo0);
  gr[1] = fmaf(y - floorf(y), hi1 - lo1, lo1);
  gr[2] = fmaf(z - floorf(z), hi2 - lo2, lo2);
  *cell = c;
  return w0;
}

// One learned move of this lane's mover r (partners pv, nv when hp, hn).
template <typename WT, typename Net>
__device__ __forceinline__ bool learned_move(const Geom& g, Net& net, const WT* wt, bool isA,
                                             bool hp, bool hn, float& rx, float& ry, float& rz,
                                             uint32_t& cell, float px, float py, float pz, float qx,
                                             float qy, float qz, const float xi[3], float lnu,
                                             float sigma0, float K_b, bool valid) {
  float f[12], gr[3], o[4], orv[4];
  uint32_t c_old, c_new;
  const float w_old = grad_at<WT>(g, wt, rx, ry, rz, gr, &c_old);
  f[0] = hp ? rx - px : 0.f; f[1] = hp ? ry - py : 0.f; f[2] = hp ? rz - pz : 0.f;
  f[3] = hn ? qx - rx : 0.f; f[4] = hn ? qy - ry : 0.f; f[5] = hn ? qz - rz : 0.f;
  f[6] = gr[0]; f[7] = gr[1]; f[8] = gr[2];
  f[9] = isA ? 1.f : 0.f;
  f[10] = hp ? 1.f : 0.f;
  f[11] = hn ? 1.f : 0.f;
  net.eval(f, o);
  const float sig = sigma0 * __expf(2.f * tanhf(0.5f * o[3]));
  const float tx = __fadd_rn(rx, fmaf(sig, xi[0], o[0]));
  const float ty = __fadd_rn(ry, fmaf(sig, xi[1], o[1]));
  const float tz = __fadd_rn(rz, fmaf(sig, xi[2], o[2]));
  const float w_new = grad_at<WT>(g, wt, tx, ty, tz, gr, &c_new);
  f[0] = hp ? tx - px : 0.f; f[1] = hp ? ty - py : 0.f; f[2] = hp ? tz - pz : 0.f;
  f[3] = hn ? qx - tx : 0.f; f[4] = hn ? qy - ty : 0.f; f[5] = hn ? qz - tz : 0.f;
  f[6] = gr[0]; f[7] = gr[1]; f[8] = gr[2];
  net.eval(f, orv);
  const float sigr = sigma0 * __expf(2.f * tanhf(0.5f * orv[3]));
  const float dx = tx - rx, dy = ty - ry, dz = tz - rz;
  float ux = 0.f, uy = 0.f, uz = 0.f;
  if (hp) { ux += rx - px; uy += ry - py; uz += rz - pz; }
  if (hn) { ux += rx - qx; uy += ry - qy; uz += rz - qz; }
  const float k = (float)((int)hp + (int)hn);
  const float du = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
  const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float dE = fmaf(K_b, fmaf(2.f, du, k * dd), w_new - w_old);
  const float ax = dx - o[0], ay = dy - o[1], az = dz - o[2];
  const float bx = -dx - orv[0], by = -dy - orv[1], bz = -dz - orv[2];
  const float lq_fwd = -fmaf(ax, ax, fmaf(ay, ay, az * az)) / (2.f * sig * sig) - 3.f * __logf(sig);
  const float lq_rev = -fmaf(bx, bx, fmaf(by, by, bz * bz)) / (2.f * sigr * sigr) - 3.f * __logf(sigr);
  const float log_alpha = -dE + lq_rev - lq_fwd;
  const bool acc = valid && (log_alpha >= 0.f || lnu < log_alpha);
  if (acc) {
    rx = tx;
    ry = ty;
    rz = tz;
    cell = c_new;
  } else {
    cell = c_old;
  }
  return acc;
}

// One tile of the paired learned sweep for this lane (particles base, base+1);
// valid: this lane's pair exists.  Returns the accepted moves.
template <typename WT, typename Net>
__device__ __forceinline__ unsigned learned_pair_tile(const SweepArgs& p, const PairLane<WT>& L,
                                                      Net& net, uint32_t* __restrict__ nacc,
                                                      uint32_t base, bool valid, uint32_t sweep,
                                                      bool A0, bool A1) {
  const int lane = L.lane;
  const uint32_t ctr3a = (PURPOSE_MOVE << 24) | (p.g.replica & 0xFFFFFFu);
  const uint32_t ctr3b = (PURPOSE_MOVE2 << 24) | (p.g.replica & 0xFFFFFFu);
  float x0 = 0.f, x1 = 0.f, y0 = 0.f, y1 = 0.f, z0 = 0.f, z1 = 0.f;
  if (valid) {
    const float2 a = __ldcs(reinterpret_cast<const float2*>(p.x + base));
    const float2 b = __ldcs(reinterpret_cast<const float2*>(p.y + base));
    const float2 c = __ldcs(reinterpret_cast<const float2*>(p.z + base));
    x0 = a.x; x1 = a.y; y0 = b.x; y1 = b.y; z0 = c.x; z1 = c.y;
  }
  // normals by Box-Muller with the hardware log and sincos: the acceptance
  // uses the realised trial position, so the move stays exact
  float xi0[3], xi1[3], lnu0, lnu1;
  uint32_t w3first;
  {
    const uint32_t cb = base + (uint32_t)p.g.id_base;
    const uint4 r1 = philox_rk(make_uint4(cb, 0u, sweep, ctr3a), p.g);
    const uint4 r2 = philox_rk(make_uint4(cb, 0u, sweep, ctr3b), p.g);
    const uint4 s1 = philox_rk(make_uint4(cb + 1u, 0u, sweep, ctr3a), p.g);
    const uint4 s2 = philox_rk(make_uint4(cb + 1u, 0u, sweep, ctr3b), p.g);
    float sn, cs;
    float rad = sqrtf(-2.f * log_uniform_open(r1.x));
    sincos_2pi_uniform_fast(r1.y, &sn, &cs);
    xi0[0] = rad * cs; xi0[1] = rad * sn;
    rad = sqrtf(-2.f * log_uniform_open(r1.z));
    sincos_2pi_uniform_fast(r1.w, &sn, &cs);
    xi0[2] = rad * cs;
    lnu0 = log_uniform_open(r2.x);
    rad = sqrtf(-2.f * log_uniform_open(s1.x));
    sincos_2pi_uniform_fast(s1.y, &sn, &cs);
    xi1[0] = rad * cs; xi1[1] = rad * sn;
    rad = sqrtf(-2.f * log_uniform_open(s1.z));
    sincos_2pi_uniform_fast(s1.w, &sn, &cs);
    xi1[2] = rad * cs;
    lnu1 = log_uniform_open(s2.x);
    w3first = r1.w;
  }
  const bool sw = p.set_order_random && (__shfl_sync(FULL, w3first, L.first_lane) & 1u);
  uint32_t c0 = 0, c1 = 0;
  unsigned n_acc = 0;
  // first set moves slot sw, second set slot !sw
#pragma unroll
  for (int ph = 0; ph < 2; ++ph) {
    const bool odd = (ph == 0) ? sw : !sw;   // the mover is slot 1
    // the adjacent lane's non-moving slot: slot 1 of lane-1 when slot 0 moves,
    // slot 0 of lane+1 when slot 1 moves
    const float ox = odd ? x0 : x1, oy = odd ? y0 : y1, oz = odd ? z0 : z1;
    const int src = odd ? lane + 1 : lane - 1;
    const float sx = __shfl_sync(FULL, ox, src & 31);
    const float sy = __shfl_sync(FULL, oy, src & 31);
    const float sz = __shfl_sync(FULL, oz, src & 31);
    float rx = odd ? x1 : x0, ry = odd ? y1 : y0, rz = odd ? z1 : z0;
    const bool hp = odd ? true : L.has_prev0, hn = odd ? L.has_next1 : true;
    const float px = odd ? x0 : sx, py = odd ? y0 : sy, pz = odd ? z0 : sz;
    const float qx = odd ? sx : x1, qy = odd ? sy : y1, qz = odd ? sz : z1;
    uint32_t cell;
    const bool acc = learned_move<WT, Net>(p.g, net, odd ? L.w1 : L.w0, odd ? A1 : A0, hp, hn, rx,
                                           ry, rz, cell, px, py, pz, qx, qy, qz,
                                           odd ? xi1 : xi0, odd ? lnu1 : lnu0, p.learned_sigma0,
                                           p.K_b, valid);
    if (odd) { x1 = rx; y1 = ry; z1 = rz; c1 = cell; }
    else { x0 = rx; y0 = ry; z0 = rz; c0 = cell; }
    n_acc += acc;
  }
  if (valid) {
    __stcs(reinterpret_cast<float2*>(p.x + base), make_float2(x0, x1));
    __stcs(reinterpret_cast<float2*>(p.y + base), make_float2(y0, y1));
    __stcs(reinterpret_cast<float2*>(p.z + base), make_float2(z0, z1));
    if (c0 == c1) {
      atomicAdd(nacc + c0, L.v0 + L.v1);
    } else {
      atomicAdd(nacc + c0, L.v0);
      atomicAdd(nacc + c1, L.v1);
    }
  }
  return n_acc;
}

// mma.sync network: every warp walks its own tiles.
template <typename WT>
__global__ void __launch_bounds__(128) sweep_learned_tc_kernel(const SweepArgs p,
                                                               const __nv_bfloat16* __restrict__ wq) {
  __shared__ __align__(16) __nv_bfloat16 s_feat[4][32 * 16];
  __shared__ __align__(16) float s_out[4][32 * 4];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  MlpFrag R;
  mlp_load(R, wq, lane);
  WarpNet net{&R, s_feat[wib], s_out[wib], lane};
  const uint32_t n_tiles_all = (uint32_t)p.n_tiles;
  const uint32_t chunk = (n_tiles_all + gridDim.x - 1) / gridDim.x;
  const uint32_t t_begin = blockIdx.x * chunk;
  const uint32_t t_end = min(t_begin + chunk, n_tiles_all);
  const unsigned long long s64 = *p.d_sweep;
  const uint32_t sweep = (uint32_t)s64;
  uint32_t* __restrict__ nacc = ((s64 + 1ull) & 1ull) ? p.n1 : p.n0;
  PairLane<WT> L;
  L.init(lane, p.g.N, p.g.N_A, p.wA, p.wB);
  const uint32_t ci0 = L.li0 % p.g.N;
  const bool A0 = ci0 < p.g.N_A, A1 = ci0 + 1 < p.g.N_A;
  const uint32_t TN = p.G * p.g.N;
  unsigned my_acc = 0;
  for (uint32_t tile = t_begin + wib; tile < t_end; tile += 4) {
    const bool valid = tile < (uint32_t)p.full_tiles || L.li0 < p.last_rows;
    my_acc += learned_pair_tile<WT, WarpNet>(p, L, net, nacc, tile * TN + L.li0, valid, sweep, A0, A1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_acc += __shfl_xor_sync(FULL, my_acc, o);
  if (lane == 0 && my_acc) atomicAdd(p.acc, (unsigned long long)my_acc);
}

// tcgen05 network: the block's four warps step through their tiles together
// (every network evaluation is one block-wide M = 128 product); a warp
// without a tile of its own takes part with empty rows.
template <typename WT>
__global__ void __launch_bounds__(128) sweep_learned_umma_kernel(const SweepArgs p,
                                                                 const __nv_bfloat16* __restrict__ wq) {
  __shared__ UmmaSmem sm;
  const uint32_t t = threadIdx.x;
  const int lane = (int)(t & 31u), wib = (int)(t >> 5);
  // weights as the B operands (N x K, K-major), biases of layers 2 and 3
  for (uint32_t i = t; i < 32 * 16; i += 128) {
    const uint32_t n = i >> 4, k = i & 15u;
    const float v = k < 12 ? __bfloat162float(wq[TC_W1 + 12 * n + k])
                  : (k == 12 ? __bfloat162float(wq[TC_B1 + n]) : 0.f);
    *reinterpret_cast<__nv_bfloat16*>(sm.w1 + cm_off(n, k, 2)) = __float2bfloat16_rn(v);
  }
  for (uint32_t i = t; i < 32 * 32; i += 128) {
    const uint32_t n = i >> 5, k = i & 31u;
    *reinterpret_cast<__nv_bfloat16*>(sm.w2 + cm_off(n, k, 4)) = wq[TC_W2 + 32 * n + k];
  }
  for (uint32_t i = t; i < 16 * 32; i += 128) {
    const uint32_t n = i >> 5, k = i & 31u;
    *reinterpret_cast<__nv_bfloat16*>(sm.w3 + cm_off(n, k, 4)) =
        n < 4 ? wq[TC_W3 + 32 * n + k] : __float2bfloat16_rn(0.f);
  }
  if (t < 32) sm.b2[t] = __bfloat162float(wq[TC_B2 + t]);
  if (t < 4) sm.b3[t] = __bfloat162float(wq[TC_B3 + t]);
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&sm.bar);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (wib == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(&sm.tmem_base)), "r"(UMMA_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  UmmaNet net{&sm, sm.tmem_base, bar, 0u, t, (uint32_t)(32 * wib) << 16, true};

  const uint32_t n_tiles_all = (uint32_t)p.n_tiles;
  const uint32_t chunk = (n_tiles_all + gridDim.x - 1) / gridDim.x;
  const uint32_t t_begin = blockIdx.x * chunk;
  const uint32_t t_end = min(t_begin + chunk, n_tiles_all);
  const uint32_t rounds = t_end > t_begin ? (t_end - t_begin + 3) / 4 : 0;
  const unsigned long long s64 = *p.d_sweep;
  const uint32_t sweep = (uint32_t)s64;
  uint32_t* __restrict__ nacc = ((s64 + 1ull) & 1ull) ? p.n1 : p.n0;
  PairLane<WT> L;
  L.init(lane, p.g.N, p.g.N_A, p.wA, p.wB);
  const uint32_t ci0 = L.li0 % p.g.N;
  const bool A0 = ci0 < p.g.N_A, A1 = ci0 + 1 < p.g.N_A;
  const uint32_t TN = p.G * p.g.N;
  unsigned my_acc = 0;
  for (uint32_t r = 0; r < rounds; ++r) {
    const uint32_t tile = t_begin + 4 * r + (uint32_t)wib;
    const bool valid = tile < t_end && (tile < (uint32_t)p.full_tiles || L.li0 < p.last_rows);
    const uint32_t base = (tile < t_end ? tile : t_begin) * TN + L.li0;
    my_acc += learned_pair_tile<WT, UmmaNet>(p, L, net, nacc, base, valid && net.ok, sweep, A0, A1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_acc += __shfl_xor_sync(FULL, my_acc, o);
  if (lane == 0 && my_acc) atomicAdd(p.acc, (unsigned long long)my_acc);
  if (!net.ok) {
    // a wait gave up: report it, give the last product a bounded chance to
    // finish, then release the accumulator columns as usual
    if (t == 0) atomicOr(p.err, ERR_TIMEOUT);
    mbar_wait(bar, net.phase ^ 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (wib == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(net.tmem), "r"(UMMA_TMEM_COLS) : "memory");
}

// Diagnostic of the bounded waits: one warp waits, with the given iteration
// limit, for an mbarrier phase that never completes, and records the timeout.
__global__ void wait_probe_kernel(uint32_t limit, unsigned* err) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool done = mbar_wait(b, 0u, limit);
  if (!done && threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
}

cudaError_t launch_wait_probe(uint32_t limit, unsigned* err, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(limit, err);
  return cudaGetLastError();
}

const void* learned_tc_kernel_ptr(int grid_dtype, bool umma) {
  if (umma)
    return grid_dtype == 1 ? (const void*)sweep_learned_umma_kernel<__nv_bfloat16>
         : grid_dtype == 2 ? (const void*)sweep_learned_umma_kernel<__half>
                           : (const void*)sweep_learned_umma_kernel<float>;
  return grid_dtype == 1 ? (const void*)sweep_learned_tc_kernel<__nv_bfloat16>
       : grid_dtype == 2 ? (const void*)sweep_learned_tc_kernel<__half>
                         : (const void*)sweep_learned_tc_kernel<float>;
}

}  // namespace soma
