// learned.cu -- the learned Metropolis-Hastings proposal (no counterpart in the
// paper, whose force-biased proposal is the smart Monte Carlo move of Sec. 2.2).
//
// A multilayer perceptron 12 -> 32 -> 32 -> 4 (ReLU hidden units) maps the
// features of a particle (bond vectors to its partners, the interpolated field
// gradient, is_A / has_prev / has_next) to a drift mu and a log step scale
// s = 2 tanh(o3/2); the trial move r' = r + mu + sigma0 e^s xi is accepted with
// min(1, exp(-dE) q(r|r') / q(r'|r)), the reverse density evaluating the network
// at r', so the move is exact for any weights.  Weights are stored BF16 for the
// sweep (FP32 arithmetic); an FP32 master copy is trained by maximising the
// expected squared jump E[alpha |r'-r|^2] with hand-written forward and
// backward passes and Adam, on configurations the plain method generates.
//
// Parameter layout (1604): W1[32][12] b1[32] W2[32][32] b2[32] W3[4][32] b3[4].
#include "kernels.h"
#include "draws.cuh"

namespace soma {

constexpr int L_W1 = 0, L_B1 = 384, L_W2 = 416, L_B2 = 1440, L_W3 = 1472, L_B3 = 1600;

// Forward pass; h1, h2 receive the hidden activations (for back-propagation).
__device__ __forceinline__ void mlp_fwd(const float* __restrict__ W, const float f[12], float h1[32],
                                        float h2[32], float o[4]) {
#pragma unroll 4
  for (int j = 0; j < 32; ++j) {
    float a = W[L_B1 + j];
#pragma unroll
    for (int k = 0; k < 12; ++k) a = fmaf(W[L_W1 + 12 * j + k], f[k], a);
    h1[j] = fmaxf(a, 0.f);
  }
#pragma unroll 4
  for (int j = 0; j < 32; ++j) {
    float a = W[L_B2 + j];
#pragma unroll
    for (int k = 0; k < 32; ++k) a = fmaf(W[L_W2 + 32 * j + k], h1[k], a);
    h2[j] = fmaxf(a, 0.f);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float a = W[L_B3 + j];
#pragma unroll
    for (int k = 0; k < 32; ++k) a = fmaf(W[L_W3 + 32 * j + k], h2[k], a);
    o[j] = a;
  }
}

// Per-axis field gradient at r: face differences of the cell interpolated
// linearly in the position inside the cell; dg receives their slopes.
template <typename WT>
__device__ __forceinline__ void interp_gradient(const Geom& g, const WT* w, float x, float y, float z,
                                                float gr[3], float dg[3], uint32_t* cell) {
  const uint32_t cx = fold_axis(g, 0, x, (uint32_t)g.nx);
  const uint32_t cy = fold_axis(g, 1, y, (uint32_t)g.ny);
  const uint32_t cz = fold_axis(g, 2, z, (uint32_t)g.nz);
  const uint32_t nx = g.nx, ny = g.ny, nz = g.nz;
  const uint32_t c = (cz * ny + cy) * nx + cx;
  const uint32_t xm = cx == 0 ? nx - 1 : cx - 1, xp = cx + 1 == nx ? 0 : cx + 1;
  const uint32_t ym = cy == 0 ? ny - 1 : cy - 1, yp = cy + 1 == ny ? 0 : cy + 1;
  const uint32_t zm = cz == 0 ? nz - 1 : cz - 1, zp = cz + 1 == nz ? 0 : cz + 1;
  const float w0 = load_w<WT>(w, c);
  const float lo[3] = {w0 - load_w<WT>(w, (cz * ny + cy) * nx + xm),
                       w0 - load_w<WT>(w, (cz * ny + ym) * nx + cx),
                       w0 - load_w<WT>(w, (zm * ny + cy) * nx + cx)};
  const float hi[3] = {load_w<WT>(w, (cz * ny + cy) * nx + xp) - w0,
                       load_w<WT>(w, (cz * ny + yp) * nx + cx) - w0,
                       load_w<WT>(w, (zp * ny + cy) * nx + cx) - w0};
  const float t[3] = {x - floorf(x), y - floorf(y), z - floorf(z)};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    gr[d] = fmaf(t[d], hi[d] - lo[d], lo[d]);
    dg[d] = hi[d] - lo[d];
  }
  *cell = c;
}

// ---------------------------------------------------------------------------
// The learned sweep (any N; the tiling of the generic kernels).
template <int Q, typename WT>
__global__ void __launch_bounds__(256) sweep_learned_kernel(const SweepArgs p,
                                                            const __nv_bfloat16* __restrict__ wq) {
  constexpr int S = 2 * Q;
  __shared__ float W[1604];
  for (int k = threadIdx.x; k < 1604; k += blockDim.x) W[k] = __bfloat162float(wq[k]);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned long long s64 = *p.d_sweep;
  const uint32_t sweep = (uint32_t)s64;
  uint32_t* __restrict__ nacc = ((s64 + 1ull) & 1ull) ? p.n1 : p.n0;
  const WT* __restrict__ wA = static_cast<const WT*>(p.wA);
  const WT* __restrict__ wB = static_cast<const WT*>(p.wB);
  const uint32_t N = p.g.N, N_A = p.g.N_A;
  const uint32_t ctr3a = (PURPOSE_MOVE << 24) | (p.g.replica & 0xFFFFFFu);
  const uint32_t ctr3b = (PURPOSE_MOVE2 << 24) | (p.g.replica & 0xFFFFFFu);
  const uint32_t li0 = (uint32_t)lane * S;
  const float sigma0 = p.learned_sigma0;
  const float K_b = p.K_b;

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
    float x[S], y[S], z[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const bool ok = li0 + j < nmono;
      x[j] = ok ? __ldcs(p.x + base + j) : 0.f;
      y[j] = ok ? __ldcs(p.y + base + j) : 0.f;
      z[j] = ok ? __ldcs(p.z + base + j) : 0.f;
    }
    float gx[S], gy[S], gz[S], lnu[S];
    uint32_t co[S];
    uint32_t lowbits = 0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const uint64_t m = base + j;
      const uint64_t mc = m + p.g.id_base;
      const uint4 r1 = philox_rk(make_uint4((uint32_t)mc, (uint32_t)(mc >> 32), sweep, ctr3a), p.g);
      const uint4 r2 = philox_rk(make_uint4((uint32_t)mc, (uint32_t)(mc >> 32), sweep, ctr3b), p.g);
      lowbits |= (r1.w & 1u) << j;
      float sn, cs;
      const float rad0 = sqrtf(-2.f * log_uniform_open_accurate(r1.x));
      sincos_2pi_uniform(r1.y, &sn, &cs);
      gx[j] = rad0 * cs;
      gy[j] = rad0 * sn;
      const float rad1 = sqrtf(-2.f * log_uniform_open_accurate(r1.z));
      sincos_2pi_uniform(r1.w, &sn, &cs);
      gz[j] = rad1 * cs;
      lnu[j] = log_uniform_open_accurate(r2.x);
      co[j] = cell_of(p.g, x[j], y[j], z[j]);
    }
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
        const bool hp = ci[j] > 0, hn = ci[j] + 1 < N;
        const float qx = (j > 0) ? x[j - 1] : pxl, qy = (j > 0) ? y[j - 1] : pyl,
                    qz = (j > 0) ? z[j - 1] : pzl;
        const float rx = (j < S - 1) ? x[j + 1] : nxl, ry = (j < S - 1) ? y[j + 1] : nyl,
                    rz = (j < S - 1) ? z[j + 1] : nzl;
        const WT* wt = (ci[j] < N_A) ? wA : wB;
        float f[12], h1[32], h2[32], o[4], orv[4], grad[3], dg[3];
        uint32_t c_old, c_new;
        f[0] = hp ? x[j] - qx : 0.f; f[1] = hp ? y[j] - qy : 0.f; f[2] = hp ? z[j] - qz : 0.f;
        f[3] = hn ? rx - x[j] : 0.f; f[4] = hn ? ry - y[j] : 0.f; f[5] = hn ? rz - z[j] : 0.f;
        interp_gradient<WT>(p.g, wt, x[j], y[j], z[j], grad, dg, &c_old);
        f[6] = grad[0]; f[7] = grad[1]; f[8] = grad[2];
        f[9] = ci[j] < N_A ? 1.f : 0.f;
        f[10] = hp ? 1.f : 0.f;
        f[11] = hn ? 1.f : 0.f;
        mlp_fwd(W, f, h1, h2, o);
        const float sig = sigma0 * expf(2.f * tanhf(0.5f * o[3]));
        const float tx = __fadd_rn(x[j], fmaf(sig, gx[j], o[0]));
        const float ty = __fadd_rn(y[j], fmaf(sig, gy[j], o[1]));
        const float tz = __fadd_rn(z[j], fmaf(sig, gz[j], o[2]));
        f[0] = hp ? tx - qx : 0.f; f[1] = hp ? ty - qy : 0.f; f[2] = hp ? tz - qz : 0.f;
        f[3] = hn ? rx - tx : 0.f; f[4] = hn ? ry - ty : 0.f; f[5] = hn ? rz - tz : 0.f;
        interp_gradient<WT>(p.g, wt, tx, ty, tz, grad, dg, &c_new);
        f[6] = grad[0]; f[7] = grad[1]; f[8] = grad[2];
        mlp_fwd(W, f, h1, h2, orv);
        const float sigr = sigma0 * expf(2.f * tanhf(0.5f * orv[3]));
        // energies
        const float dx = tx - x[j], dy = ty - y[j], dz = tz - z[j];
        float ux = 0.f, uy = 0.f, uz = 0.f;
        if (hp) { ux += x[j] - qx; uy += y[j] - qy; uz += z[j] - qz; }
        if (hn) { ux += x[j] - rx; uy += y[j] - ry; uz += z[j] - rz; }
        const float k = (float)((int)hp + (int)hn);
        const float du = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
        const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float dE = fmaf(K_b, fmaf(2.f, du, k * dd), load_w<WT>(wt, c_new) - load_w<WT>(wt, c_old));
        const float fx_ = dx - o[0], fy_ = dy - o[1], fz_ = dz - o[2];
        const float bx_ = -dx - orv[0], by_ = -dy - orv[1], bz_ = -dz - orv[2];
        const float lq_fwd = -fmaf(fx_, fx_, fmaf(fy_, fy_, fz_ * fz_)) / (2.f * sig * sig) - 3.f * logf(sig);
        const float lq_rev = -fmaf(bx_, bx_, fmaf(by_, by_, bz_ * bz_)) / (2.f * sigr * sigr) - 3.f * logf(sigr);
        const float log_alpha = -dE + lq_rev - lq_fwd;
        if (log_alpha >= 0.f || lnu[j] < log_alpha) {
          x[j] = tx;
          y[j] = ty;
          z[j] = tz;
          co[j] = c_new;
          ++my_acc;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if (li0 + j < nmono) {
        __stcs(p.x + base + j, x[j]);
        __stcs(p.y + base + j, y[j]);
        __stcs(p.z + base + j, z[j]);
        atomicAdd(nacc + co[j], (ci[j] < N_A) ? 1u : 0x10000u);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_acc += __shfl_xor_sync(FULL, my_acc, o);
  if (lane == 0 && my_acc) atomicAdd(p.acc, (unsigned long long)my_acc);
}

const void* learned_kernel_ptr(int Q, int grid_dtype) {
#define PICK(q)                                                                      \
  (grid_dtype == 1 ? (const void*)sweep_learned_kernel<q, __nv_bfloat16>             \
   : grid_dtype == 2 ? (const void*)sweep_learned_kernel<q, __half>                  \
                     : (const void*)sweep_learned_kernel<q, float>)
  return Q == 1 ? PICK(1) : (Q == 2 ? PICK(2) : PICK(4));
#undef PICK
}

cudaError_t launch_sweep_learned(const SweepArgs& a, const SweepShape& s, int grid_dtype,
                                 const void* wq, cudaStream_t st) {
  void* args[] = {const_cast<SweepArgs*>(&a), const_cast<void**>(&wq)};
  const void* fn = s.learned_tc ? learned_tc_kernel_ptr(grid_dtype, s.learned_umma)
                                : learned_kernel_ptr(s.Q, grid_dtype);
  return cudaLaunchKernel(fn, dim3(s.grid), dim3(s.block), args, 0, st);
}

// ---------------------------------------------------------------------------
// Training: the expected-squared-jump objective of one sample and its
// reparameterised gradient (positions not rounded: a smooth surrogate of the
// move), accumulated over a batch.  One thread per sample; the FP32 master
// weights are in shared memory; weight gradients are reduced in shared memory
// and then added to the global gradient.

__device__ __forceinline__ void mlp_bwd(const float* __restrict__ W, const float f[12],
                                        const float h1[32], const float h2[32], const float go[4],
                                        float* __restrict__ gW, float gx[12]) {
  float gz2[32], gz1[32];
#pragma unroll 4
  for (int k = 0; k < 32; ++k) {
    float a = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) a = fmaf(W[L_W3 + 32 * j + k], go[j], a);
    gz2[k] = h2[k] > 0.f ? a : 0.f;
  }
#pragma unroll 4
  for (int k = 0; k < 32; ++k) {
    float a = 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) a = fmaf(W[L_W2 + 32 * j + k], gz2[j], a);
    gz1[k] = h1[k] > 0.f ? a : 0.f;
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    float a = 0.f;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) a = fmaf(W[L_W1 + 12 * j + k], gz1[j], a);
    gx[k] = a;
  }
  for (int j = 0; j < 4; ++j) {
    atomicAdd(gW + L_B3 + j, go[j]);
    for (int k = 0; k < 32; ++k) atomicAdd(gW + L_W3 + 32 * j + k, go[j] * h2[k]);
  }
  for (int j = 0; j < 32; ++j) {
    atomicAdd(gW + L_B2 + j, gz2[j]);
    for (int k = 0; k < 32; ++k) atomicAdd(gW + L_W2 + 32 * j + k, gz2[j] * h1[k]);
  }
  for (int j = 0; j < 32; ++j) {
    atomicAdd(gW + L_B1 + j, gz1[j]);
    for (int k = 0; k < 12; ++k) atomicAdd(gW + L_W1 + 12 * j + k, gz1[j] * f[k]);
  }
}

template <typename WT>
__global__ void __launch_bounds__(128) esjd_grad_kernel(TrainArgs t) {
  __shared__ float W[1604];
  __shared__ float gW[1604];
  for (int k = threadIdx.x; k < 1604; k += blockDim.x) {
    W[k] = t.w[k];
    gW[k] = 0.f;
  }
  __syncthreads();
  const Geom& g = t.g;
  const uint32_t N = g.N;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < t.n; b += gridDim.x * blockDim.x) {
    uint64_t chain;
    uint32_t i;
    float xi[3];
    if (t.samples) {
      chain = t.samples[2 * b];
      i = t.samples[2 * b + 1];
      xi[0] = t.xi[3 * b]; xi[1] = t.xi[3 * b + 1]; xi[2] = t.xi[3 * b + 2];
    } else {
      const uint64_t id = (uint64_t)t.step * t.n + b;
      const uint32_t c3 = (PURPOSE_TRAIN << 24) | (g.replica & 0xFFFFFFu);
      const uint4 r1 = philox_rk(make_uint4((uint32_t)id, (uint32_t)(id >> 32), 0u, c3), g);
      const uint4 r2 = philox_rk(make_uint4((uint32_t)id, (uint32_t)(id >> 32), 1u, c3), g);
      chain = (uint64_t)(((uint64_t)r1.x << 32 | r1.y) % g.n_chains);
      i = r2.w % N;
      float sn, cs;
      const float rad0 = sqrtf(-2.f * log_uniform_open_accurate(r1.z));
      sincos_2pi_uniform(r1.w, &sn, &cs);
      xi[0] = rad0 * cs;
      xi[1] = rad0 * sn;
      const float rad1 = sqrtf(-2.f * log_uniform_open_accurate(r2.x));
      sincos_2pi_uniform(r2.y, &sn, &cs);
      xi[2] = rad1 * cs;
    }
    const uint64_t m = chain * N + i;
    const bool hp = i > 0, hn = i + 1 < N;
    const WT* wt = static_cast<const WT*>(i < g.N_A ? t.wA : t.wB);
    const float r[3] = {t.x[m], t.y[m], t.z[m]};
    float q[3] = {0.f, 0.f, 0.f}, nx[3] = {0.f, 0.f, 0.f};
    if (hp) { q[0] = t.x[m - 1]; q[1] = t.y[m - 1]; q[2] = t.z[m - 1]; }
    if (hn) { nx[0] = t.x[m + 1]; nx[1] = t.y[m + 1]; nx[2] = t.z[m + 1]; }
    float f[12], fr[12], h1[32], h2[32], h1r[32], h2r[32], o[4], orv[4], gr[3], dg[3];
    uint32_t c0, c1;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      f[d] = hp ? r[d] - q[d] : 0.f;
      f[3 + d] = hn ? nx[d] - r[d] : 0.f;
    }
    interp_gradient<WT>(g, wt, r[0], r[1], r[2], gr, dg, &c0);
    f[6] = gr[0]; f[7] = gr[1]; f[8] = gr[2];
    f[9] = i < g.N_A ? 1.f : 0.f;
    f[10] = hp ? 1.f : 0.f;
    f[11] = hn ? 1.f : 0.f;
    mlp_fwd(W, f, h1, h2, o);
    const float th = tanhf(0.5f * o[3]);
    const float sig = t.sigma0 * expf(2.f * th);
    float dv[3], rp[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      dv[d] = fmaf(sig, xi[d], o[d]);
      rp[d] = r[d] + dv[d];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      fr[d] = hp ? rp[d] - q[d] : 0.f;
      fr[3 + d] = hn ? nx[d] - rp[d] : 0.f;
    }
    interp_gradient<WT>(g, wt, rp[0], rp[1], rp[2], gr, dg, &c1);
    fr[6] = gr[0]; fr[7] = gr[1]; fr[8] = gr[2];
    fr[9] = f[9]; fr[10] = f[10]; fr[11] = f[11];
    mlp_fwd(W, fr, h1r, h2r, orv);
    const float thr = tanhf(0.5f * orv[3]);
    const float sigr = t.sigma0 * expf(2.f * thr);
    float e[3], e2 = 0.f, D = 0.f, Eb_new = 0.f, Eb_old = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      e[d] = r[d] - rp[d] - orv[d];
      e2 = fmaf(e[d], e[d], e2);
      D = fmaf(dv[d], dv[d], D);
      if (hp) {
        Eb_new += (rp[d] - q[d]) * (rp[d] - q[d]);
        Eb_old += (r[d] - q[d]) * (r[d] - q[d]);
      }
      if (hn) {
        Eb_new += (rp[d] - nx[d]) * (rp[d] - nx[d]);
        Eb_old += (r[d] - nx[d]) * (r[d] - nx[d]);
      }
    }
    const float xi2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
    const float dE = t.K_b * (Eb_new - Eb_old) + (load_w<WT>(wt, c1) - load_w<WT>(wt, c0));
    const float lq_rev = -e2 / (2.f * sigr * sigr) - 3.f * logf(sigr);
    const float lq_fwd = -0.5f * xi2 - 3.f * logf(sig);
    const float l = -dE + lq_rev - lq_fwd;
    const float alpha = l >= 0.f ? 1.f : expf(l);
    const float J = alpha * D;
    if (t.J) t.J[b] = J;
    if (t.log_alpha) t.log_alpha[b] = l;
    const float cl = l < 0.f ? alpha * D : 0.f;
    float g_rp[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      g_rp[d] = alpha * 2.f * dv[d];
      if (hp) g_rp[d] += cl * (-2.f * t.K_b * (rp[d] - q[d]));
      if (hn) g_rp[d] += cl * (-2.f * t.K_b * (rp[d] - nx[d]));
      g_rp[d] += cl * e[d] / (sigr * sigr);
    }
    float go_r[4], gfr[12];
#pragma unroll
    for (int d = 0; d < 3; ++d) go_r[d] = cl * e[d] / (sigr * sigr);
    go_r[3] = cl * (e2 / (sigr * sigr) - 3.f) * (1.f - thr * thr);
    mlp_bwd(W, fr, h1r, h2r, go_r, gW, gfr);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (hp) g_rp[d] += gfr[d];
      if (hn) g_rp[d] -= gfr[3 + d];
      g_rp[d] += gfr[6 + d] * dg[d];
    }
    float go_f[4], gf[12];
    float dls = cl * 3.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      go_f[d] = g_rp[d];
      dls = fmaf(g_rp[d], sig * xi[d], dls);
    }
    go_f[3] = dls * (1.f - th * th);
    mlp_bwd(W, f, h1, h2, go_f, gW, gf);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 1604; k += blockDim.x) atomicAdd(t.grad + k, gW[k]);
}

cudaError_t launch_esjd_grad(const TrainArgs& t, int grid_dtype, int sm_count, cudaStream_t st) {
  uint64_t blocks = (t.n + 127) / 128;
  const uint64_t cap = (uint64_t)sm_count * 4;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  switch (grid_dtype) {
    case 1: esjd_grad_kernel<__nv_bfloat16><<<(unsigned)blocks, 128, 0, st>>>(t); break;
    case 2: esjd_grad_kernel<__half><<<(unsigned)blocks, 128, 0, st>>>(t); break;
    default: esjd_grad_kernel<float><<<(unsigned)blocks, 128, 0, st>>>(t); break;
  }
  return cudaGetLastError();
}

// Adam (Kingma & Ba) on -grad/n (the objective is maximised); the BF16 copy
// used by the sweep is refreshed from the FP32 master weights.
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ mom, float* __restrict__ vel,
                            const float* __restrict__ grad, __nv_bfloat16* __restrict__ wq,
                            float lr, float b1, float b2, float eps, float c1, float c2,
                            float inv_n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 1604) return;
  const float g = -grad[k] * inv_n;
  const float m = b1 * mom[k] + (1.f - b1) * g;
  const float v = b2 * vel[k] + (1.f - b2) * g * g;
  mom[k] = m;
  vel[k] = v;
  w[k] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  wq[k] = __float2bfloat16_rn(w[k]);
}

cudaError_t launch_adam(float* w, float* m, float* v, const float* grad, void* wq, float lr,
                        float b1, float b2, float eps, int step, float inv_n, cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<(1604 + 255) / 256, 256, 0, st>>>(w, m, v, grad, (__nv_bfloat16*)wq, lr, b1, b2,
                                                  eps, c1, c2, inv_n);
  return cudaGetLastError();
}

__global__ void quantize_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wq) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < 1604) wq[k] = __float2bfloat16_rn(w[k]);
}

cudaError_t launch_quantize(const float* w, void* wq, cudaStream_t st) {
  quantize_kernel<<<(1604 + 255) / 256, 256, 0, st>>>(w, (__nv_bfloat16*)wq);
  return cudaGetLastError();
}

}  // namespace soma
