// smc.cu -- the smart Monte Carlo (force-biased) sweep kernels.
//
// Trial move dr = A F(r) + sqrt(2A) xi with A = a^2/6, F the bonded force
// minus the central-difference gradient of omega_t over the six neighbouring
// cells, accepted with min(1, exp(-dE) T(r'->r)/T(r->r')) (Sec. 2.2 names the
// force-biased proposal; the Rossky-Doll-Friedman form is used).  One Philox
// draw per move (purpose 1): normals by Box-Muller from the top 24 bits of its
// four words, the acceptance uniform from the 24 bits they leave (the low
// bytes of words 0-2).  The radius sqrt(-2 ln u) takes ln u accurate to about an
// ulp (near u = 1 a small absolute error of ln u would be a large one of the
// radius); the angle takes the hardware sincos (absolute error about 2^-21,
// below 1e-6 dL in the displacement) and the acceptance test the hardware log,
// as the uniform move does.  The move stays exact whatever the normals'
// rounding: the acceptance evaluates both proposal densities at the realised
// trial position.
#include "kernels.h"
#include "pair_body.cuh"
#include "draws.cuh"

namespace soma {

// ---------------------------------------------------------------------------
// Smart Monte Carlo (force-biased) step, any N (the tiling of
// sweep_uniform_kernel).  Trial move dr = A F(r) + sqrt(2A) xi, F = bonded
// force minus the central-difference gradient of omega_t over the six
// neighbouring cells; accepted with min(1, exp(-dE) T(r'->r)/T(r->r')),
// T(r->r') = exp(-|r'-r-A F(r)|^2/(4A)).  Normals and the acceptance uniform
// from one draw (purpose 1), as above.
__device__ __forceinline__ void cell3(const Geom& g, float x, float y, float z, uint32_t& cx,
                                      uint32_t& cy, uint32_t& cz) {
  cx = fold_axis(g, 0, x, (uint32_t)g.nx);
  cy = fold_axis(g, 1, y, (uint32_t)g.ny);
  cz = fold_axis(g, 2, z, (uint32_t)g.nz);
}

// omega at the cell and minus its central-difference gradient (the field force).
template <typename WT>
__device__ __forceinline__ float field_and_force(const Geom& g, const WT* w, uint32_t cx, uint32_t cy,
                                                 uint32_t cz, float& fx, float& fy, float& fz) {
  const uint32_t nx = g.nx, ny = g.ny, nz = g.nz;
  const uint32_t row = (cz * ny + cy) * nx;
  const uint32_t xm = cx == 0 ? nx - 1 : cx - 1, xp = cx + 1 == nx ? 0 : cx + 1;
  const uint32_t ym = cy == 0 ? ny - 1 : cy - 1, yp = cy + 1 == ny ? 0 : cy + 1;
  const uint32_t zm = cz == 0 ? nz - 1 : cz - 1, zp = cz + 1 == nz ? 0 : cz + 1;
  fx = -0.5f * (load_w<WT>(w, row + xp) - load_w<WT>(w, row + xm));
  fy = -0.5f * (load_w<WT>(w, (cz * ny + yp) * nx + cx) - load_w<WT>(w, (cz * ny + ym) * nx + cx));
  fz = -0.5f * (load_w<WT>(w, (zp * ny + cy) * nx + cx) - load_w<WT>(w, (zm * ny + cy) * nx + cx));
  return load_w<WT>(w, row + cx);
}

// The smart Monte Carlo table, rebuilt after every field update: per type and
// cell, omega_t(c) and minus its central difference along each axis (the
// field force of field_and_force, bit for bit), one float4 per cell, A then
// B.  A move reads it with one 16-byte load at its old and one at its trial
// cell instead of gathering seven field values at each.
template <typename WT>
__global__ void smc_table_kernel(const Geom g, const WT* __restrict__ wA, const WT* __restrict__ wB,
                                 float4* __restrict__ tab) {
  const uint32_t nx = g.nx, ny = g.ny;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < g.cells;
       c += gridDim.x * blockDim.x) {
    const uint32_t cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    float fx, fy, fz;
    float w = field_and_force<WT>(g, wA, cx, cy, cz, fx, fy, fz);
    tab[c] = make_float4(w, fx, fy, fz);
    w = field_and_force<WT>(g, wB, cx, cy, cz, fx, fy, fz);
    tab[g.cells + c] = make_float4(w, fx, fy, fz);
  }
}

// The same table for n_t types: one plane of float4 per type from the FP32
// field planes w (n_types * cells).
__global__ void smc_table_planes_kernel(const Geom g, const float* __restrict__ w, uint32_t planes,
                                        float4* __restrict__ tab) {
  const uint32_t nx = g.nx, ny = g.ny;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < g.cells;
       c += gridDim.x * blockDim.x) {
    const uint32_t cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    for (uint32_t t = 0; t < planes; ++t) {
      float fx, fy, fz;
      const float v = field_and_force<float>(g, w + (size_t)t * g.cells, cx, cy, cz, fx, fy, fz);
      tab[(size_t)t * g.cells + c] = make_float4(v, fx, fy, fz);
    }
  }
}

cudaError_t launch_smc_table_planes(const Geom& g, const float* w, uint32_t planes, float4* tab,
                                    int sm_count, cudaStream_t st) {
  smc_table_planes_kernel<<<4 * sm_count, 256, 0, st>>>(g, w, planes, tab);
  return cudaGetLastError();
}

cudaError_t launch_smc_table(const Geom& g, const void* wA, const void* wB, float4* tab,
                             int grid_dtype, int sm_count, cudaStream_t st) {
  const int grid = 4 * sm_count;
  switch (grid_dtype) {
    case 1:
      smc_table_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(
          g, static_cast<const __nv_bfloat16*>(wA), static_cast<const __nv_bfloat16*>(wB), tab);
      break;
    case 2:
      smc_table_kernel<__half><<<grid, 256, 0, st>>>(g, static_cast<const __half*>(wA),
                                                     static_cast<const __half*>(wB), tab);
      break;
    default:
      smc_table_kernel<float><<<grid, 256, 0, st>>>(g, static_cast<const float*>(wA),
                                                    static_cast<const float*>(wB), tab);
  }
  return cudaGetLastError();
}

template <int Q>
__global__ void __launch_bounds__(256) sweep_smc_kernel(const SweepArgs p) {
  constexpr int S = 2 * Q;
  const int lane = threadIdx.x & 31;
  const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned long long s64 = *p.d_sweep;
  const uint32_t sweep = (uint32_t)s64;
  uint32_t* __restrict__ nacc = ((s64 + 1ull) & 1ull) ? p.n1 : p.n0;
  const float4* __restrict__ tabA = p.smc_tab;
  const float4* __restrict__ tabB = p.smc_tab + p.g.cells;
  const uint32_t N = p.g.N, N_A = p.g.N_A;
  const uint32_t ctr3a = (PURPOSE_MOVE << 24) | (p.g.replica & 0xFFFFFFu);
  const uint32_t li0 = (uint32_t)lane * S;
  const float A = p.smc_A, s2A = p.smc_s2A, inv4A = p.smc_inv4A, K2 = 2.f * p.K_b;

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

    // configuration-independent part: old cell, field and field force at the
    // old cell (loaded first, so that the loads are in flight during the
    // draws), normals, acceptance uniform
    float gx[S], gy[S], gz[S], lnu[S], w_old[S], fox[S], foy[S], foz[S];
    uint32_t co[S];
    uint32_t lowbits = 0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
      uint32_t cx, cy, cz;
      cell3(p.g, x[j], y[j], z[j], cx, cy, cz);
      co[j] = (cz * (uint32_t)p.g.ny + cy) * (uint32_t)p.g.nx + cx;
      const float4* tab = (ci[j] < N_A) ? tabA : tabB;
      w_old[j] = 0.f;
      fox[j] = foy[j] = foz[j] = 0.f;
      if (li0 + j < nmono) w_old[j] = smc_field(tab, co[j], fox[j], foy[j], foz[j]);
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const uint64_t m = base + j + p.g.id_base;
      const uint4 r1 = philox_rk(make_uint4((uint32_t)m, (uint32_t)(m >> 32), sweep, ctr3a), p.g);
      lowbits |= (r1.w & 1u) << j;
      smc_normals(r1, gx[j], gy[j], gz[j]);
      lnu[j] = log_uniform_open(spare_uniform_word(r1));
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
        // U = sum over bonded partners of (r - n); bonded force = -2 K_b U
        float ux = 0.f, uy = 0.f, uz = 0.f;
        if (hp) { ux += x[j] - qx; uy += y[j] - qy; uz += z[j] - qz; }
        if (hn) { ux += x[j] - rx; uy += y[j] - ry; uz += z[j] - rz; }
        const float k = (float)((int)hp + (int)hn);
        const float Fx = fmaf(-K2, ux, fox[j]), Fy = fmaf(-K2, uy, foy[j]), Fz = fmaf(-K2, uz, foz[j]);
        const float tx = __fadd_rn(x[j], fmaf(s2A, gx[j], A * Fx));
        const float ty = __fadd_rn(y[j], fmaf(s2A, gy[j], A * Fy));
        const float tz = __fadd_rn(z[j], fmaf(s2A, gz[j], A * Fz));
        uint32_t cx, cy, cz;
        cell3(p.g, tx, ty, tz, cx, cy, cz);
        const float4* tab = (ci[j] < N_A) ? tabA : tabB;
        const uint32_t cn = (cz * (uint32_t)p.g.ny + cy) * (uint32_t)p.g.nx + cx;
        float fnx, fny, fnz;
        const float w_new = smc_field(tab, cn, fnx, fny, fnz);
        const float dx = tx - x[j], dy = ty - y[j], dz = tz - z[j];
        // bonded energy change d.(2U + k d); partners' new U' = U + k d
        const float du = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
        const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float dE = fmaf(p.K_b, fmaf(2.f, du, k * dd), w_new - w_old[j]);
        const float Gx = fmaf(-K2, fmaf(k, dx, ux), fnx), Gy = fmaf(-K2, fmaf(k, dy, uy), fny),
                    Gz = fmaf(-K2, fmaf(k, dz, uz), fnz);
        const float ax = dx - A * Fx, ay = dy - A * Fy, az = dz - A * Fz;   // forward residual
        const float bx = -dx - A * Gx, by = -dy - A * Gy, bz = -dz - A * Gz;  // reverse residual
        const float fwd = fmaf(ax, ax, fmaf(ay, ay, az * az));
        const float rev = fmaf(bx, bx, fmaf(by, by, bz * bz));
        const float log_alpha = fmaf(fwd - rev, inv4A, -dE);
        if (log_alpha >= 0.f || lnu[j] < log_alpha) {
          x[j] = tx;
          y[j] = ty;
          z[j] = tz;
          co[j] = cn;
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

// ---------------------------------------------------------------------------
// Smart Monte Carlo step for even N <= 64 in the paired layout of
// pair_body.cuh: lane l holds the even particle 2l and the odd particle 2l+1
// of one chain; after the draws the pair is relabelled with the chain's
// set-order bit into A (moves in the first set) and B (second set), so that
// every lane moves one particle per set without divergent branches.  The move
// is the one of sweep_smc_kernel (same draws, same arithmetic per particle).
struct SmcSlot {
  float x, y, z;      // position
  float gx, gy, gz;   // standard normals
  float lnu;          // log of the acceptance uniform
  float w;            // omega at the old cell
  float fx, fy, fz;   // field force at the old cell
  uint32_t c;         // old cell
};

__device__ __forceinline__ SmcSlot smc_slot(const Geom& g, const float4* tab, float x, float y, float z,
                                            uint32_t m, uint32_t sweep, uint32_t ctr3a,
                                            bool valid, uint32_t* first_word) {
  SmcSlot q;
  q.x = x; q.y = y; q.z = z;
  // the old cell's table entry first: in flight during the draw and normals
  uint32_t cx, cy, cz;
  cell3(g, x, y, z, cx, cy, cz);
  q.c = (cz * (uint32_t)g.ny + cy) * (uint32_t)g.nx + cx;
  q.w = 0.f;
  q.fx = q.fy = q.fz = 0.f;
  if (valid) q.w = smc_field(tab, q.c, q.fx, q.fy, q.fz);
  const uint4 r1 = philox_rk(make_uint4(m, 0u, sweep, ctr3a), g);
  *first_word = r1.w;
  smc_normals(r1, q.gx, q.gy, q.gz);
  q.lnu = log_uniform_open(spare_uniform_word(r1));
  return q;
}

// One smart Monte Carlo move of M against the fixed partner sum
// U = sum (r - n) over its k bonded partners; returns acceptance.
__device__ __forceinline__ bool smc_move(const SweepArgs& p, const float4* tab, SmcSlot& M, float ux,
                                         float uy, float uz, float k, bool valid) {
  const float A = p.smc_A, s2A = p.smc_s2A, K2 = 2.f * p.K_b;
  const float Fx = fmaf(-K2, ux, M.fx), Fy = fmaf(-K2, uy, M.fy), Fz = fmaf(-K2, uz, M.fz);
  const float tx = __fadd_rn(M.x, fmaf(s2A, M.gx, A * Fx));
  const float ty = __fadd_rn(M.y, fmaf(s2A, M.gy, A * Fy));
  const float tz = __fadd_rn(M.z, fmaf(s2A, M.gz, A * Fz));
  uint32_t cx, cy, cz;
  cell3(p.g, tx, ty, tz, cx, cy, cz);
  const uint32_t cn = (cz * (uint32_t)p.g.ny + cy) * (uint32_t)p.g.nx + cx;
  float fnx = 0.f, fny = 0.f, fnz = 0.f, w_new = 0.f;
  if (valid) w_new = smc_field(tab, cn, fnx, fny, fnz);
  const float dx = tx - M.x, dy = ty - M.y, dz = tz - M.z;
  const float du = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
  const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float dE = fmaf(p.K_b, fmaf(2.f, du, k * dd), w_new - M.w);
  const float Gx = fmaf(-K2, fmaf(k, dx, ux), fnx), Gy = fmaf(-K2, fmaf(k, dy, uy), fny),
              Gz = fmaf(-K2, fmaf(k, dz, uz), fnz);
  const float ax = dx - A * Fx, ay = dy - A * Fy, az = dz - A * Fz;
  const float bx = -dx - A * Gx, by = -dy - A * Gy, bz = -dz - A * Gz;
  const float fwd = fmaf(ax, ax, fmaf(ay, ay, az * az));
  const float rev = fmaf(bx, bx, fmaf(by, by, bz * bz));
  const float log_alpha = fmaf(fwd - rev, p.smc_inv4A, -dE);
  const bool acc = valid && (log_alpha >= 0.f || M.lnu < log_alpha);
  M.x = acc ? tx : M.x;
  M.y = acc ? ty : M.y;
  M.z = acc ? tz : M.z;
  M.c = acc ? cn : M.c;
  return acc;
}

// Paired smart Monte Carlo sweep (even N <= 64).  One block of 24 warps per
// SM owns a contiguous range of tiles, which its warps take in order from a
// shared-memory counter, so all of them finish within a tile of each other.
__global__ void __launch_bounds__(768, 1) sweep_smc_pair_kernel(const SweepArgs p) {
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
  const uint32_t ctr3a = (PURPOSE_MOVE << 24) | (p.g.replica & 0xFFFFFFu);
  PairLane<float> L;
  L.init(lane, p.g.N, p.g.N_A, p.wA, p.wB);
  const float4* tab0 = p.smc_tab + (L.v0 == 1u ? 0u : p.g.cells);   // table plane of slot 0
  const float4* tab1 = p.smc_tab + (L.v1 == 1u ? 0u : p.g.cells);
  const uint32_t TN = p.G * p.g.N;
  unsigned my_acc = 0;
  // positions of the warp's next tile, loaded while the current one is moved
  float2 nx = make_float2(0.f, 0.f), ny = nx, nz = nx;
  auto load_pos = [&](uint32_t t) {
    if (t < t_end && (t < (uint32_t)p.full_tiles || L.li0 < p.last_rows)) {
      const uint32_t b = t * TN + L.li0;
      nx = __ldcs(reinterpret_cast<const float2*>(p.x + b));
      ny = __ldcs(reinterpret_cast<const float2*>(p.y + b));
      nz = __ldcs(reinterpret_cast<const float2*>(p.z + b));
    }
  };
  uint32_t tile = claim();
  load_pos(tile);
  while (tile < t_end) {
    const bool valid = tile < (uint32_t)p.full_tiles || L.li0 < p.last_rows;
    const uint32_t base = tile * TN + L.li0;
    float2 px = make_float2(0.f, 0.f), py = px, pz = px;
    if (valid) {
      px = nx;
      py = ny;
      pz = nz;
    }
    const uint32_t next_tile = claim();
    load_pos(next_tile);
    uint32_t w0, w1;
    const uint32_t cbase = base + (uint32_t)p.g.id_base;
    const SmcSlot s0 = smc_slot(p.g, tab0, px.x, py.x, pz.x, cbase, sweep, ctr3a, valid, &w0);
    const SmcSlot s1 = smc_slot(p.g, tab1, px.y, py.y, pz.y, cbase + 1u, sweep, ctr3a, valid, &w1);
    const bool sw = p.set_order_random && (__shfl_sync(FULL, w0, L.first_lane) & 1u);
    SmcSlot A = sw ? s1 : s0, B = sw ? s0 : s1;
    const float4* tA = sw ? tab1 : tab0;
    const float4* tB = sw ? tab0 : tab1;
    {  // first set: A moves against B and the adjacent lane's B
      const int src = sw ? L.src_next : L.src_prev;
      const float cf = sw ? L.cf_next1 : L.cf_prev0;
      const float sx = __shfl_sync(FULL, B.x, src);
      const float sy = __shfl_sync(FULL, B.y, src);
      const float sz = __shfl_sync(FULL, B.z, src);
      my_acc += smc_move(p, tA, A, fmaf(cf, A.x - sx, A.x - B.x), fmaf(cf, A.y - sy, A.y - B.y),
                             fmaf(cf, A.z - sz, A.z - B.z), 1.f + cf, valid);
    }
    {  // second set: B moves against A and the adjacent lane's A
      const int src = sw ? L.src_prev : L.src_next;
      const float cf = sw ? L.cf_prev0 : L.cf_next1;
      const float sx = __shfl_sync(FULL, A.x, src);
      const float sy = __shfl_sync(FULL, A.y, src);
      const float sz = __shfl_sync(FULL, A.z, src);
      my_acc += smc_move(p, tB, B, fmaf(cf, B.x - sx, B.x - A.x), fmaf(cf, B.y - sy, B.y - A.y),
                             fmaf(cf, B.z - sz, B.z - A.z), 1.f + cf, valid);
    }
    if (valid) {
      __stcs(reinterpret_cast<float2*>(p.x + base), sw ? make_float2(B.x, A.x) : make_float2(A.x, B.x));
      __stcs(reinterpret_cast<float2*>(p.y + base), sw ? make_float2(B.y, A.y) : make_float2(A.y, B.y));
      __stcs(reinterpret_cast<float2*>(p.z + base), sw ? make_float2(B.z, A.z) : make_float2(A.z, B.z));
      const uint32_t vA = sw ? L.v1 : L.v0, vB = sw ? L.v0 : L.v1;
      const bool same = A.c == B.c;
      atomicAdd(nacc + A.c, same ? vA + vB : vA);
      if (!same) atomicAdd(nacc + B.c, vB);
    }
    tile = next_tile;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_acc += __shfl_xor_sync(FULL, my_acc, o);
  if (lane == 0 && my_acc) atomicAdd(p.acc, (unsigned long long)my_acc);
}

const void* smc_kernel_ptr(int Q, bool pair, int /*grid_dtype: the table is FP32*/) {
  if (pair) return (const void*)sweep_smc_pair_kernel;
  return Q == 1 ? (const void*)sweep_smc_kernel<1>
                : (Q == 2 ? (const void*)sweep_smc_kernel<2> : (const void*)sweep_smc_kernel<4>);
}

}  // namespace soma
