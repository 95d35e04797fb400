// pair_body.cuh -- one tile of the paired SET sweep (even N <= 64), shared by
// the single-system kernel (sweep.cu) and the batched kernel (batch.cu).
//
// Lane l of a tile holds particles 2l (even chain position, slot 0) and 2l+1
// (odd, slot 1) of the SAME chain.  Each SET phase moves exactly one of the
// two, so every lane does one move per phase with no predicated duplicate
// work.  After the draws the pair is re-labelled once per tile into A (moves
// in the first phase) and B (moves in the second) with the chain's set-order
// bit, so the phases need no selects:
//   phase 1 moves A; its bond partners are B (same lane) and the adjacent
//     lane's B (lane-1 if A is the even particle, lane+1 if it is odd);
//   phase 2 moves B; its partners are A (same lane, already updated) and the
//     adjacent lane's A (lane+1 if B is odd, lane-1 if it is even).
// Bond energy change of a move r -> r + d with k partners n:
//   sum_n |r+d-n|^2 - |r-n|^2 = 2 d.U + k d.d,  U = sum_n (r - n),
// where every difference r - n is exact for bonded neighbours.
#pragma once

#include "common.cuh"

namespace soma {

// Per-lane constants of one system (depend on N and the lane only).
template <typename WT>
struct PairLane {
  int lane, first_lane;
  bool has_prev0, has_next1;
  float cf_prev0, cf_next1;     // the same as 1.f / 0.f
  int src_prev, src_next;       // lane - 1, lane + 1 (mod 32)
  const WT* w0;
  const WT* w1;
  uint32_t v0, v1;
  uint32_t li0;
  uint32_t ci0;         // chain position of slot 0
  uint32_t lane_chain;  // chain of this lane within the tile

  __device__ __forceinline__ void init(int lane_, uint32_t N, uint32_t N_A, const void* wA,
                                       const void* wB) {
    lane = lane_;
    li0 = 2u * (uint32_t)lane;
    ci0 = li0 % N;                                // chain position of slot 0 (even)
    lane_chain = li0 / N;
    first_lane = (int)((li0 - ci0) >> 1);         // lane holding the chain's particle 0
    has_prev0 = ci0 > 0u;                         // slot 0 has a partner in lane-1
    has_next1 = ci0 + 2u < N;                     // slot 1 has a partner in lane+1
    cf_prev0 = has_prev0 ? 1.f : 0.f;
    cf_next1 = has_next1 ? 1.f : 0.f;
    src_prev = (lane - 1) & 31;
    src_next = (lane + 1) & 31;
    set_types(ci0 >= N_A, ci0 + 1u >= N_A, wA, wB);
  }

  // Types of the two slots (true: B): field planes and count increments.
  __device__ __forceinline__ void set_types(bool b0, bool b1, const void* wA, const void* wB) {
    w0 = static_cast<const WT*>(b0 ? wB : wA);
    w1 = static_cast<const WT*>(b1 ? wB : wA);
    v0 = b0 ? 0x10000u : 1u;
    v1 = b1 ? 0x10000u : 1u;
  }
};

// One tile of the paired sweep in two stages, so that a warp can issue the
// field gathers of its next tile before it finishes the current one:
//   pair_prepare: the draws of the pair (particles base and base+1, counter
//     indices cbase and cbase+1), its trial positions and the cells of the old
//     and trial positions, and the loads of the four field values (issued
//     here, used in pair_finish);
//   pair_finish: the acceptance uniforms, the chain's set order, both SET
//     phases, the stores and the occupation count.
// pair_tile runs both back to back.  valid says whether this lane's pair
// exists (the tile may hold fewer rows than lanes).
//
// Exactness notes: a missing bond partner enters as 0 * (A - s) with a finite
// s, i.e. as an exact zero; the acceptance test is dE <= -ln u, which is the
// rule "dE <= 0 or ln u < -dE" for every ln u < 0 except on the measure-zero
// set dE = -ln u.
struct PairState {
  float x0, x1, y0, y1, z0, z1;        // positions
  float xn0, xn1, yn0, yn1, zn0, zn1;  // trial positions
  uint32_t c0, c1, cn0, cn1;           // old and trial cells
  float wn0, wo0, wn1, wo1;            // omega at the trial and old cells
  uint32_t u0, u1;                     // draw words of the acceptance uniforms
  bool valid;
};

template <typename WT, typename IDX, bool WIDE>
__device__ __forceinline__ void pair_prepare(const Geom& g, const Geom& keys, const PairLane<WT>& L,
                                             IDX cbase, bool valid, uint32_t sweep, uint32_t ctr3,
                                             float a, float x0, float x1, float y0, float y1,
                                             float z0, float z1, PairState& P) {
  // the old cells and their field values first: they wait on nothing but the
  // positions, so the gathers are in flight during the draws
  const unsigned long long MAG = f2_pack(12582912.0f, 12582912.0f);
  const unsigned long long X = f2_pack(x0, x1), Y = f2_pack(y0, y1), Z = f2_pack(z0, z1);
  float fx0, fx1, fy0, fy1, fz0, fz1, gx0, gx1, gy0, gy1, gz0, gz1;
  f2_unpack(f2_add_rm(X, MAG), fx0, fx1);
  f2_unpack(f2_add_rm(Y, MAG), fy0, fy1);
  f2_unpack(f2_add_rm(Z, MAG), fz0, fz1);
  P.c0 = cell_of_floor_bits<WIDE>(g, __float_as_uint(fx0), __float_as_uint(fy0), __float_as_uint(fz0));
  P.c1 = cell_of_floor_bits<WIDE>(g, __float_as_uint(fx1), __float_as_uint(fy1), __float_as_uint(fz1));
  P.wo0 = P.wo1 = 0.f;
  if (valid) {
    P.wo0 = load_w<WT>(L.w0, P.c0);
    P.wo1 = load_w<WT>(L.w1, P.c1);
  }
  const uint32_t hi = sizeof(IDX) > 4 ? (uint32_t)((uint64_t)cbase >> 32) : 0u;
  const uint4 r0 = philox_rk(make_uint4((uint32_t)cbase, hi, sweep, ctr3), keys);
  const IDX m1 = cbase + 1u;
  const uint32_t hi1 = sizeof(IDX) > 4 ? (uint32_t)((uint64_t)m1 >> 32) : 0u;
  const uint4 r1 = philox_rk(make_uint4((uint32_t)m1, hi1, sweep, ctr3), keys);
  // Both slots at once with the packed FP32x2 instructions: the symmetric
  // uniforms k 2^-23 + (2^-24 - 1) (one rounding), the trial positions
  // r + a v (one rounding, a fused multiply-add), and the floor bits of the
  // cell fold (sum with 1.5 2^23 rounded toward -inf) -- bit for bit the
  // scalar arithmetic of uniform_sym, __fmaf_rn and fold_raw.
  const unsigned long long S = f2_pack(1.1920928955078125e-7f, 1.1920928955078125e-7f);
  const unsigned long long C = f2_pack(-0.99999994039535522461f, -0.99999994039535522461f);
  const unsigned long long A2 = f2_pack(a, a);
  const unsigned long long XN = f2_fma_rn(
      A2, f2_fma_rn(f2_pack(__uint2float_rn(r0.x >> 8), __uint2float_rn(r1.x >> 8)), S, C), X);
  const unsigned long long YN = f2_fma_rn(
      A2, f2_fma_rn(f2_pack(__uint2float_rn(r0.y >> 8), __uint2float_rn(r1.y >> 8)), S, C), Y);
  const unsigned long long ZN = f2_fma_rn(
      A2, f2_fma_rn(f2_pack(__uint2float_rn(r0.z >> 8), __uint2float_rn(r1.z >> 8)), S, C), Z);
  f2_unpack(XN, P.xn0, P.xn1);
  f2_unpack(YN, P.yn0, P.yn1);
  f2_unpack(ZN, P.zn0, P.zn1);
  f2_unpack(f2_add_rm(XN, MAG), gx0, gx1);
  f2_unpack(f2_add_rm(YN, MAG), gy0, gy1);
  f2_unpack(f2_add_rm(ZN, MAG), gz0, gz1);
  P.cn0 = cell_of_floor_bits<WIDE>(g, __float_as_uint(gx0), __float_as_uint(gy0), __float_as_uint(gz0));
  P.cn1 = cell_of_floor_bits<WIDE>(g, __float_as_uint(gx1), __float_as_uint(gy1), __float_as_uint(gz1));
  P.wn0 = P.wn1 = 0.f;
  if (valid) {
    P.wn0 = load_w<WT>(L.w0, P.cn0);
    P.wn1 = load_w<WT>(L.w1, P.cn1);
  }
  P.x0 = x0; P.x1 = x1; P.y0 = y0; P.y1 = y1; P.z0 = z0; P.z1 = z1;
  P.u0 = r0.w;
  P.u1 = r1.w;
  P.valid = valid;
}

// Returns this lane's accepted moves.
template <typename WT, typename IDX>
__device__ __forceinline__ unsigned pair_finish(const PairLane<WT>& L, float* __restrict__ px,
                                                float* __restrict__ py, float* __restrict__ pz,
                                                uint32_t* __restrict__ nacc, IDX base,
                                                const PairState& P, bool set_order_random,
                                                float K1) {
  const bool valid = P.valid;
  const float K2 = 2.f * K1;
  const float x0 = P.x0, x1 = P.x1, y0 = P.y0, y1 = P.y1, z0 = P.z0, z1 = P.z1;
  const float xn0 = P.xn0, xn1 = P.xn1, yn0 = P.yn0, yn1 = P.yn1, zn0 = P.zn0, zn1 = P.zn1;
  const uint32_t c0 = P.c0, c1 = P.c1, cn0 = P.cn0, cn1 = P.cn1;
  const float dEf0 = P.wn0 - P.wo0, dEf1 = P.wn1 - P.wo1;
  float lnu0, lnu1;
  {  // ln of the open uniforms (k + 1/2) 2^-24 of both slots
    float u0, u1;
    f2_unpack(f2_fma_rn(f2_pack(__uint2float_rn(P.u0 >> 8), __uint2float_rn(P.u1 >> 8)),
                        f2_pack(5.9604644775390625e-8f, 5.9604644775390625e-8f),
                        f2_pack(2.98023223876953125e-8f, 2.98023223876953125e-8f)), u0, u1);
    lnu0 = __logf(u0);
    lnu1 = __logf(u1);
  }
  const bool sw = set_order_random && (__shfl_sync(FULL, P.u0, L.first_lane) & 1u);

  // A moves first, B second.
  float Ax = sw ? x1 : x0, Ay = sw ? y1 : y0, Az = sw ? z1 : z0;
  float Bx = sw ? x0 : x1, By = sw ? y0 : y1, Bz = sw ? z0 : z1;
  const float tAx = sw ? xn1 : xn0, tAy = sw ? yn1 : yn0, tAz = sw ? zn1 : zn0;
  const float tBx = sw ? xn0 : xn1, tBy = sw ? yn0 : yn1, tBz = sw ? zn0 : zn1;
  uint32_t cA = sw ? c1 : c0, cB = sw ? c0 : c1;
  const uint32_t cnA = sw ? cn1 : cn0, cnB = sw ? cn0 : cn1;
  const float fA = sw ? dEf1 : dEf0, fB = sw ? dEf0 : dEf1;
  const float lA = sw ? lnu1 : lnu0, lB = sw ? lnu0 : lnu1;
  unsigned acc_count = 0;

  {  // first set: A moves against B and the adjacent lane's B
    const int src = sw ? L.src_next : L.src_prev;
    const float cf = sw ? L.cf_next1 : L.cf_prev0;
    const float sx = __shfl_sync(FULL, Bx, src);
    const float sy = __shfl_sync(FULL, By, src);
    const float sz = __shfl_sync(FULL, Bz, src);
    const float dx = tAx - Ax, dy = tAy - Ay, dz = tAz - Az;
    const float ux = fmaf(cf, Ax - sx, Ax - Bx);
    const float uy = fmaf(cf, Ay - sy, Ay - By);
    const float uz = fmaf(cf, Az - sz, Az - Bz);
    const float du = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
    const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float dE = fmaf(fmaf(cf, K1, K1), dd, fmaf(K2, du, fA));
    const bool acc = valid && dE <= -lA;
    Ax = acc ? tAx : Ax;
    Ay = acc ? tAy : Ay;
    Az = acc ? tAz : Az;
    cA = acc ? cnA : cA;
    acc_count += acc;
  }
  {  // second set: B moves against A and the adjacent lane's A
    const int src = sw ? L.src_prev : L.src_next;
    const float cf = sw ? L.cf_prev0 : L.cf_next1;
    const float sx = __shfl_sync(FULL, Ax, src);
    const float sy = __shfl_sync(FULL, Ay, src);
    const float sz = __shfl_sync(FULL, Az, src);
    const float dx = tBx - Bx, dy = tBy - By, dz = tBz - Bz;
    const float ux = fmaf(cf, Bx - sx, Bx - Ax);
    const float uy = fmaf(cf, By - sy, By - Ay);
    const float uz = fmaf(cf, Bz - sz, Bz - Az);
    const float du = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
    const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float dE = fmaf(fmaf(cf, K1, K1), dd, fmaf(K2, du, fB));
    const bool acc = valid && dE <= -lB;
    Bx = acc ? tBx : Bx;
    By = acc ? tBy : By;
    Bz = acc ? tBz : Bz;
    cB = acc ? cnB : cB;
    acc_count += acc;
  }

  if (valid) {
    __stcs(reinterpret_cast<float2*>(px + base), sw ? make_float2(Bx, Ax) : make_float2(Ax, Bx));
    __stcs(reinterpret_cast<float2*>(py + base), sw ? make_float2(By, Ay) : make_float2(Ay, By));
    __stcs(reinterpret_cast<float2*>(pz + base), sw ? make_float2(Bz, Az) : make_float2(Az, Bz));
    // one atomic when both end in the same cell, else one each
    const uint32_t vA = sw ? L.v1 : L.v0, vB = sw ? L.v0 : L.v1;
    const bool same = cA == cB;
    atomicAdd(nacc + cA, same ? vA + vB : vA);
    if (!same) atomicAdd(nacc + cB, vB);
  }
  return acc_count;
}

template <typename WT, typename IDX, bool PARTIAL, bool WIDE>
__device__ __forceinline__ unsigned pair_tile(const Geom& g, const Geom& keys, const PairLane<WT>& L,
                                              float* __restrict__ px, float* __restrict__ py,
                                              float* __restrict__ pz, uint32_t* __restrict__ nacc,
                                              IDX base, IDX cbase, bool valid, uint32_t sweep,
                                              uint32_t ctr3, bool set_order_random, float a,
                                              float K1, float x0, float x1, float y0, float y1,
                                              float z0, float z1) {
  PairState P;
  pair_prepare<WT, IDX, WIDE>(g, keys, L, cbase, PARTIAL ? valid : true, sweep, ctr3, a, x0, x1, y0,
                              y1, z0, z1, P);
  return pair_finish<WT, IDX>(L, px, py, pz, nacc, base, P, set_order_random, K1);
}

}  // namespace soma
