// draws.cuh -- what the smart Monte Carlo and learned moves make of their
// Philox draws: the accurate ln of an open uniform, the phase of a uniform
// angle, the acceptance uniform from a draw's spare bits, and the three
// Box-Muller normals of a move (internal; the uniform move's transforms are
// in common.cuh).
#pragma once

#include "common.cuh"

namespace soma {

// log1p(f) for the reduced argument f in [sqrt(1/2) - 1, sqrt(2) - 1] by the
// series log(1 + f) = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...), s = f/(2 + f),
// |s| <= 3 - 2 sqrt(2) < 0.1716: five terms leave a truncation below s^10/11 <
// 5e-9 relative, under the FP32 rounding of the terms; s is the correctly
// rounded quotient of f and the rounded 2 + f (about one ulp).  Near f = 0 the
// result keeps the relative accuracy of f itself.
__device__ __forceinline__ float log1p_reduced(float f) {
  const float s = __fdiv_rn(f, 2.f + f);
  const float z = s * s;
  float t = fmaf(z, 0.111111111111111111f, 0.142857142857142857f);   // 1/9, 1/7
  t = fmaf(z, t, 0.2f);
  t = fmaf(z, t, 0.333333333333333333f);
  const float ss = s + s;
  return fmaf(ss * z, t, ss);
}

// ln of the open uniform u = (k + 1/2)/2^24, accurate to about one FP32 ulp of
// the result for every k, without a branch on k (a warp's lanes fall on both
// sides of u = 1/2 at random).  Below 1/2, u itself is exact in FP32; above,
// v = 1 - u = (2^24 - k - 1/2)/2^24 is exact instead.  Either is reduced to
// ln u = e ln 2 + log1p(f) with f = m - 1 exact and m in [sqrt(1/2), sqrt(2))
// (Cody and Waite's argument reduction): u = 2^e m from the exponent bits
// below 1/2; above, m = u (e = 0, f = -v) for u >= sqrt(1/2) and m = 2u
// (e = -1, f = 1 - 2v) below it.  ln 2 enters split in a part whose products
// with e are exact and a small correction.
__device__ __forceinline__ float log_uniform_open_accurate(uint32_t r) {
  const uint32_t k = r >> 8;
  const bool upper = k >= (1u << 23);
  const float u = fmaf(__uint2float_rn(k), 5.9604644775390625e-8f, 2.98023223876953125e-8f);
  const float v = fmaf(__uint2float_rn((1u << 24) - k), 5.9604644775390625e-8f,
                       -2.98023223876953125e-8f);
  // lower half: u = 2^e m, m in [1, 2), then halved into [sqrt(1/2), sqrt(2))
  const uint32_t b = __float_as_uint(u);
  float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
  int e = (int)(b >> 23) - 127;
  const bool halve = m >= 1.41421356237309505f;
  m = halve ? 0.5f * m : m;
  e += halve ? 1 : 0;
  // upper half: e = 0 above sqrt(1/2), else -1
  const bool e0 = v <= 0.29289321881345248f;   // 1 - sqrt(1/2)
  const float f = upper ? (e0 ? -v : fmaf(-2.f, v, 1.f)) : m - 1.f;
  const float ef = (float)(upper ? (e0 ? 0 : -1) : e);
  return fmaf(ef, 0.693145751953125f, fmaf(ef, 1.428606820309417232e-6f, log1p_reduced(f)));
}

// The 24 bits of a move draw r that its four top-24-bit uniforms leave over
// (the low bytes of words x, y, z; x's lowest), as the top 24 bits of a word:
// the acceptance uniform of a move whose four uniforms are all taken.
__device__ __forceinline__ uint32_t spare_uniform_word(const uint4& r) {
  return ((r.x & 0xFFu) | (r.y & 0xFFu) << 8 | (r.z & 0xFFu) << 16) << 8;
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

// The same with the hardware approximations (__sincosf of the phase reduced
// to [-pi, pi)): absolute error about 2^-21, for proposals whose acceptance
// uses the realised trial position rather than the draw.
__device__ __forceinline__ void sincos_2pi_uniform_fast(uint32_t r, float* s, float* c) {
  const float u = fmaf(__uint2float_rn(r >> 8), 5.9604644775390625e-8f, 2.98023223876953125e-8f);
  __sincosf(fmaf(6.2831853071795865f, u, -3.1415926535897932f), s, c);
  *s = -*s;
  *c = -*c;
}

// The three standard normals of a smart Monte Carlo move from its one draw r:
// Box-Muller of the uniforms of the top 24 bits of (x, y) and (z, w), the
// radius from the accurate log (a small absolute error of ln u near u = 1
// would be a large one of the radius), the angle by the hardware sincos.
__device__ __forceinline__ void smc_normals(const uint4& r, float& gx, float& gy, float& gz) {
  float sn, cs;
  const float rad0 = sqrtf(-2.f * log_uniform_open_accurate(r.x));
  sincos_2pi_uniform_fast(r.y, &sn, &cs);
  gx = rad0 * cs;
  gy = rad0 * sn;
  const float rad1 = sqrtf(-2.f * log_uniform_open_accurate(r.z));
  sincos_2pi_uniform_fast(r.w, &sn, &cs);
  gz = rad1 * cs;
}

}  // namespace soma
