/* mcmc32.c -- FP32 decision arithmetic of the sampler's random draws
 * (TEST INFRASTRUCTURE, part of the oracle; built into liboracle.so).
 *
 * The split and merge transitions of the codebook sampler (Sec. 4.4,
 * Appendix A.1) accept or reject a proposal by comparing a uniform draw with
 * min(1, e^(...)), where the exponent depends on Gaussian draws u.  An
 * accept/reject outcome is an integer result decided by floating point, so
 * the kernels and this oracle take it with the same written FP32 operation
 * order: Box-Muller (1958) normals from 24-bit uniforms, with a logarithm
 * and a sine/cosine of 2 pi u built only from IEEE-754 binary32 +, -, *, /,
 * sqrt and fused multiply-add.  The uniform bits come from Philox4x32-10
 * (Salmon et al., SC'11), which the Python side of the oracle implements.
 *
 * Every operation below is one IEEE binary32 operation rounded to nearest
 * (compiled with contraction off); fmaf is the IEEE fused multiply-add. */
#include <math.h>
#include <stdint.h>

float or_e32(float x); /* oracle.c */

static float bits_to_float(uint32_t u) {
  union { uint32_t u; float f; } c;
  c.u = u;
  return c.f;
}

static uint32_t float_to_bits(float f) {
  union { uint32_t u; float f; } c;
  c.f = f;
  return c.u;
}

/* Natural logarithm of a positive normal binary32 value: x = m 2^e with m
 * in [sqrt(1/2), sqrt(2)), log m = 2 atanh(s) with s = (m - 1) / (m + 1),
 * the atanh series to s^11 (|s| <= 0.1716: truncation below 1e-10 relative),
 * then e ln 2 added with ln 2 split into a 15-bit head and the remainder. */
float or_log32(float x) {
  const uint32_t b = float_to_bits(x);
  int e = (int)(b >> 23) - 127;
  float m = bits_to_float((b & 0x007fffffu) | 0x3f800000u);
  if (m > 1.41421353816986083984375f) {
    m = m * 0.5f;
    e = e + 1;
  }
  const float s = (m - 1.0f) / (m + 1.0f);
  const float z = s * s;
  float p = 1.0f / 11.0f;
  p = fmaf(p, z, 1.0f / 9.0f);
  p = fmaf(p, z, 1.0f / 7.0f);
  p = fmaf(p, z, 1.0f / 5.0f);
  p = fmaf(p, z, 1.0f / 3.0f);
  p = fmaf(p, z, 1.0f);
  const float lm = (s + s) * p;
  const float fe = (float)e;
  const float ln2_hi = 0.693145751953125f;
  const float ln2_lo = 1.42860682030941723212e-6f;
  return fmaf(fe, ln2_hi, fmaf(fe, ln2_lo, lm));
}

/* sin and cos of 2 pi u for u in [0, 1): quadrant q = floor(4u) and the
 * fraction f = 4u - q (both exact), the angle (pi/2) g with g = min(f, 1 - f)
 * in [0, 1/2], Taylor polynomials of sin to x^9 and cos to x^10 (|x| <= pi/4),
 * then the quadrant's signs and swaps. */
void or_sincos2pi32(float u, float *s_out, float *c_out) {
  const float t = u * 4.0f;
  const int q = (int)t;
  const float f = t - (float)q;
  const int sw = f > 0.5f;
  const float g = sw ? 1.0f - f : f;
  const float x = g * 1.57079632679489661923f;
  const float x2 = x * x;
  float ps = 1.0f / 362880.0f;
  ps = fmaf(ps, x2, -1.0f / 5040.0f);
  ps = fmaf(ps, x2, 1.0f / 120.0f);
  ps = fmaf(ps, x2, -1.0f / 6.0f);
  ps = fmaf(ps, x2, 1.0f);
  const float sn = x * ps;
  float pc = -1.0f / 3628800.0f;
  pc = fmaf(pc, x2, 1.0f / 40320.0f);
  pc = fmaf(pc, x2, -1.0f / 720.0f);
  pc = fmaf(pc, x2, 1.0f / 24.0f);
  pc = fmaf(pc, x2, -0.5f);
  const float cs = fmaf(pc, x2, 1.0f);
  const float s0 = sw ? cs : sn, c0 = sw ? sn : cs;
  switch (q & 3) {
    case 0: *s_out = s0; *c_out = c0; break;
    case 1: *s_out = c0; *c_out = -s0; break;
    case 2: *s_out = -s0; *c_out = -c0; break;
    default: *s_out = -c0; *c_out = s0; break;
  }
}

/* Uniform in [0, 1) from the top 24 bits of a draw. */
float or_uniform32(uint32_t a) { return (float)(a >> 8) * 5.9604644775390625e-8f; }

/* Two standard normals from two 32-bit draws (Box-Muller): u1 in (0, 1]
 * from the first, u2 in [0, 1) from the second, r = sqrt(-2 log u1),
 * z0 = r cos(2 pi u2), z1 = r sin(2 pi u2). */
void or_normal_pair32(uint32_t a, uint32_t b, float *z0, float *z1) {
  const float u1 = (float)((a >> 8) + 1u) * 5.9604644775390625e-8f;
  const float u2 = (float)(b >> 8) * 5.9604644775390625e-8f;
  const float r = sqrtf(-2.0f * or_log32(u1));
  float s, c;
  or_sincos2pi32(u2, &s, &c);
  *z0 = r * c;
  *z1 = r * s;
}

/* Batches for the Python side: bits holds count x 4 Philox outputs; z gets
 * the four normals of each (pairs (0, 1) and (2, 3)). */
void or_normals32(int64_t count, const uint32_t *bits, float *z) {
  for (int64_t i = 0; i < count; ++i) {
    or_normal_pair32(bits[4 * i], bits[4 * i + 1], z + 4 * i, z + 4 * i + 1);
    or_normal_pair32(bits[4 * i + 2], bits[4 * i + 3], z + 4 * i + 2, z + 4 * i + 3);
  }
}

void or_log32_batch(int64_t count, const float *x, float *y) {
  for (int64_t i = 0; i < count; ++i) y[i] = or_log32(x[i]);
}

void or_sincos2pi32_batch(int64_t count, const float *u, float *s, float *c) {
  for (int64_t i = 0; i < count; ++i) or_sincos2pi32(u[i], s + i, c + i);
}

void or_e32_batch(int64_t count, const float *x, float *y) {
  for (int64_t i = 0; i < count; ++i) y[i] = or_e32(x[i]);
}
