// cg_random.cuh -- counter-based random draws of the sampler transitions.
//
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): a 128-bit counter and a 64-bit key give four
// 32-bit outputs, so every draw is a pure function of (seed, step, stream,
// index) and any thread can produce any draw without state.
//
// Standard normals are Box-Muller pairs (1958).  Split and merge decisions
// depend on them, so the normals are part of the decision arithmetic: a
// written binary32 operation order (IEEE +, -, *, /, sqrt and fmaf only,
// compiled with -fmad=false) for the logarithm and for sin / cos of 2 pi u.
#pragma once

#include "cg_common.cuh"

namespace cg {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

// Draw streams (counter word c1 = stream | call << 8).
constexpr uint32_t kStreamPos = 0, kStreamLogit = 1, kStreamSR = 2, kStreamSH = 3;
constexpr uint32_t kStreamSplitU = 16, kStreamSplitV = 18, kStreamMerge = 20, kStreamGrow = 24;

// Ten rounds; each maps (c0, c1, c2, c3) under key (k0, k1) to
// (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)), and the
// key advances by (W0, W1) before every round but the first.
CG_HD uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c.x;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
  }
  return c;
}

// Draws for counter (index, stream | call << 8, step low, step high), key = seed.
CG_HD uint4 draw4(uint32_t index, uint32_t stream, uint32_t call, uint64_t step, uint64_t seed) {
  return philox4x32_10(make_uint4(index, stream | (call << 8), (uint32_t)step, (uint32_t)(step >> 32)),
                       (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Uniform in [0, 1) from the top 24 bits of a draw (exact).
CG_HD float uniform24(uint32_t a) { return (float)(a >> 8) * 5.9604644775390625e-8f; }

// Natural log of a positive normal binary32 value (decision arithmetic):
// x = m 2^e with m in [sqrt(1/2), sqrt(2)), log m = 2 atanh(s),
// s = (m - 1) / (m + 1), the atanh series through s^11 by Horner's rule in
// z = s^2, then e ln 2 added with ln 2 as a 15-bit head plus remainder.
CG_HD float log32(float x) {
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
  return fmaf(fe, 0.693145751953125f, fmaf(fe, 1.42860682030941723212e-6f, lm));
}

// sin and cos of 2 pi u, u in [0, 1) (decision arithmetic): quadrant
// q = floor(4u), fraction f = 4u - q, angle (pi/2) g with g = min(f, 1 - f),
// Taylor polynomials of sin (to x^9) and cos (to x^10) on [0, pi/4], then
// the swap for f > 1/2 and the quadrant's signs.
CG_HD void sincos2pi32(float u, float* s_out, float* c_out) {
  const float t = u * 4.0f;
  const int q = (int)t;
  const float f = t - (float)q;
  const bool sw = f > 0.5f;
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

// Box-Muller: u1 = ((a >> 8) + 1) 2^-24 in (0, 1], u2 = (b >> 8) 2^-24,
// r = sqrt(-2 log u1), (z0, z1) = (r cos 2 pi u2, r sin 2 pi u2).
CG_HD float2 normal_pair(uint32_t a, uint32_t b) {
  const float u1 = (float)((a >> 8) + 1u) * 5.9604644775390625e-8f;
  const float u2 = (float)(b >> 8) * 5.9604644775390625e-8f;
  const float r = sqrtf(-2.0f * log32(u1));
  float s, c;
  sincos2pi32(u2, &s, &c);
  return make_float2(r * c, r * s);
}

// Four normals of one draw: pairs (x, y) and (z, w).
CG_HD float4 normal4(uint4 d) {
  const float2 a = normal_pair(d.x, d.y);
  const float2 b = normal_pair(d.z, d.w);
  return make_float4(a.x, a.y, b.x, b.y);
}

// Coefficients of the split / merge acceptance (decision arithmetic):
// log q_sm(u) = -|u|^2 kc with kc = (1/eps_split^2 - 1/eps_merge^2) / 2, and
// the merge proposal kernel exp(-|c - c'|^2 km) with km = 1 / (2 eps_merge^2).
struct MhCoef {
  float es, kc, km;
};
CG_HD MhCoef mh_coef(float eps_split, float eps_merge) {
  const float inv_s = 1.0f / (eps_split * eps_split);
  const float inv_m = 1.0f / (eps_merge * eps_merge);
  MhCoef c;
  c.es = eps_split;
  c.kc = 0.5f * (inv_s - inv_m);
  c.km = 0.5f * inv_m;
  return c;
}

// ---------------------------------------------------------------------------
// launch arguments of k_mcmc.cu
// ---------------------------------------------------------------------------

// One tensor of the parameter update: x (count values of float or bf16,
// updated in place), its gradient g (float), a = -eps/2, b = sqrt(eps).
struct SgldSeg {
  void* x;
  const float* g;
  int64_t count;
  float a, b;
  uint32_t stream;
  int bf16;   // x holds bfloat16
  int vec;    // x is 16-byte (float) / 8-byte (bf16) aligned: 4 values per access
  int gvec;   // g is 16-byte aligned
  int skip7;  // rows of 8 with the last value fixed (SR rows)
};
struct SgldArgs {
  SgldSeg seg[4];
  int64_t calls[4];  // draws per tensor, ceil(count / 4)
  uint64_t seed, step;
};

struct MhArgs {
  int codebook;  // 0 SR, 1 SH
  int n, k, k_cap;
  int dims, width, dtype;
  float lam;
  MhCoef coef;
  uint64_t seed, step;
  void* rows;
  int32_t* parent;
  uint16_t* g2x;
  int32_t* k_out;
};

// Byte offsets of the split / merge workspace.
struct MhLayout {
  uint64_t hdr, members, first, flags, scan, target, rows_copy, parent_copy, blocksums, total;
  int64_t scan_blocks_cap;
};

// Growth: m copies appended after the n Gaussians (arrays hold n + m).
struct GrowArgs {
  int64_t n, m;
  float* pos;
  float* logit;
  uint16_t* g2sr;
  uint16_t* g2sh;
  int32_t* src_out;
  uint64_t seed, step;
};

uint64_t grow_workspace_bytes(int64_t n);
cudaError_t launch_grow(const GrowArgs& a, void* ws, cudaStream_t s);
MhLayout mh_layout(int n, int k_cap, int width);
cudaError_t launch_sgld(const SgldArgs& a, cudaStream_t s);
cudaError_t launch_split(const MhArgs& a, const MhLayout& M, void* ws, cudaStream_t s);
cudaError_t launch_merge(const MhArgs& a, const MhLayout& M, void* ws, cudaStream_t s);

}  // namespace cg
