// Even-odd Wilson stencils with two right-hand sides per thread (the iteration's V and T steps in
// FP16 / BF16 / FP32 storage with FP32 arithmetic).
//
// The two right-hand sides of a thread (slots A and B of one lattice, same site) sit in the two
// lanes of the packed FP32x2 instructions of sm_100+ (fma.rn.f32x2 and friends): every link
// element is loaded and converted once for both and enters the SU(3) products as a broadcast
// pair, so one packed instruction does the work of two scalar ones.  The spin projection of a
// half-precision neighbour takes one conversion and one mixed-precision add (add.f32.f16: a
// binary16 operand plus an FP32 one, result FP32) per real, instead of two conversions and an add.
// The blocks of all slot pairs of a tile are launched next to each other (grid x = slot pairs),
// so a tile's links come from DRAM once per launch instead of once per group of slots.
#pragma once

typedef float2 f2;

__device__ __forceinline__ f2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }

// a complex number of each lane: re = (re_A, re_B), im = (im_A, im_B)
struct c2 {
  f2 re, im;
};

// ---------------------------------------------------------------- storage words
// One spinor as stored (12 complex): FP16 / BF16 as 6 words of two binary16 (re, im) plus the
// per-site norm; FP32 as 12 (re, im) float pairs.
template <int SPR>
struct Raw2;
template <int PR>
struct RawHalf {
  uint4 c[3];
  float n;
  __device__ __forceinline__ void load(FieldPtr f, int Vmax, int slot, int h) {
    const uint4* b = (const uint4*)f.p + (size_t)slot * 3 * Vmax + h;
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = __ldg(b + (size_t)k * Vmax);
    n = __ldg(f.nrm + (size_t)slot * Vmax + h);
  }
  __device__ __forceinline__ unsigned word(int idx) const {   // complex component idx = 3 spin + colour
    const uint4& q = c[idx % 3];                               // chunk = colour, word = spin
    const int j = idx / 3;
    return j == 0 ? q.x : j == 1 ? q.y : j == 2 ? q.z : q.w;
  }
  // real and imaginary part in FP32
  __device__ __forceinline__ float re(int idx) const;
  __device__ __forceinline__ float im(int idx) const;
  // x + b with x the real (imaginary) part of component idx kept in binary16: one mixed add
  __device__ __forceinline__ float re_add(int idx, float b) const;
  __device__ __forceinline__ float re_sub(int idx, float b) const;
  __device__ __forceinline__ float im_add(int idx, float b) const;
  __device__ __forceinline__ float im_sub(int idx, float b) const;
};

// binary16: conversion as h + 0 and add / sub.rn.f32.f16 on the halves of the 32-bit word (all at the
// full FP32 rate)
template <>
__device__ __forceinline__ float RawHalf<PR16>::re(int idx) const {
  return h16lo_to_f32(word(idx));
}
template <>
__device__ __forceinline__ float RawHalf<PR16>::im(int idx) const {
  return h16hi_to_f32(word(idx));
}
template <>
__device__ __forceinline__ float RawHalf<PR16>::re_add(int idx, float b) const {
  float r;
  asm("{.reg .f16 l, h; mov.b32 {l, h}, %1; add.rn.f32.f16 %0, l, %2;}" : "=f"(r) : "r"(word(idx)), "f"(b));
  return r;
}
template <>
__device__ __forceinline__ float RawHalf<PR16>::re_sub(int idx, float b) const {
  float r;
  asm("{.reg .f16 l, h; mov.b32 {l, h}, %1; sub.rn.f32.f16 %0, l, %2;}" : "=f"(r) : "r"(word(idx)), "f"(b));
  return r;
}
template <>
__device__ __forceinline__ float RawHalf<PR16>::im_add(int idx, float b) const {
  float r;
  asm("{.reg .f16 l, h; mov.b32 {l, h}, %1; add.rn.f32.f16 %0, h, %2;}" : "=f"(r) : "r"(word(idx)), "f"(b));
  return r;
}
template <>
__device__ __forceinline__ float RawHalf<PR16>::im_sub(int idx, float b) const {
  float r;
  asm("{.reg .f16 l, h; mov.b32 {l, h}, %1; sub.rn.f32.f16 %0, h, %2;}" : "=f"(r) : "r"(word(idx)), "f"(b));
  return r;
}
// bfloat16: the upper half of an FP32 number, so a conversion is a shift or a mask
template <>
__device__ __forceinline__ float RawHalf<PRB16>::re(int idx) const { return __uint_as_float(word(idx) << 16); }
template <>
__device__ __forceinline__ float RawHalf<PRB16>::im(int idx) const {
  return __uint_as_float(word(idx) & 0xffff0000u);
}
template <>
__device__ __forceinline__ float RawHalf<PRB16>::re_add(int idx, float b) const {
  float r;
  asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; add.rn.f32.bf16 %0, l, %2;}" : "=f"(r) : "r"(word(idx)), "f"(b));
  return r;
}
template <>
__device__ __forceinline__ float RawHalf<PRB16>::re_sub(int idx, float b) const {
  float r;
  asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; sub.rn.f32.bf16 %0, l, %2;}" : "=f"(r) : "r"(word(idx)), "f"(b));
  return r;
}
template <>
__device__ __forceinline__ float RawHalf<PRB16>::im_add(int idx, float b) const {
  float r;
  asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; add.rn.f32.bf16 %0, h, %2;}" : "=f"(r) : "r"(word(idx)), "f"(b));
  return r;
}
template <>
__device__ __forceinline__ float RawHalf<PRB16>::im_sub(int idx, float b) const {
  float r;
  asm("{.reg .b16 l, h; mov.b32 {l, h}, %1; sub.rn.f32.bf16 %0, h, %2;}" : "=f"(r) : "r"(word(idx)), "f"(b));
  return r;
}
template <>
struct Raw2<PR16> : RawHalf<PR16> {};
template <>
struct Raw2<PRB16> : RawHalf<PRB16> {};

template <>
struct Raw2<PR32> {
  float4 c[6];
  float n;
  __device__ __forceinline__ void load(FieldPtr f, int Vmax, int slot, int h) {
    const float4* b = (const float4*)f.p + (size_t)slot * 6 * Vmax + h;
#pragma unroll
    for (int k = 0; k < 6; ++k) c[k] = __ldg(b + (size_t)k * Vmax);
    n = 1.0f;
  }
  __device__ __forceinline__ float re(int idx) const { return (idx & 1) ? c[idx >> 1].z : c[idx >> 1].x; }
  __device__ __forceinline__ float im(int idx) const { return (idx & 1) ? c[idx >> 1].w : c[idx >> 1].y; }
  __device__ __forceinline__ float re_add(int idx, float b) const { return re(idx) + b; }
  __device__ __forceinline__ float re_sub(int idx, float b) const { return re(idx) - b; }
  __device__ __forceinline__ float im_add(int idx, float b) const { return im(idx) + b; }
  __device__ __forceinline__ float im_sub(int idx, float b) const { return im(idx) - b; }
};

// the canonical component (3 spin + colour) of word j of 16-byte chunk k of a stored spinor:
// FP32 chunks hold components 4k .. 4k+3, binary16 / bfloat16 chunks colour k of spins 0-3
template <int SPR>
__device__ __forceinline__ constexpr int chunk_comp(int k, int j) {
  return SPR == PR32 ? 4 * k + j : 3 * j + k;
}

// the four (re, im) binary16 / bfloat16 pairs of one 16-byte chunk in FP32
template <int SPR>
__device__ __forceinline__ void chunk_words(const uint4& q, float (&re)[4], float (&im)[4]) {
  const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 v = Half2Ops<SPR>::to_f2(w[j]);
    re[j] = v.x;
    im[j] = v.y;
  }
}

// words 0-3 of chunk k (FP32: chunks 2k, 2k+1) of a stored spinor in FP32, without the per-site
// norm: the components chunk_comp<SPR>(k, 0..3)
template <int SPR>
__device__ __forceinline__ void load_comp4(FieldPtr f, int Vmax, int slot, int h, int k, float (&re)[4],
                                           float (&im)[4]) {
  if constexpr (SPR == PR32) {
    const float4* b = (const float4*)f.p + (size_t)slot * 6 * Vmax + h;
    const float4 u = __ldg(b + (size_t)(2 * k) * Vmax), v = __ldg(b + (size_t)(2 * k + 1) * Vmax);
    re[0] = u.x, im[0] = u.y, re[1] = u.z, im[1] = u.w, re[2] = v.x, im[2] = v.y, re[3] = v.z, im[3] = v.w;
  } else {
    const uint4 q = __ldg((const uint4*)f.p + ((size_t)slot * 3 + k) * Vmax + h);
    chunk_words<SPR>(q, re, im);
  }
}
template <int SPR>
__device__ __forceinline__ float load_norm(FieldPtr f, int Vmax, int slot, int h) {
  if constexpr (SPR == PR32) return 1.0f;
  else return __ldg(f.nrm + (size_t)slot * Vmax + h);
}

// ---------------------------------------------------------------- asynchronous copies to shared memory
// The odd-site kernels need the site's own input (and r^) only after the hop: the thread copies
// them to its slice of shared memory with cp.async before the hop, so the loads overlap the hop's
// arithmetic without holding registers.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// one stored spinor in shared memory: its 16-byte words and its norm
template <int SPR>
struct SmemSpinor {
  static constexpr int W = SPR == PR32 ? 6 : 3;
  uint4 w[W];
  float n;
  __device__ __forceinline__ void fetch(FieldPtr f, int Vmax, int slot, int h) {
    const uint4* b = (const uint4*)f.p + (size_t)slot * W * Vmax + h;
#pragma unroll
    for (int k = 0; k < W; ++k) cp_async16(&w[k], b + (size_t)k * Vmax);
    if (SPR == PR32) n = 1.0f;
    else cp_async4(&n, f.nrm + (size_t)slot * Vmax + h);
  }
  // the components chunk_comp<SPR>(k, 0..3) in FP32, without the norm
  __device__ __forceinline__ void comp4(int k, float (&re)[4], float (&im)[4]) const {
    if constexpr (SPR == PR32) {
      const float4 u = *reinterpret_cast<const float4*>(&w[2 * k]), v = *reinterpret_cast<const float4*>(&w[2 * k + 1]);
      re[0] = u.x, im[0] = u.y, re[1] = u.z, im[1] = u.w, re[2] = v.x, im[2] = v.y, re[3] = v.z, im[3] = v.w;
    } else {
      chunk_words<SPR>(w[k], re, im);
    }
  }
};

// ---------------------------------------------------------------- spin projection
// (1 -+ g_mu) psi = [h ; -+A^H h] with h = psi_up -+ A psi_dn (chiral basis): for the upper spin
// s in {0, 1}, h_s = p_s + coef p_t with partner spin t and coef in {+1, -1, +i, -i}
// (PC_ONE, PC_MONE, PC_I, PC_MI), the same projection hp_fields.cuh's project<> performs.
enum { PC_ONE = 0, PC_MONE = 1, PC_I = 2, PC_MI = 3 };
template <int MU, int SIGN, int S>
struct ProjCoef {
  // MU 0: p0 +- i p3, p1 +- i p2;  MU 1: p0 +- p3, p1 -+ p2;  MU 2: p0 +- i p2, p1 -+ i p3;  MU 3: p0 -+ p2, p1 -+ p3
  static constexpr int t = MU == 0 ? (S == 0 ? 3 : 2) : MU == 1 ? (S == 0 ? 3 : 2) : MU == 2 ? (S == 0 ? 2 : 3) : (S == 0 ? 2 : 3);
  static constexpr bool neg = SIGN < 0 ? (MU == 1 ? S == 1 : MU == 2 ? S == 1 : MU == 3) : (MU == 1 ? S == 0 : MU == 2 ? S == 0 : MU == 3 ? false : true);
  static constexpr int coef = (MU == 0 || MU == 2) ? (neg ? PC_MI : PC_I) : (neg ? PC_MONE : PC_ONE);
};

// h_s[c] of one right-hand side (scalar outputs re, im) from its stored spinor
template <int MU, int SIGN, int S, class RAW>
__device__ __forceinline__ void project_one(const RAW& p, int c, float& hre, float& him) {
  constexpr int t = ProjCoef<MU, SIGN, S>::t, cf = ProjCoef<MU, SIGN, S>::coef;
  const int up = 3 * S + c, dn = 3 * t + c;
  if (cf == PC_ONE) {
    hre = p.re_add(up, p.re(dn));
    him = p.im_add(up, p.im(dn));
  } else if (cf == PC_MONE) {
    hre = p.re_sub(up, p.re(dn));
    him = p.im_sub(up, p.im(dn));
  } else if (cf == PC_I) {   // p_up + i p_dn = (re_up - im_dn, im_up + re_dn)
    hre = p.re_sub(up, p.im(dn));
    him = p.im_add(up, p.re(dn));
  } else {                   // p_up - i p_dn = (re_up + im_dn, im_up - re_dn)
    hre = p.re_add(up, p.im(dn));
    him = p.im_sub(up, p.re(dn));
  }
}

// projected half spinors of the two lanes: h[s][c] for s = 0, 1
template <int MU, int SIGN, class RAW>
__device__ __forceinline__ void project2(const RAW& pa, const RAW& pb, c2 (&h)[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float ar, ai, br, bi;
    project_one<MU, SIGN, 0>(pa, c, ar, ai);
    project_one<MU, SIGN, 0>(pb, c, br, bi);
    h[0][c].re = make_float2(ar, br);
    h[0][c].im = make_float2(ai, bi);
    project_one<MU, SIGN, 1>(pa, c, ar, ai);
    project_one<MU, SIGN, 1>(pb, c, br, bi);
    h[1][c].re = make_float2(ar, br);
    h[1][c].im = make_float2(ai, bi);
  }
}

// ---------------------------------------------------------------- links (18 reals, no reconstruction)
template <int LPR>
struct Link2;
template <>
struct Link2<PR16> {   // binary16: 2 uint4 + 1 word per link
  uint4 a, b;
  unsigned c;
  __device__ __forceinline__ void load(const LatGeom& g, int mu, int site) {
    const uint4* p = g.U16f + (size_t)mu * 2 * g.V + site;
    a = __ldg(p);
    b = __ldg(p + g.V);
    c = __ldg(g.U16g + (size_t)mu * g.V + site);
  }
  __device__ __forceinline__ unsigned word(int k) const {
    return k == 0 ? a.x : k == 1 ? a.y : k == 2 ? a.z : k == 3 ? a.w : k == 4 ? b.x : k == 5 ? b.y : k == 6 ? b.z : k == 7 ? b.w : c;
  }
  __device__ __forceinline__ void elem(int k, float& x, float& y) const {
    const unsigned w = word(k);
    x = h16lo_to_f32(w);
    y = h16hi_to_f32(w);
  }
};
template <>
struct Link2<PR32> {   // FP32: 4 float4 + 1 float2 per link
  float4 a[4];
  float2 c;
  __device__ __forceinline__ void load(const LatGeom& g, int mu, int site) {
    const float4* p = g.U32f + (size_t)mu * 4 * g.V + site;
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = __ldg(p + (size_t)k * g.V);
    c = __ldg(g.U32g + (size_t)mu * g.V + site);
  }
  __device__ __forceinline__ void elem(int k, float& x, float& y) const {
    if (k == 8) {
      x = c.x;
      y = c.y;
    } else {
      const float4& q = a[k >> 1];
      x = (k & 1) ? q.z : q.x;
      y = (k & 1) ? q.w : q.y;
    }
  }
};

// ---------------------------------------------------------------- one direction of the hop
// acc += sc * (spin reconstruction of U h) for both lanes; sc = (sc_A, sc_B)
template <int MU, int SIGN>
__device__ __forceinline__ void accumulate2(c2 (&acc)[12], const c2& w0, const c2& w1, int r, f2 sc, f2 msc) {
  // upper spins: acc[r] += sc w0, acc[3 + r] += sc w1
  acc[r].re = fma2(sc, w0.re, acc[r].re);
  acc[r].im = fma2(sc, w0.im, acc[r].im);
  acc[3 + r].re = fma2(sc, w1.re, acc[3 + r].re);
  acc[3 + r].im = fma2(sc, w1.im, acc[3 + r].im);
  // lower spins (the reconstruction rules of accumulate_s): a += k sc w with k = +-1 or +-i;
  // a += i s w is (a.re - s w.im, a.im + s w.re)
  c2& a6 = acc[6 + r];
  c2& a9 = acc[9 + r];
  if (MU == 0) {   // a6 += -+ i w1, a9 += -+ i w0
    const f2 s = SIGN < 0 ? msc : sc, ms = SIGN < 0 ? sc : msc;
    a6.re = fma2(ms, w1.im, a6.re);
    a6.im = fma2(s, w1.re, a6.im);
    a9.re = fma2(ms, w0.im, a9.re);
    a9.im = fma2(s, w0.re, a9.im);
  } else if (MU == 1) {   // a6 += -+ w1, a9 += +- w0
    const f2 s6 = SIGN < 0 ? msc : sc, s9 = SIGN < 0 ? sc : msc;
    a6.re = fma2(s6, w1.re, a6.re);
    a6.im = fma2(s6, w1.im, a6.im);
    a9.re = fma2(s9, w0.re, a9.re);
    a9.im = fma2(s9, w0.im, a9.im);
  } else if (MU == 2) {   // a6 += -+ i w0, a9 += +- i w1
    const f2 s6 = SIGN < 0 ? msc : sc, m6 = SIGN < 0 ? sc : msc;
    a6.re = fma2(m6, w0.im, a6.re);
    a6.im = fma2(s6, w0.re, a6.im);
    a9.re = fma2(s6, w1.im, a9.re);
    a9.im = fma2(m6, w1.re, a9.im);
  } else {   // a6 += -+ w0, a9 += -+ w1
    const f2 s = SIGN < 0 ? msc : sc;
    a6.re = fma2(s, w0.re, a6.re);
    a6.im = fma2(s, w0.im, a6.im);
    a9.re = fma2(s, w1.re, a9.re);
    a9.im = fma2(s, w1.im, a9.im);
  }
}

// the hop term of direction mu, sign SIGN (-1: forward neighbour with U_mu(x); +1: backward with
// U_mu(x - mu)^H), neighbour half-site nb, link site ls
template <int SPR, int LPR, int MU, int SIGN>
__device__ __forceinline__ void hop_dir2(const LatGeom& g, FieldPtr in, int Vmax, int sa, int sb, int nb, int ls,
                                         f2 scale, c2 (&acc)[12]) {
  Raw2<SPR> pa, pb;
  pa.load(in, Vmax, sa, nb);
  pb.load(in, Vmax, sb, nb);
  Link2<LPR> u;
  u.load(g, MU, ls);
  c2 h[2][3];
  project2<MU, SIGN>(pa, pb, h);
  const f2 sc = mul2(scale, make_float2(pa.n, pb.n));
  const f2 msc = make_float2(-sc.x, -sc.y);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    c2 w0, w1;
    w0.re = w0.im = w1.re = w1.im = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float x, y;
      u.elem(SIGN < 0 ? 3 * r + c : 3 * c + r, x, y);
      const f2 ux = bc2(x), uy = bc2(y), muy = bc2(-y);
      if (SIGN < 0) {   // u h:       re += x h.re - y h.im, im += x h.im + y h.re
        w0.re = fma2(ux, h[0][c].re, w0.re);
        w0.re = fma2(muy, h[0][c].im, w0.re);
        w0.im = fma2(ux, h[0][c].im, w0.im);
        w0.im = fma2(uy, h[0][c].re, w0.im);
        w1.re = fma2(ux, h[1][c].re, w1.re);
        w1.re = fma2(muy, h[1][c].im, w1.re);
        w1.im = fma2(ux, h[1][c].im, w1.im);
        w1.im = fma2(uy, h[1][c].re, w1.im);
      } else {          // conj(u) h: re += x h.re + y h.im, im += x h.im - y h.re
        w0.re = fma2(ux, h[0][c].re, w0.re);
        w0.re = fma2(uy, h[0][c].im, w0.re);
        w0.im = fma2(ux, h[0][c].im, w0.im);
        w0.im = fma2(muy, h[0][c].re, w0.im);
        w1.re = fma2(ux, h[1][c].re, w1.re);
        w1.re = fma2(uy, h[1][c].im, w1.re);
        w1.im = fma2(ux, h[1][c].im, w1.im);
        w1.im = fma2(muy, h[1][c].re, w1.im);
      }
    }
    accumulate2<MU, SIGN>(acc, w0, w1, r, sc, msc);
  }
}

// acc += scale * hop(in) at full site `site` (parity par of the output; `in` holds the other parity)
template <int SPR, int LPR>
__device__ __forceinline__ void eo_hop2(const LatGeom& g, FieldPtr in, int Vmax, int sa, int sb, int site,
                                        const int (&x)[4], const int (&st)[4], f2 scale, c2 (&acc)[12]) {
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int L = g.L[mu];
    const int fw = (x[mu] + 1 == L) ? site - (L - 1) * st[mu] : site + st[mu];
    const int bw = (x[mu] == 0) ? site + (L - 1) * st[mu] : site - st[mu];
    if (mu == 0) {
      hop_dir2<SPR, LPR, 0, -1>(g, in, Vmax, sa, sb, fw >> 1, site, scale, acc);
      hop_dir2<SPR, LPR, 0, 1>(g, in, Vmax, sa, sb, bw >> 1, bw, scale, acc);
    } else if (mu == 1) {
      hop_dir2<SPR, LPR, 1, -1>(g, in, Vmax, sa, sb, fw >> 1, site, scale, acc);
      hop_dir2<SPR, LPR, 1, 1>(g, in, Vmax, sa, sb, bw >> 1, bw, scale, acc);
    } else if (mu == 2) {
      hop_dir2<SPR, LPR, 2, -1>(g, in, Vmax, sa, sb, fw >> 1, site, scale, acc);
      hop_dir2<SPR, LPR, 2, 1>(g, in, Vmax, sa, sb, bw >> 1, bw, scale, acc);
    } else {
      hop_dir2<SPR, LPR, 3, -1>(g, in, Vmax, sa, sb, fw >> 1, site, scale, acc);
      hop_dir2<SPR, LPR, 3, 1>(g, in, Vmax, sa, sb, bw >> 1, bw, scale, acc);
    }
  }
}

// lane L (0: A, 1: B) of the pair accumulator as the 12 complex numbers of one right-hand side
__device__ __forceinline__ void lane_of(const c2 (&acc)[12], int L, cplx<float> (&out)[12]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) out[k] = L ? cplx<float>{acc[k].re.y, acc[k].im.y} : cplx<float>{acc[k].re.x, acc[k].im.x};
}

// the slot pair of a block: lanes A and B; a pair with one active slot computes it in both lanes
// (the second lane reads the same addresses) and stores it once
#define EO2_PREAMBLE(MASK)                                                          \
  const int pair = blockIdx.z * gridDim.x + blockIdx.x;                             \
  const int s0 = 2 * pair, s1 = 2 * pair + 1;                                       \
  if (s0 >= nslots) return;                                                         \
  const bool on0 = eo_mask(a.st + s0, MASK), on1 = s1 < nslots && eo_mask(a.st + s1, MASK); \
  if (!on0 && !on1) return;                                                         \
  const int sa = on0 ? s0 : s1, sb = (on0 && on1) ? s1 : sa;                        \
  const bool two = sb != sa;                                                        \
  const LatGeom g = a.lats[a.st[sa].lat];                                           \
  const int nsite = g.V >> 1;                                                       \
  const int ntiles = (nsite + NT - 1) / NT;                                         \
  if ((int)blockIdx.y >= ntiles) return;                                            \
  const int nparts = min((int)gridDim.y, ntiles);                                   \
  (void)nparts;

// ---- even sites: mid = A_e^-1 hop(in_o) for two right-hand sides per thread (MINB: resident blocks of
// NT threads the register budget allows, 4 -> 128 registers, 3 -> 168; chosen by timing)
template <int SPR, int LPR, int NT, int MINB, bool CL>
__global__ void __launch_bounds__(NT, MINB) k_eo2_even(WArgs a, FieldPtr in, FieldPtr mid, int nslots) {
  EO2_PREAMBLE(MASK_RUN)
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int h = tile * NT + threadIdx.x;
    if (h >= nsite) continue;
    int x[4], st[4];
    const int site = eo_site(g, h, 0, x, st);
    const bool clov = CL && g.clover;
    const float inv = clov ? 1.0f : 1.0f / site_diag<float>(g, site);
    c2 acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k].re = acc[k].im = make_float2(0.f, 0.f);
    eo_hop2<SPR, LPR>(g, in, a.Vmax, sa, sb, site, x, st, bc2(inv), acc);
#pragma unroll
    for (int L = 0; L < 2; ++L) {
      if (L == 1 && !two) break;
      cplx<float> v[12];
      lane_of(acc, L, v);
      if (CL && clov) {
        cplx<float> t[12];
        clover_mul<float>(g, true, site, v, t);
        SpinorIO<SPR>::store(mid, a.Vmax, L ? sb : sa, h, t);
      } else {
        SpinorIO<SPR>::store(mid, a.Vmax, L ? sb : sa, h, v);
      }
    }
  }
}

// per-slot partial sums of the pair kernels: NQ values per lane, warp shuffles in FP32, across
// warps in FP64, written for each distinct slot
template <int NQ, int NT>
__device__ __forceinline__ void reduce_pair(const float (&v)[2][NQ], double* part_a, double* part_b, int gy,
                                            bool two) {
  __shared__ double sh[2][NQ][NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int L = 0; L < 2; ++L)
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      float t = v[L][q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) sh[L][q][warp] = (double)t;
    }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int L = 0; L < 2; ++L) {
      if (L == 1 && !two) break;
      double* part = L ? part_b : part_a;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += sh[L][q][w];
        part[(size_t)q * gy + blockIdx.y] = t;
      }
    }
  }
}

// ---- odd sites: out = A_o in - k^2 hop(mid) with the solver epilogues, two right-hand sides per thread
//   EPI_V: v = S p, (r^, v), alpha       EPI_T: t = S s, (t, s), (t, t), omega
template <int SPR, int LPR, int NT, int MINB, int EPI, bool CL, int TPB>
__global__ void __launch_bounds__(NT, MINB) k_eo2_odd(WArgs a, FieldPtr in, FieldPtr mid, FieldPtr out, int nslots) {
  // TPB consecutive tiles per block (one reduction per TPB tiles; consecutive, so that the sweep
  // of the lattice stays one front and the neighbours of a tile are still in L2)
  const int pair = blockIdx.z * gridDim.x + blockIdx.x;
  const int s0 = 2 * pair, s1 = 2 * pair + 1;
  if (s0 >= nslots) return;
  const bool on0 = eo_mask(a.st + s0, MASK_RUN), on1 = s1 < nslots && eo_mask(a.st + s1, MASK_RUN);
  if (!on0 && !on1) return;
  const int sa = on0 ? s0 : s1, sb = (on0 && on1) ? s1 : sa;
  const bool two = sb != sa;
  const LatGeom g = a.lats[a.st[sa].lat];
  const int nsite = g.V >> 1;
  const int ntiles = (nsite + NT - 1) / NT;
  const int nchunks = (ntiles + TPB - 1) / TPB;
  if ((int)blockIdx.y >= nchunks) return;
  const int nparts = min((int)gridDim.y, nchunks);
  constexpr int NQ = EPI == EPI_V ? 2 : 3;
  constexpr int NF = 1;   // own-site field prefetched: the input (r^ of the V step is loaded after the hop)
  // (binary16 fields: 16 KB per field and block; the FP32 iteration's would exceed the 48 KB of
  // static shared memory, so it loads them after the hop)
  constexpr bool PREF = SPR != PR32;
  __shared__ SmemSpinor<SPR> own[PREF ? NT : 1][NF][2];
  float dots[2][NQ];
#pragma unroll
  for (int L = 0; L < 2; ++L)
#pragma unroll
    for (int q = 0; q < NQ; ++q) dots[L][q] = 0.f;
  const float mk2 = -(float)(g.kappa * g.kappa);
  for (int tile = blockIdx.y * TPB; tile < min(ntiles, (int)(blockIdx.y + 1) * TPB); ++tile) {
    const int h = tile * NT + threadIdx.x;
    if (h >= nsite) continue;
    int x[4], st[4];
    const int site = eo_site(g, h, 1, x, st);
    const bool clov = CL && g.clover;
    if (PREF && !clov) {
      own[threadIdx.x][0][0].fetch(in, a.Vmax, sa, h);
      own[threadIdx.x][0][1].fetch(in, a.Vmax, sb, h);
      cp_async_commit();
    }
    c2 acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k].re = acc[k].im = make_float2(0.f, 0.f);
    eo_hop2<SPR, LPR>(g, mid, a.Vmax, sa, sb, site, x, st, bc2(mk2), acc);
    if (clov) {   // the 6x6 clover blocks need the whole spinor: lane by lane
#pragma unroll
      for (int L = 0; L < 2; ++L) {
        if (L == 1 && !two) break;
        const int slot = L ? sb : sa;
        cplx<float> v[12], c[12];
        lane_of(acc, L, v);
        float nc;
        SpinorIO<SPR>::load_nc_raw(in, a.Vmax, slot, h, c, nc);
        add_diag<float, CL>(g, site, c, nc, v);
        SpinorIO<SPR>::store(out, a.Vmax, slot, h, v);
        if (EPI == EPI_V) {
          cplx<float> rh[12];
          SpinorIO<SPR>::load(a.rh, a.Vmax, slot, h, rh);
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            const cplx<float> d = cconjmul(rh[k], v[k]);
            dots[L][0] += d.x;
            dots[L][1] += d.y;
          }
        } else {
          float d0 = 0.f, d1 = 0.f;
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            const cplx<float> d = cconjmul(v[k], c[k]);
            d0 += d.x;
            d1 += d.y;
            dots[L][NQ - 1] += v[k].x * v[k].x + v[k].y * v[k].y;
          }
          dots[L][0] += nc * d0;
          dots[L][1] += nc * d1;
        }
      }
      continue;
    }
    // diagonal term and dot products four components at a time (few live registers):
    // v = acc + d n c (c the stored input, n its norm), then (r^, v) or (v, n c) and (v, v)
    if (PREF) cp_async_wait_all();
    const SmemSpinor<SPR>(&my)[NF][2] = own[PREF ? threadIdx.x : 0];
    const float dg = site_diag<float>(g, site);
    const f2 ncs = PREF ? make_float2(my[0][0].n, my[0][1].n) : make_float2(1.0f, 1.0f);
    const f2 nd = mul2(bc2(dg), ncs);
    f2 q0 = make_float2(0.f, 0.f), q1 = q0, q2 = q0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float ar[4], ai[4], br[4], bi[4];
      float rr[2][4], ri[2][4];
      if (PREF) {
        my[0][0].comp4(k, ar, ai);
        my[0][1].comp4(k, br, bi);
      } else {
        load_comp4<SPR>(in, a.Vmax, sa, h, k, ar, ai);
        load_comp4<SPR>(in, a.Vmax, sb, h, k, br, bi);
      }
      if (EPI == EPI_V) {
        load_comp4<SPR>(a.rh, a.Vmax, sa, h, k, rr[0], ri[0]);
        load_comp4<SPR>(a.rh, a.Vmax, sb, h, k, rr[1], ri[1]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        c2& t = acc[chunk_comp<SPR>(k, j)];
        const f2 cr = make_float2(ar[j], br[j]), ci = make_float2(ai[j], bi[j]);
        t.re = fma2(nd, cr, t.re);
        t.im = fma2(nd, ci, t.im);
        if (EPI == EPI_V) {   // conj(r^) v
          const f2 hr = make_float2(rr[0][j], rr[1][j]), hi = make_float2(ri[0][j], ri[1][j]);
          q0 = fma2(hr, t.re, q0);
          q0 = fma2(hi, t.im, q0);
          q1 = fma2(hr, t.im, q1);
          q1 = fma2(make_float2(-hi.x, -hi.y), t.re, q1);
        } else {              // conj(v) c and |v|^2
          q0 = fma2(t.re, cr, q0);
          q0 = fma2(t.im, ci, q0);
          q1 = fma2(t.re, ci, q1);
          q1 = fma2(make_float2(-t.im.x, -t.im.y), cr, q1);
          q2 = fma2(t.re, t.re, q2);
          q2 = fma2(t.im, t.im, q2);
        }
      }
    }
    if (EPI == EPI_V) {   // r^ is stored with its own norm
      const f2 rn = make_float2(load_norm<SPR>(a.rh, a.Vmax, sa, h), load_norm<SPR>(a.rh, a.Vmax, sb, h));
      q0 = mul2(q0, rn);
      q1 = mul2(q1, rn);
    } else {
      q0 = mul2(q0, ncs);
      q1 = mul2(q1, ncs);
      dots[0][2 % NQ] += q2.x;
      dots[1][2 % NQ] += q2.y;
    }
    dots[0][0] += q0.x;
    dots[1][0] += q0.y;
    dots[0][1] += q1.x;
    dots[1][1] += q1.y;
#pragma unroll
    for (int L = 0; L < 2; ++L) {
      if (L == 1 && !two) break;
      cplx<float> v[12];
      lane_of(acc, L, v);
      SpinorIO<SPR>::store(out, a.Vmax, L ? sb : sa, h, v);
    }
  }
  reduce_pair<NQ, NT>(dots, a.part + (size_t)sa * 4 * a.gy, a.part + (size_t)sb * 4 * a.gy, a.gy, two);
#pragma unroll
  for (int L = 0; L < 2; ++L) {
    if (L == 1 && !two) break;
    const int slot = L ? sb : sa;
    SlotState* S = a.st + slot;
    if (last_block(a.cnt + slot, nparts)) {
      double tot[NQ];
      block_sum_partials<NQ, NT>(a.part + (size_t)slot * 4 * a.gy, a.gy, nparts, tot);
      if (threadIdx.x == 0) {
        if (EPI == EPI_V) {
          S->alpha = cdiv(S->rho, make_double2(tot[0], tot[1]));
          S->restart = 0;
          if (S->need_update == 3) S->need_update = 0;
          S->sloppy_mv += 1;
        } else {
          S->omega = tot[NQ - 1] > 0.0 ? make_double2(tot[0] / tot[NQ - 1], tot[1] / tot[NQ - 1]) : make_double2(0.0, 0.0);
          S->sloppy_mv += 1;
        }
        a.cnt[slot] = 0;
      }
      __syncthreads();
    }
  }
}
