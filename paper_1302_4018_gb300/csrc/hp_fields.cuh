// Device-side field storage and the Wilson stencil core.
//
// Spinor fields hold the right-hand sides of all solver slots:
//   chunk k of site s of slot q lives at  base[(q * NCH + k) * Vmax + s]
// so consecutive threads (consecutive sites) read consecutive 16-byte
// chunks (fully coalesced 128-bit accesses).
//   FP64: 12 chunks of double2 (one complex each)
//   FP32:  6 chunks of float4  (two complex each)
//   FP16 / BF16: 3 chunks of uint4 (four complex each, scaled by a per-site
//         FP32 norm = max |component| so the stored values lie in [-1, 1]);
//         chunk c holds colour c, its words the spins 0-3 (component 3 s + c),
//         so that one 16-byte load gives a tensor-core lane the four spins of
//         one colour
// Links of one lattice ([4][chunks][V], same coalescing):
//   FP64: 9 double2 per link (full 3x3)
//   FP32, 12 reals: 3 float4 per link (rows 1-2); row 3 = conj(row1 x row2)
//   FP32, 18 reals: 4 float4 + 1 float2 per link (all entries, no reconstruction)
//   FP16, 12 reals: 3 uint2 per link (rows 1-2 in binary16), row 3 reconstructed
//   FP16, 18 reals: 2 uint4 + 1 half2 per link
// (the 18-real forms trade bytes, shared by all right-hand sides of a launch,
// for the reconstruction arithmetic of the ALU-bound sloppy stencil)
#pragma once
#include "hp_internal.h"

// ----------------------------------------------------------------- float-float
// An unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2): a 48-bit
// significand on the FP32 pipes.  GB300 executes FP64 at 1/58 of the FP32 rate,
// so the true-residual stencil of the mixed-precision solver runs in this
// arithmetic.  Addition is Knuth's TwoSum followed by renormalisation; the
// product uses an FMA to obtain the exact rounding error of hi*hi (TwoProduct)
// plus the cross terms.  The intrinsics keep the compiler from contracting or
// reassociating the error-free transformations.
struct ffl {
  float hi, lo;
  __host__ __device__ ffl() {}
  __host__ __device__ ffl(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ ffl(float h) : hi(h), lo(0.f) {}
  __host__ __device__ ffl(int i) : hi((float)i), lo(0.f) {}
  __host__ __device__ ffl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};
__device__ __forceinline__ ffl ffl_renorm(float s, float e) {   // |s| >= |e|
  float h = __fadd_rn(s, e);
  return ffl(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ ffl operator+(ffl a, ffl b) {
  float s = __fadd_rn(a.hi, b.hi);
  float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ffl_renorm(s, e);
}
__device__ __forceinline__ ffl operator-(ffl a) { return ffl(-a.hi, -a.lo); }
__device__ __forceinline__ ffl operator-(ffl a, ffl b) { return a + (-b); }
__device__ __forceinline__ ffl operator*(ffl a, ffl b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ffl_renorm(p, e);
}
__device__ __forceinline__ ffl fma(ffl a, ffl b, ffl c) { return a * b + c; }
__device__ __forceinline__ ffl& operator+=(ffl& a, ffl b) {
  a = a + b;
  return a;
}
__device__ __forceinline__ ffl& operator-=(ffl& a, ffl b) {
  a = a - b;
  return a;
}
__device__ __forceinline__ double ffl_to_double(ffl a) { return (double)a.hi + (double)a.lo; }
template <typename T>
struct is_ffl {
  static constexpr bool value = false;
};
template <>
struct is_ffl<ffl> {
  static constexpr bool value = true;
};

template <int PR>
struct Real_of {
  typedef float T;
};
template <>
struct Real_of<PR64> {
  typedef double T;
};
template <>
struct Real_of<PRFF> {
  typedef ffl T;
};

struct FieldPtr {
  void* p;
  float* nrm;   // half precisions only
  void* lo;     // float-float fields: the FP32 field of low parts (p holds the high parts)
};

template <int PR>
struct SpinorIO;

template <>
struct SpinorIO<PR64> {
  static constexpr int NCH = 12;
  static constexpr int BYTES = 192;
  template <typename R>
  __device__ static __forceinline__ void load(FieldPtr f, int Vmax, int slot, int site, cplx<R> (&s)[12]) {
    const double2* b = (const double2*)f.p + (size_t)slot * 12 * Vmax + site;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 v = b[(size_t)k * Vmax];
      s[k].x = (R)v.x;
      s[k].y = (R)v.y;
    }
  }
  template <typename R>
  __device__ static __forceinline__ void load_nc(FieldPtr f, int Vmax, int slot, int site, cplx<R> (&s)[12]) {
    const double2* b = (const double2*)f.p + (size_t)slot * 12 * Vmax + site;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 v = __ldg(b + (size_t)k * Vmax);
      s[k].x = (R)v.x;
      s[k].y = (R)v.y;
    }
  }
  template <typename R>
  __device__ static __forceinline__ void load_nc_raw(FieldPtr f, int Vmax, int slot, int site, cplx<R> (&s)[12],
                                                     R& n) {
    load_nc(f, Vmax, slot, site, s);
    n = (R)1;
  }
  template <typename R>
  __device__ static __forceinline__ void store(FieldPtr f, int Vmax, int slot, int site, const cplx<R> (&s)[12]) {
    double2* b = (double2*)f.p + (size_t)slot * 12 * Vmax + site;
#pragma unroll
    for (int k = 0; k < 12; ++k) b[(size_t)k * Vmax] = make_double2((double)s[k].x, (double)s[k].y);
  }
};

template <>
struct SpinorIO<PR32> {
  static constexpr int NCH = 6;
  static constexpr int BYTES = 96;
  template <typename R>
  __device__ static __forceinline__ void unpack(const float4 (&c)[6], cplx<R> (&s)[12]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      s[2 * k].x = c[k].x;
      s[2 * k].y = c[k].y;
      s[2 * k + 1].x = c[k].z;
      s[2 * k + 1].y = c[k].w;
    }
  }
  template <typename R>
  __device__ static __forceinline__ void load(FieldPtr f, int Vmax, int slot, int site, cplx<R> (&s)[12]) {
    const float4* b = (const float4*)f.p + (size_t)slot * 6 * Vmax + site;
    float4 c[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) c[k] = b[(size_t)k * Vmax];
    unpack(c, s);
  }
  template <typename R>
  __device__ static __forceinline__ void load_nc(FieldPtr f, int Vmax, int slot, int site, cplx<R> (&s)[12]) {
    const float4* b = (const float4*)f.p + (size_t)slot * 6 * Vmax + site;
    float4 c[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) c[k] = __ldg(b + (size_t)k * Vmax);
    unpack(c, s);
  }
  template <typename R>
  __device__ static __forceinline__ void load_nc_raw(FieldPtr f, int Vmax, int slot, int site, cplx<R> (&s)[12],
                                                     R& n) {
    load_nc(f, Vmax, slot, site, s);
    n = (R)1;
  }
  template <typename R>
  __device__ static __forceinline__ void store(FieldPtr f, int Vmax, int slot, int site, const cplx<R> (&s)[12]) {
    float4* b = (float4*)f.p + (size_t)slot * 6 * Vmax + site;
#pragma unroll
    for (int k = 0; k < 6; ++k)
      b[(size_t)k * Vmax] = make_float4((float)s[2 * k].x, (float)s[2 * k].y, (float)s[2 * k + 1].x, (float)s[2 * k + 1].y);
  }
};

template <>
struct SpinorIO<PRFF> {
  static constexpr int NCH = 6;
  static constexpr int BYTES = 192;
  template <typename R>
  __device__ static __forceinline__ void load(FieldPtr f, int Vmax, int slot, int site, cplx<R> (&s)[12]) {
    cplx<float> h[12], l[12];
    SpinorIO<PR32>::load(FieldPtr{f.p, nullptr, nullptr}, Vmax, slot, site, h);
    SpinorIO<PR32>::load(FieldPtr{f.lo, nullptr, nullptr}, Vmax, slot, site, l);
#pragma unroll
    for (int k = 0; k < 12; ++k) s[k] = {R(ffl(h[k].x, l[k].x)), R(ffl(h[k].y, l[k].y))};
  }
  template <typename R>
  __device__ static __forceinline__ void load_nc(FieldPtr f, int Vmax, int slot, int site, cplx<R> (&s)[12]) {
    cplx<float> h[12], l[12];
    SpinorIO<PR32>::load_nc(FieldPtr{f.p, nullptr, nullptr}, Vmax, slot, site, h);
    SpinorIO<PR32>::load_nc(FieldPtr{f.lo, nullptr, nullptr}, Vmax, slot, site, l);
#pragma unroll
    for (int k = 0; k < 12; ++k) s[k] = {R(ffl(h[k].x, l[k].x)), R(ffl(h[k].y, l[k].y))};
  }
  template <typename R>
  __device__ static __forceinline__ void load_nc_raw(FieldPtr f, int Vmax, int slot, int site, cplx<R> (&s)[12],
                                                     R& n) {
    load_nc(f, Vmax, slot, site, s);
    n = R(1);
  }
  __device__ static __forceinline__ void store(FieldPtr f, int Vmax, int slot, int site, const cplx<ffl> (&s)[12]) {
    cplx<float> h[12], l[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      h[k] = {s[k].x.hi, s[k].y.hi};
      l[k] = {s[k].x.lo, s[k].y.lo};
    }
    SpinorIO<PR32>::store(FieldPtr{f.p, nullptr, nullptr}, Vmax, slot, site, h);
    SpinorIO<PR32>::store(FieldPtr{f.lo, nullptr, nullptr}, Vmax, slot, site, l);
  }
};

template <int PR>
struct Half2Ops;
// binary16 -> FP32 as the mixed-precision add h + 0.0f (add.rn.f32.f16): exact, since every binary16
// value is an FP32 value (a negative zero comes out positive), and on sm_100+ it issues at the full
// FP32 rate, where cvt.f32.f16 takes two slots of the FP32 pipe
__device__ __forceinline__ float h16lo_to_f32(unsigned int u) {
  float r;
  asm("{.reg .f16 l, h; mov.b32 {l, h}, %1; add.rn.f32.f16 %0, l, %2;}" : "=f"(r) : "r"(u), "f"(0.0f));
  return r;
}
__device__ __forceinline__ float h16hi_to_f32(unsigned int u) {
  float r;
  asm("{.reg .f16 l, h; mov.b32 {l, h}, %1; add.rn.f32.f16 %0, h, %2;}" : "=f"(r) : "r"(u), "f"(0.0f));
  return r;
}
template <>
struct Half2Ops<PR16> {
  __device__ static __forceinline__ float2 to_f2(unsigned int u) { return make_float2(h16lo_to_f32(u), h16hi_to_f32(u)); }
  __device__ static __forceinline__ unsigned int from_f2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<unsigned int*>(&h);
  }
};
template <>
struct Half2Ops<PRB16> {
  __device__ static __forceinline__ float2 to_f2(unsigned int u) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&u);
    return __bfloat1622float2(h);
  }
  __device__ static __forceinline__ unsigned int from_f2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<unsigned int*>(&h);
  }
};

template <int PR>
struct SpinorIOHalf {
  static constexpr int NCH = 3;
  static constexpr int BYTES = 52;   // 48 bytes of values + 4 bytes of norm
  template <typename R>
  __device__ static __forceinline__ void unpack(const uint4 (&c)[3], float n, cplx<R> (&s)[12]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {   // chunk k = colour k, word j = spin j
      float2 a = Half2Ops<PR>::to_f2(c[k].x), b = Half2Ops<PR>::to_f2(c[k].y);
      float2 d = Half2Ops<PR>::to_f2(c[k].z), e = Half2Ops<PR>::to_f2(c[k].w);
      s[k + 0] = {a.x * n, a.y * n};
      s[k + 3] = {b.x * n, b.y * n};
      s[k + 6] = {d.x * n, d.y * n};
      s[k + 9] = {e.x * n, e.y * n};
    }
  }
  template <typename R>
  __device__ static __forceinline__ void load(FieldPtr f, int Vmax, int slot, int site, cplx<R> (&s)[12]) {
    const uint4* b = (const uint4*)f.p + (size_t)slot * 3 * Vmax + site;
    uint4 c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = b[(size_t)k * Vmax];
    unpack(c, f.nrm[(size_t)slot * Vmax + site], s);
  }
  template <typename R>
  __device__ static __forceinline__ void load_nc(FieldPtr f, int Vmax, int slot, int site, cplx<R> (&s)[12]) {
    const uint4* b = (const uint4*)f.p + (size_t)slot * 3 * Vmax + site;
    uint4 c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = __ldg(b + (size_t)k * Vmax);
    unpack(c, __ldg(f.nrm + (size_t)slot * Vmax + site), s);
  }
  // values without the per-site norm, which is returned in n
  template <typename R>
  __device__ static __forceinline__ void load_nc_raw(FieldPtr f, int Vmax, int slot, int site, cplx<R> (&s)[12],
                                                     R& n) {
    const uint4* b = (const uint4*)f.p + (size_t)slot * 3 * Vmax + site;
    uint4 c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = __ldg(b + (size_t)k * Vmax);
    n = __ldg(f.nrm + (size_t)slot * Vmax + site);
    unpack(c, 1.0f, s);
  }
  template <typename R>
  __device__ static __forceinline__ void store(FieldPtr f, int Vmax, int slot, int site, const cplx<R> (&s)[12]) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf((float)s[k].x), fabsf((float)s[k].y)));
    float inv = m > 0.f ? 1.0f / m : 0.f;
    uint4* b = (uint4*)f.p + (size_t)slot * 3 * Vmax + site;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 c;
      c.x = Half2Ops<PR>::from_f2((float)s[k].x * inv, (float)s[k].y * inv);
      c.y = Half2Ops<PR>::from_f2((float)s[k + 3].x * inv, (float)s[k + 3].y * inv);
      c.z = Half2Ops<PR>::from_f2((float)s[k + 6].x * inv, (float)s[k + 6].y * inv);
      c.w = Half2Ops<PR>::from_f2((float)s[k + 9].x * inv, (float)s[k + 9].y * inv);
      b[(size_t)k * Vmax] = c;
    }
    f.nrm[(size_t)slot * Vmax + site] = m;
  }
};
template <>
struct SpinorIO<PR16> : SpinorIOHalf<PR16> {};
template <>
struct SpinorIO<PRB16> : SpinorIOHalf<PRB16> {};

// ------------------------------------------------------------------- links
template <typename R>
__device__ __forceinline__ void reconstruct_row3(cplx<R> (&u)[9]) {
  // row 3 = conj(row1 x row2), exact for special-unitary links
  cplx<R> a = cmul(u[1], u[5]), b = cmul(u[2], u[4]);
  u[6] = {a.x - b.x, -(a.y - b.y)};
  a = cmul(u[2], u[3]);
  b = cmul(u[0], u[5]);
  u[7] = {a.x - b.x, -(a.y - b.y)};
  a = cmul(u[0], u[4]);
  b = cmul(u[1], u[3]);
  u[8] = {a.x - b.x, -(a.y - b.y)};
}

// REC = 12: rows 1-2 stored, row 3 reconstructed; REC = 18: all nine entries stored
template <int LPR, int REC = 12>
struct LinkIO;

template <int REC>
struct LinkIO<PR64, REC> {
  static constexpr int BYTES = 144;
  template <typename R>
  __device__ static __forceinline__ void load(const LatGeom& g, int mu, int site, cplx<R> (&u)[9]) {
    const double2* b = g.U64 + (size_t)mu * 9 * g.V + site;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 v = __ldg(b + (size_t)k * g.V);
      u[k].x = (R)v.x;
      u[k].y = (R)v.y;
    }
  }
};

template <>
struct LinkIO<PR32, 12> {
  static constexpr int BYTES = 48;
  template <typename R>
  __device__ static __forceinline__ void load(const LatGeom& g, int mu, int site, cplx<R> (&u)[9]) {
    const float4* b = g.U32 + (size_t)mu * 3 * g.V + site;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float4 v = __ldg(b + (size_t)k * g.V);
      u[2 * k] = {v.x, v.y};
      u[2 * k + 1] = {v.z, v.w};
    }
    reconstruct_row3(u);
  }
};

template <>
struct LinkIO<PR16, 12> {
  static constexpr int BYTES = 24;
  template <typename R>
  __device__ static __forceinline__ void load(const LatGeom& g, int mu, int site, cplx<R> (&u)[9]) {
    const uint2* b = g.U16 + (size_t)mu * 3 * g.V + site;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint2 v = __ldg(b + (size_t)k * g.V);
      float2 a = Half2Ops<PR16>::to_f2(v.x), c = Half2Ops<PR16>::to_f2(v.y);
      u[2 * k] = {a.x, a.y};
      u[2 * k + 1] = {c.x, c.y};
    }
    reconstruct_row3(u);
  }
};

template <>
struct LinkIO<PR32, 18> {
  static constexpr int BYTES = 72;
  template <typename R>
  __device__ static __forceinline__ void load(const LatGeom& g, int mu, int site, cplx<R> (&u)[9]) {
    const float4* b = g.U32f + (size_t)mu * 4 * g.V + site;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float4 v = __ldg(b + (size_t)k * g.V);
      u[2 * k] = {v.x, v.y};
      u[2 * k + 1] = {v.z, v.w};
    }
    float2 e = __ldg(g.U32g + (size_t)mu * g.V + site);
    u[8] = {e.x, e.y};
  }
};

template <int REC>
struct LinkIO<PRFF, REC> {
  static constexpr int BYTES = 144;
  template <typename R>
  __device__ static __forceinline__ void load(const LatGeom& g, int mu, int site, cplx<R> (&u)[9]) {
    const float4* b = g.U32f + (size_t)mu * 4 * g.V + site;
    const float4* c = g.U32fl + (size_t)mu * 4 * g.V + site;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float4 v = __ldg(b + (size_t)k * g.V), w = __ldg(c + (size_t)k * g.V);
      u[2 * k] = {ffl(v.x, w.x), ffl(v.y, w.y)};
      u[2 * k + 1] = {ffl(v.z, w.z), ffl(v.w, w.w)};
    }
    float2 e = __ldg(g.U32g + (size_t)mu * g.V + site), f = __ldg(g.U32gl + (size_t)mu * g.V + site);
    u[8] = {ffl(e.x, f.x), ffl(e.y, f.y)};
  }
};

template <>
struct LinkIO<PR16, 18> {
  static constexpr int BYTES = 36;
  template <typename R>
  __device__ static __forceinline__ void load(const LatGeom& g, int mu, int site, cplx<R> (&u)[9]) {
    const uint4* b = g.U16f + (size_t)mu * 2 * g.V + site;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      uint4 v = __ldg(b + (size_t)k * g.V);
      float2 a = Half2Ops<PR16>::to_f2(v.x), c = Half2Ops<PR16>::to_f2(v.y);
      float2 d = Half2Ops<PR16>::to_f2(v.z), e = Half2Ops<PR16>::to_f2(v.w);
      u[4 * k + 0] = {a.x, a.y};
      u[4 * k + 1] = {c.x, c.y};
      u[4 * k + 2] = {d.x, d.y};
      u[4 * k + 3] = {e.x, e.y};
    }
    float2 f8 = Half2Ops<PR16>::to_f2(__ldg(g.U16g + (size_t)mu * g.V + site));
    u[8] = {f8.x, f8.y};
  }
};

template <int SPR>
struct LinkPrecOf {
  static constexpr int v = (SPR == PR64) ? PR64 : (SPR == PR32 ? PR32 : PR16);
};

// ------------------------------------------------------------- stencil core
// Spin projection in the chiral basis: g_mu = [[0, A], [A^H, 0]] with
// A_1 = -i s_1, A_2 = -i s_2, A_3 = -i s_3, A_4 = 1.
//   (1 - g_mu) psi = [h ; -A^H h],  h = psi_up - A psi_dn
//   (1 + g_mu) psi = [h ;  A^H h],  h = psi_up + A psi_dn
// Component index 3*spin + colour.
template <typename R>
__device__ __forceinline__ cplx<R> c_add(cplx<R> a, cplx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R>
__device__ __forceinline__ cplx<R> c_sub(cplx<R> a, cplx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R>
__device__ __forceinline__ cplx<R> c_addi(cplx<R> a, cplx<R> b) { return {a.x - b.y, a.y + b.x}; }  // a + i b
template <typename R>
__device__ __forceinline__ cplx<R> c_subi(cplx<R> a, cplx<R> b) { return {a.x + b.y, a.y - b.x}; }  // a - i b

template <int MU, int SIGN, typename R>   // SIGN = -1: (1 - g), +1: (1 + g)
__device__ __forceinline__ void project(const cplx<R> (&p)[12], cplx<R> (&h)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cplx<R> p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
    if (MU == 0) {
      h[c] = SIGN < 0 ? c_addi(p0, p3) : c_subi(p0, p3);
      h[3 + c] = SIGN < 0 ? c_addi(p1, p2) : c_subi(p1, p2);
    } else if (MU == 1) {
      h[c] = SIGN < 0 ? c_add(p0, p3) : c_sub(p0, p3);
      h[3 + c] = SIGN < 0 ? c_sub(p1, p2) : c_add(p1, p2);
    } else if (MU == 2) {
      h[c] = SIGN < 0 ? c_addi(p0, p2) : c_subi(p0, p2);
      h[3 + c] = SIGN < 0 ? c_subi(p1, p3) : c_addi(p1, p3);
    } else {
      h[c] = SIGN < 0 ? c_sub(p0, p2) : c_add(p0, p2);
      h[3 + c] = SIGN < 0 ? c_sub(p1, p3) : c_add(p1, p3);
    }
  }
}

template <int MU, int SIGN, typename R>
__device__ __forceinline__ void accumulate(cplx<R> (&acc)[12], const cplx<R> (&w)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cplx<R> w0 = w[c], w1 = w[3 + c];
    acc[c] = c_add(acc[c], w0);
    acc[3 + c] = c_add(acc[3 + c], w1);
    if (MU == 0) {   // -A^H v = (-i v1, -i v0);  A^H w = (i w1, i w0)
      acc[6 + c] = SIGN < 0 ? c_subi(acc[6 + c], w1) : c_addi(acc[6 + c], w1);
      acc[9 + c] = SIGN < 0 ? c_subi(acc[9 + c], w0) : c_addi(acc[9 + c], w0);
    } else if (MU == 1) {   // -A^H v = (-v1, v0);  A^H w = (w1, -w0)
      acc[6 + c] = SIGN < 0 ? c_sub(acc[6 + c], w1) : c_add(acc[6 + c], w1);
      acc[9 + c] = SIGN < 0 ? c_add(acc[9 + c], w0) : c_sub(acc[9 + c], w0);
    } else if (MU == 2) {   // -A^H v = (-i v0, i v1);  A^H w = (i w0, -i w1)
      acc[6 + c] = SIGN < 0 ? c_subi(acc[6 + c], w0) : c_addi(acc[6 + c], w0);
      acc[9 + c] = SIGN < 0 ? c_addi(acc[9 + c], w1) : c_subi(acc[9 + c], w1);
    } else {   // -A^H v = -v;  A^H w = w
      acc[6 + c] = SIGN < 0 ? c_sub(acc[6 + c], w0) : c_add(acc[6 + c], w0);
      acc[9 + c] = SIGN < 0 ? c_sub(acc[9 + c], w1) : c_add(acc[9 + c], w1);
    }
  }
}

// acc += sc * (the spin reconstruction of w), as FMAs: the per-site norm of a
// half-precision spinor and the factor -kappa ride along for free
template <typename R>
__device__ __forceinline__ void fadd_s(cplx<R>& a, cplx<R> w, R sc) {   // a += sc w
  a.x = fma(sc, w.x, a.x);
  a.y = fma(sc, w.y, a.y);
}
template <typename R>
__device__ __forceinline__ void faddi_s(cplx<R>& a, cplx<R> w, R sc) {  // a += i sc w
  a.x = fma(-sc, w.y, a.x);
  a.y = fma(sc, w.x, a.y);
}
template <int MU, int SIGN, typename R>
__device__ __forceinline__ void accumulate_s(cplx<R> (&acc)[12], const cplx<R> (&w)[6], R sc) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cplx<R> w0 = w[c], w1 = w[3 + c];
    fadd_s(acc[c], w0, sc);
    fadd_s(acc[3 + c], w1, sc);
    if (MU == 0) {   // -A^H v = (-i v1, -i v0);  A^H w = (i w1, i w0)
      faddi_s(acc[6 + c], w1, SIGN < 0 ? -sc : sc);
      faddi_s(acc[9 + c], w0, SIGN < 0 ? -sc : sc);
    } else if (MU == 1) {   // -A^H v = (-v1, v0);  A^H w = (w1, -w0)
      fadd_s(acc[6 + c], w1, SIGN < 0 ? -sc : sc);
      fadd_s(acc[9 + c], w0, SIGN < 0 ? sc : -sc);
    } else if (MU == 2) {   // -A^H v = (-i v0, i v1);  A^H w = (i w0, -i w1)
      faddi_s(acc[6 + c], w0, SIGN < 0 ? -sc : sc);
      faddi_s(acc[9 + c], w1, SIGN < 0 ? sc : -sc);
    } else {   // -A^H v = -v;  A^H w = w
      fadd_s(acc[6 + c], w0, SIGN < 0 ? -sc : sc);
      fadd_s(acc[9 + c], w1, SIGN < 0 ? -sc : sc);
    }
  }
}

template <typename R, bool DAG>
__device__ __forceinline__ void su3_mul(const cplx<R> (&u)[9], const cplx<R> (&h)[6], cplx<R> (&w)[6]) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      cplx<R> acc = {0, 0};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cplx<R> a = DAG ? u[3 * c + r] : u[3 * r + c];
        cplx<R> b = h[3 * s + c];
        if (DAG) {   // conj(a) * b
          acc.x = fma(a.x, b.x, acc.x);
          acc.x = fma(a.y, b.y, acc.x);
          acc.y = fma(a.x, b.y, acc.y);
          acc.y = fma(-a.y, b.x, acc.y);
        } else {
          acc.x = fma(a.x, b.x, acc.x);
          acc.x = fma(-a.y, b.y, acc.x);
          acc.y = fma(a.x, b.y, acc.y);
          acc.y = fma(a.y, b.x, acc.y);
        }
      }
      w[3 * s + r] = acc;
    }
  }
}

struct SiteCoords {
  int x[4];
};

__device__ __forceinline__ void site_coords(const LatGeom& g, int site, int (&x)[4], int (&st)[4]) {
  int r = site;
  int s = 1;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    x[j] = r % g.L[j];
    r /= g.L[j];
    st[j] = s;
    s *= g.L[j];
  }
}

// ---- the float-float hop ----
// Lazily normalised float-float numbers for the hop sums: the high parts are added with TwoSum
// and products of high parts split exactly with an FMA (TwoProduct), while every rounding error
// and cross term collects in the low part without renormalising after each operation (the low
// part stays within a few ulp of the high part over the ~200 terms of a hop, so hi + lo keeps a
// 46-bit significand).  One renormalisation per result.
struct ffz {
  float hi, lo;
  __device__ __forceinline__ ffz() {}
  __device__ __forceinline__ ffz(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ ffz(int i) : hi((float)i), lo(0.f) {}
};
__device__ __forceinline__ ffz operator-(ffz a) { return ffz(-a.hi, -a.lo); }
__device__ __forceinline__ ffz operator+(ffz a, ffz b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return ffz(s, __fadd_rn(__fadd_rn(a.lo, b.lo), e));
}
__device__ __forceinline__ ffz operator-(ffz a, ffz b) { return a + (-b); }
__device__ __forceinline__ ffz fma(ffz a, ffz b, ffz c) {   // c + a b
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(c.hi, p);
  const float bb = __fsub_rn(s, c.hi);
  const float t = __fadd_rn(__fsub_rn(c.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  return ffz(s, __fadd_rn(__fadd_rn(c.lo, e), t));
}
__device__ __forceinline__ ffl ffl_of(ffz a) {   // renormalise (TwoSum: no ordering of |hi|, |lo| assumed)
  const float s = __fadd_rn(a.hi, a.lo);
  const float bb = __fsub_rn(s, a.hi);
  return ffl(s, __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(a.lo, bb)));
}

__device__ __forceinline__ int sel4(const int (&v)[4], int mu) {
  return mu == 0 ? v[0] : mu == 1 ? v[1] : mu == 2 ? v[2] : v[3];
}

// out = hop(in) at `site` in float-float (in: float-float field, HALF: one parity indexed
// site >> 1).  The eight directions run in a loop that is not unrolled: one copy of the SU(3)
// product serves all of them (a backward link enters as its adjoint, formed in registers),
// since the fully unrolled float-float hop overflows the instruction cache.
template <int SPR, int LPR, int REC, bool HALF>
__device__ __forceinline__ void hop_ff(const LatGeom& g, FieldPtr in, int Vmax, int slot, int site,
                                       const int (&x)[4], const int (&st)[4], cplx<ffl> (&out)[12]) {
  static_assert(SPR == PRFF && LPR == PRFF, "float-float field and links");
  cplx<ffz> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {ffz(0), ffz(0)};
  int L4[4] = {g.L[0], g.L[1], g.L[2], g.L[3]};
#pragma unroll 1
  for (int d = 0; d < 8; ++d) {
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    const int xm = sel4(x, mu), sm = sel4(st, mu), L = sel4(L4, mu);
    const int nb = fwd ? ((xm + 1 == L) ? site - (L - 1) * sm : site + sm)
                       : ((xm == 0) ? site + (L - 1) * sm : site - sm);
    cplx<ffz> u[9], psi[12], h[6], w[6];
    {
      cplx<ffl> ul[9], pl[12];
      LinkIO<LPR, REC>::load(g, mu, fwd ? site : nb, ul);
      SpinorIO<SPR>::load_nc(in, Vmax, slot, HALF ? nb >> 1 : nb, pl);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const cplx<ffl> e = fwd ? ul[3 * r + c] : ul[3 * c + r];   // U or U^dagger
          u[3 * r + c] = {ffz(e.x.hi, e.x.lo), fwd ? ffz(e.y.hi, e.y.lo) : ffz(-e.y.hi, -e.y.lo)};
        }
#pragma unroll
      for (int k = 0; k < 12; ++k) psi[k] = {ffz(pl[k].x.hi, pl[k].x.lo), ffz(pl[k].y.hi, pl[k].y.lo)};
    }
    switch (d) {
      case 0: project<0, -1>(psi, h); break;
      case 1: project<0, 1>(psi, h); break;
      case 2: project<1, -1>(psi, h); break;
      case 3: project<1, 1>(psi, h); break;
      case 4: project<2, -1>(psi, h); break;
      case 5: project<2, 1>(psi, h); break;
      case 6: project<3, -1>(psi, h); break;
      default: project<3, 1>(psi, h); break;
    }
    su3_mul<ffz, false>(u, h, w);
    switch (d) {
      case 0: accumulate<0, -1>(acc, w); break;
      case 1: accumulate<0, 1>(acc, w); break;
      case 2: accumulate<1, -1>(acc, w); break;
      case 3: accumulate<1, 1>(acc, w); break;
      case 4: accumulate<2, -1>(acc, w); break;
      case 5: accumulate<2, 1>(acc, w); break;
      case 6: accumulate<3, -1>(acc, w); break;
      default: accumulate<3, 1>(acc, w); break;
    }
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) out[k] = {ffl_of(acc[k].x), ffl_of(acc[k].y)};
}

// hop = sum_mu [(1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^H psi(x-mu)]
template <int SPR, int LPR, typename R>
__device__ __forceinline__ void wilson_hop(const LatGeom& g, FieldPtr in, int Vmax, int slot, int site,
                                           const int (&x)[4], const int (&st)[4], cplx<R> (&acc)[12]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {0, 0};
  if constexpr (is_ffl<R>::value) {
    hop_ff<SPR, LPR, 12, false>(g, in, Vmax, slot, site, x, st, acc);
    return;
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int L = g.L[mu];
    const int fw = (x[mu] + 1 == L) ? site - (L - 1) * st[mu] : site + st[mu];
    const int bw = (x[mu] == 0) ? site + (L - 1) * st[mu] : site - st[mu];
    cplx<R> psi[12], h[6], w[6], u[9];
    SpinorIO<SPR>::load_nc(in, Vmax, slot, fw, psi);
    LinkIO<LPR>::load(g, mu, site, u);
    if (mu == 0) project<0, -1>(psi, h);
    if (mu == 1) project<1, -1>(psi, h);
    if (mu == 2) project<2, -1>(psi, h);
    if (mu == 3) project<3, -1>(psi, h);
    su3_mul<R, false>(u, h, w);
    if (mu == 0) accumulate<0, -1>(acc, w);
    if (mu == 1) accumulate<1, -1>(acc, w);
    if (mu == 2) accumulate<2, -1>(acc, w);
    if (mu == 3) accumulate<3, -1>(acc, w);
    SpinorIO<SPR>::load_nc(in, Vmax, slot, bw, psi);
    LinkIO<LPR>::load(g, mu, bw, u);
    if (mu == 0) project<0, 1>(psi, h);
    if (mu == 1) project<1, 1>(psi, h);
    if (mu == 2) project<2, 1>(psi, h);
    if (mu == 3) project<3, 1>(psi, h);
    su3_mul<R, true>(u, h, w);
    if (mu == 0) accumulate<0, 1>(acc, w);
    if (mu == 1) accumulate<1, 1>(acc, w);
    if (mu == 2) accumulate<2, 1>(acc, w);
    if (mu == 3) accumulate<3, 1>(acc, w);
  }
}

// ---- the clover diagonal A(x) (or A(x)^-1): two packed Hermitian 6x6 blocks per site
template <typename R>
struct ClovLoad;
template <>
struct ClovLoad<double> {
  __device__ static __forceinline__ void load(const LatGeom& g, bool inv, int site, int b, double (&a)[36]) {
    const double2* p = (inv ? g.Ai64 : g.A64) + (size_t)(18 * b) * g.V + site;
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      const double2 v = __ldg(p + (size_t)k * g.V);
      a[2 * k] = v.x;
      a[2 * k + 1] = v.y;
    }
  }
};
template <>
struct ClovLoad<float> {
  __device__ static __forceinline__ void load(const LatGeom& g, bool inv, int site, int b, float (&a)[36]) {
    const float4* p = (inv ? g.Ai32 : g.A32) + (size_t)(9 * b) * g.V + site;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float4 v = __ldg(p + (size_t)k * g.V);
      a[4 * k] = v.x;
      a[4 * k + 1] = v.y;
      a[4 * k + 2] = v.z;
      a[4 * k + 3] = v.w;
    }
  }
};
template <>
struct ClovLoad<ffl> {
  __device__ static __forceinline__ void load(const LatGeom& g, bool inv, int site, int b, ffl (&a)[36]) {
    const float4* p = (inv ? g.Ai32 : g.A32) + (size_t)(9 * b) * g.V + site;
    const float4* q = (inv ? g.Ai32l : g.A32l) + (size_t)(9 * b) * g.V + site;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float4 v = __ldg(p + (size_t)k * g.V), w = __ldg(q + (size_t)k * g.V);
      a[4 * k] = ffl(v.x, w.x);
      a[4 * k + 1] = ffl(v.y, w.y);
      a[4 * k + 2] = ffl(v.z, w.z);
      a[4 * k + 3] = ffl(v.w, w.w);
    }
  }
};

// out = A(x) in (inv: A(x)^-1 in); block b acts on components 6b..6b+5 (spins 2b, 2b+1)
template <typename R>
__device__ __forceinline__ void clover_mul(const LatGeom& g, bool inv, int site, const cplx<R> (&in)[12],
                                           cplx<R> (&out)[12]) {
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    R a[36];
    ClovLoad<R>::load(g, inv, site, b, a);
    cplx<R> y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) y[i] = {a[i] * in[6 * b + i].x, a[i] * in[6 * b + i].y};
    int k = 6;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i + 1; j < 6; ++j) {
        const R ax = a[k], ay = a[k + 1];
        k += 2;
        const cplx<R> xi = in[6 * b + i], xj = in[6 * b + j];
        y[i].x = fma(ax, xj.x, y[i].x);   // y_i += A_ij x_j
        y[i].x = fma(-ay, xj.y, y[i].x);
        y[i].y = fma(ax, xj.y, y[i].y);
        y[i].y = fma(ay, xj.x, y[i].y);
        y[j].x = fma(ax, xi.x, y[j].x);   // y_j += conj(A_ij) x_i
        y[j].x = fma(ay, xi.y, y[j].x);
        y[j].y = fma(ax, xi.y, y[j].y);
        y[j].y = fma(-ay, xi.x, y[j].y);
      }
#pragma unroll
    for (int i = 0; i < 6; ++i) out[6 * b + i] = y[i];
  }
}

// float-float: the same products with lazily normalised sums (ffz), one renormalisation per entry
template <>
__device__ __forceinline__ void clover_mul<ffl>(const LatGeom& g, bool inv, int site, const cplx<ffl> (&in)[12],
                                                cplx<ffl> (&out)[12]) {
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    ffz a[36];
    {
      ffl al[36];
      ClovLoad<ffl>::load(g, inv, site, b, al);
#pragma unroll
      for (int k = 0; k < 36; ++k) a[k] = ffz(al[k].hi, al[k].lo);
    }
    cplx<ffz> x[6], y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      x[i] = {ffz(in[6 * b + i].x.hi, in[6 * b + i].x.lo), ffz(in[6 * b + i].y.hi, in[6 * b + i].y.lo)};
      y[i] = {fma(a[i], x[i].x, ffz(0)), fma(a[i], x[i].y, ffz(0))};
    }
    int k = 6;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i + 1; j < 6; ++j) {
        const ffz ax = a[k], ay = a[k + 1];
        k += 2;
        y[i].x = fma(ax, x[j].x, y[i].x);
        y[i].x = fma(-ay, x[j].y, y[i].x);
        y[i].y = fma(ax, x[j].y, y[i].y);
        y[i].y = fma(ay, x[j].x, y[i].y);
        y[j].x = fma(ax, x[i].x, y[j].x);
        y[j].x = fma(ay, x[i].y, y[j].x);
        y[j].y = fma(ax, x[i].y, y[j].y);
        y[j].y = fma(-ay, x[i].x, y[j].y);
      }
#pragma unroll
    for (int i = 0; i < 6; ++i) out[6 * b + i] = {ffl_of(y[i].x), ffl_of(y[i].y)};
  }
}

// (D psi)(x) = (1 + m + mu(x)) psi(x) - kappa hop, or A(x) psi(x) - kappa hop with the clover
// term; psi(x) returned in `center`
template <int SPR, int LPR, typename R>
__device__ __forceinline__ void wilson_site(const LatGeom& g, FieldPtr in, int Vmax, int slot, int site,
                                            cplx<R> (&out)[12], cplx<R> (&center)[12]) {
  int x[4], st[4];
  site_coords(g, site, x, st);
  cplx<R> hop[12];
  wilson_hop<SPR, LPR, R>(g, in, Vmax, slot, site, x, st, hop);
  SpinorIO<SPR>::load_nc(in, Vmax, slot, site, center);
  R kap = (R)g.kappa;
  if (g.clover) {   // A(x) psi(x) - kappa hop
    cplx<R> ac[12];
    clover_mul<R>(g, false, site, center, ac);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      out[k].x = ac[k].x - kap * hop[k].x;
      out[k].y = ac[k].y - kap * hop[k].y;
    }
    return;
  }
  R diag = (R)(1.0 + g.mass + (g.mass_field ? g.mass_field[site] : 0.0));
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    out[k].x = diag * center[k].x - kap * hop[k].x;
    out[k].y = diag * center[k].y - kap * hop[k].y;
  }
}

// the source v_{m,a}(site) = (z_0 (.) z_m)(site) e_a, value of its non-zero component
__device__ __forceinline__ double2 source_value(const LatGeom& g, int site, int m) {
  return g.ptab[probe_phase(g, (uint32_t)site, (uint32_t)m)];
}
