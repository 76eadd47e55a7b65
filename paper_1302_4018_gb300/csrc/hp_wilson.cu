// Wilson-Dirac operator: link preparation and the dispatch of the apply, stencil benchmark and
// solver calls to the per-precision translation units (hp_wilson_impl.cuh: the stencil in
// FP64/FP32/FP16/BF16 and the multi-right-hand-side BiCGStab with FP64-class reliable updates
// that computes the quadratures v^H D^-1 v of the probing sources; Section 1.1.2: quadrature
// through a linear solve; Section 5.3: full spin-colour dilution).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "hp_fields.cuh"

// ============================================================ link preparation
// canonical complex128 [V][4][3][3]  ->  internal layouts
__global__ void k_links_convert(const double2* __restrict__ in, int V, double2* __restrict__ U64,
                                float4* __restrict__ U32, uint2* __restrict__ U16, float4* __restrict__ U32f,
                                float2* __restrict__ U32g, uint4* __restrict__ U16f, unsigned int* __restrict__ U16g,
                                float4* __restrict__ U32fl, float2* __restrict__ U32gl) {
  const long long total = 4LL * V;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int site = (int)(t >> 2), mu = (int)(t & 3);
    double2 u[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = in[((size_t)site * 4 + mu) * 9 + k];
    if (U64) {
#pragma unroll
      for (int k = 0; k < 9; ++k) U64[((size_t)mu * 9 + k) * V + site] = u[k];
    }
    if (U32) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
        U32[((size_t)mu * 3 + k) * V + site] =
            make_float4((float)u[2 * k].x, (float)u[2 * k].y, (float)u[2 * k + 1].x, (float)u[2 * k + 1].y);
    }
    if (U16) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        uint2 v;
        v.x = Half2Ops<PR16>::from_f2((float)u[2 * k].x, (float)u[2 * k].y);
        v.y = Half2Ops<PR16>::from_f2((float)u[2 * k + 1].x, (float)u[2 * k + 1].y);
        U16[((size_t)mu * 3 + k) * V + site] = v;
      }
    }
    if (U32f) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        U32f[((size_t)mu * 4 + k) * V + site] =
            make_float4((float)u[2 * k].x, (float)u[2 * k].y, (float)u[2 * k + 1].x, (float)u[2 * k + 1].y);
      U32g[(size_t)mu * V + site] = make_float2((float)u[8].x, (float)u[8].y);
    }
    if (U32fl) {   // low parts of the float-float links: u - (float)u, exact in FP32
      auto lo = [](double v) { return (float)(v - (double)(float)v); };
#pragma unroll
      for (int k = 0; k < 4; ++k)
        U32fl[((size_t)mu * 4 + k) * V + site] =
            make_float4(lo(u[2 * k].x), lo(u[2 * k].y), lo(u[2 * k + 1].x), lo(u[2 * k + 1].y));
      U32gl[(size_t)mu * V + site] = make_float2(lo(u[8].x), lo(u[8].y));
    }
    if (U16f) {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        uint4 v;
        v.x = Half2Ops<PR16>::from_f2((float)u[4 * k].x, (float)u[4 * k].y);
        v.y = Half2Ops<PR16>::from_f2((float)u[4 * k + 1].x, (float)u[4 * k + 1].y);
        v.z = Half2Ops<PR16>::from_f2((float)u[4 * k + 2].x, (float)u[4 * k + 2].y);
        v.w = Half2Ops<PR16>::from_f2((float)u[4 * k + 3].x, (float)u[4 * k + 3].y);
        U16f[((size_t)mu * 2 + k) * V + site] = v;
      }
      U16g[(size_t)mu * V + site] = Half2Ops<PR16>::from_f2((float)u[8].x, (float)u[8].y);
    }
  }
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = (float)in[i];
}

hp_status hp_prepare_mass(hp_ctx* ctx, const hp_operator* op, LatGeom* g, const char* tag) {
  g->mass = op->mass;
  g->kappa = op->kappa;
  g->diag0 = (float)(1.0 + op->mass);
  g->mass_field = nullptr;
  g->mass_field32 = nullptr;
  if (op->mass_field) {
    std::string n = std::string(tag) + ".mass";
    const void* d = nullptr;
    HP_TRY(hp_device_view(ctx, op->mass_field, sizeof(double) * (size_t)g->V, n.c_str(), &d));
    g->mass_field = (const double*)d;
    void* f = nullptr;
    HP_TRY(hp_ws(ctx, (n + "32").c_str(), sizeof(float) * (size_t)g->V, &f));
    {
      ProfScope ps(ctx, "k_to_float");
      k_to_float<<<blocks_for(ctx, g->V, 256), 256, 0, ctx->stream>>>(g->mass_field, (float*)f, g->V);
    }
    HP_LAUNCH_CHECK();
    g->mass_field32 = (const float*)f;
  }
  return HP_OK;
}

// need_prec: bit mask of (1 << PR64) | (1 << PR32) | (1 << PR16)
hp_status hp_prepare_wilson(hp_ctx* ctx, const hp_operator* op, LatGeom* g, const char* tag, int need_prec) {
  if (!op->links) {
    hp_set_error("Wilson operator without links");
    return HP_EINVAL;
  }
  const size_t V = (size_t)g->V;
  std::string base(tag);
  const void* src = nullptr;
  // read once, by the conversion below: pinned host links stream in over the host link directly
  HP_TRY(hp_stream_view(ctx, op->links, sizeof(double) * 72 * V, (base + ".links_in").c_str(), &src));
  void *u64 = nullptr, *u32 = nullptr, *u16 = nullptr, *u32f = nullptr, *u32g = nullptr, *u16f = nullptr,
       *u16g = nullptr, *u32fl = nullptr, *u32gl = nullptr;
  HP_TRY(hp_ws(ctx, (base + ".U64").c_str(), sizeof(double2) * 36 * V, &u64));   // always: true residual
  if (need_prec & (1 << PR32)) {
    HP_TRY(hp_ws(ctx, (base + ".U32").c_str(), sizeof(float4) * 12 * V, &u32));
    HP_TRY(hp_ws(ctx, (base + ".U32f").c_str(), sizeof(float4) * 16 * V, &u32f));
    HP_TRY(hp_ws(ctx, (base + ".U32g").c_str(), sizeof(float2) * 4 * V, &u32g));
    HP_TRY(hp_ws(ctx, (base + ".U32fl").c_str(), sizeof(float4) * 16 * V, &u32fl));
    HP_TRY(hp_ws(ctx, (base + ".U32gl").c_str(), sizeof(float2) * 4 * V, &u32gl));
  }
  if (need_prec & (1 << PR16)) {
    HP_TRY(hp_ws(ctx, (base + ".U16").c_str(), sizeof(uint2) * 12 * V, &u16));
    HP_TRY(hp_ws(ctx, (base + ".U16f").c_str(), sizeof(uint4) * 8 * V, &u16f));
    HP_TRY(hp_ws(ctx, (base + ".U16g").c_str(), sizeof(unsigned int) * 4 * V, &u16g));
  }
  {
    ProfScope ps(ctx, "k_links_convert");
    k_links_convert<<<blocks_for(ctx, 4LL * V, 256), 256, 0, ctx->stream>>>(
        (const double2*)src, (int)V, (double2*)u64, (float4*)u32, (uint2*)u16, (float4*)u32f, (float2*)u32g,
        (uint4*)u16f, (unsigned int*)u16g, (float4*)u32fl, (float2*)u32gl);
  }
  HP_LAUNCH_CHECK();
  g->U64 = (const double2*)u64;
  g->U32 = (const float4*)u32;
  g->U16 = (const uint2*)u16;
  g->U32f = (const float4*)u32f;
  g->U32g = (const float2*)u32g;
  g->U16f = (const uint4*)u16f;
  g->U16g = (const unsigned int*)u16g;
  g->U32fl = (const float4*)u32fl;
  g->U32gl = (const float2*)u32gl;
  return hp_prepare_clover(ctx, op, g, tag);
}


// per-precision Wilson entry points (hp_wilson_<precision>.cu)
#define HP_WILSON_DECLARE(SUFFIX)                                                                             \
  hp_status hp_wilson_apply_##SUFFIX(hp_ctx* ctx, const LatGeom& g, int nrhs, const double* in, double* out); \
  hp_status hp_wilson_bench_##SUFFIX(hp_ctx* ctx, const LatGeom& g, int nrhs, int iters, double* ms);         \
  hp_status hp_wilson_schur_##SUFFIX(hp_ctx* ctx, const LatGeom& g, int nrhs, int eo_kernel, const double* in,   \
                                      double* out);                                                           \
  hp_status hp_wilson_solve_##SUFFIX(hp_ctx* ctx, SolveProblem& pb, SolveResult& res, bool eo, bool clover,   \
                                     double delta);
HP_WILSON_DECLARE(fp64)
HP_WILSON_DECLARE(fp32)
HP_WILSON_DECLARE(fp16)
HP_WILSON_DECLARE(bf16)

hp_status hp_apply_wilson(hp_ctx* ctx, const hp_operator* op, LatGeom g, int nrhs, int prec, const double* in,
                          double* out) {
  HP_TRY(hp_prepare_mass(ctx, op, &g, "apply"));
  HP_TRY(hp_prepare_wilson(ctx, op, &g, "apply", (1 << PR64) | (1 << PR32) | (1 << PR16)));
  switch (prec) {
    case HP_PREC_FP64: return hp_wilson_apply_fp64(ctx, g, nrhs, in, out);
    case HP_PREC_MIXED_FP32: return hp_wilson_apply_fp32(ctx, g, nrhs, in, out);
    case HP_PREC_MIXED_FP16: return hp_wilson_apply_fp16(ctx, g, nrhs, in, out);
    case HP_PREC_MIXED_BF16: return hp_wilson_apply_bf16(ctx, g, nrhs, in, out);
  }
  hp_set_error("unknown precision %d", prec);
  return HP_EINVAL;
}

// The red-black split behind the even-odd iteration: every hop must join sites of opposite parity,
// which holds when all four extents are even (an odd extent wraps around between sites of one
// parity; a padded extent 1 hops onto the site itself); the half-site numbering site >> 1 then
// needs L_1 even as well.
static bool eo_lattice(const LatGeom& g) {
  for (int j = 0; j < 4; ++j)
    if (g.L[j] % 2) return false;
  return true;
}

hp_status hp_schur_wilson(hp_ctx* ctx, const hp_operator* op, LatGeom g, int nrhs, int prec, int eo_kernel,
                          const double* in, double* out) {
  if (!eo_lattice(g)) {
    hp_set_error("the even-odd split needs every extent even (lattice %d x %d x %d x %d; an odd or a padded "
                 "extent joins sites of one parity)", g.L[0], g.L[1], g.L[2], g.L[3]);
    return HP_EINVAL;
  }
  if (op->kappa == 0.0) {
    hp_set_error("the Schur complement needs kappa != 0");
    return HP_EINVAL;
  }
  HP_TRY(hp_prepare_mass(ctx, op, &g, "schur"));
  HP_TRY(hp_prepare_wilson(ctx, op, &g, "schur", (1 << PR64) | (1 << PR32) | (1 << PR16)));
  switch (prec) {
    case HP_PREC_FP64: return hp_wilson_schur_fp64(ctx, g, nrhs, eo_kernel, in, out);
    case HP_PREC_MIXED_FP32: return hp_wilson_schur_fp32(ctx, g, nrhs, eo_kernel, in, out);
    case HP_PREC_MIXED_FP16: return hp_wilson_schur_fp16(ctx, g, nrhs, eo_kernel, in, out);
    case HP_PREC_MIXED_BF16: return hp_wilson_schur_bf16(ctx, g, nrhs, eo_kernel, in, out);
  }
  hp_set_error("unknown precision %d", prec);
  return HP_EINVAL;
}

hp_status hp_bench_wilson(hp_ctx* ctx, const hp_operator* op, LatGeom g, int prec, int nrhs, int iters, double* ms,
                          double* bytes, double* flops) {
  HP_TRY(hp_prepare_mass(ctx, op, &g, "bench"));
  HP_TRY(hp_prepare_wilson(ctx, op, &g, "bench", (1 << PR64) | (1 << PR32) | (1 << PR16)));
  double S = 0, L = 0;
  hp_status st = HP_EINVAL;
  switch (prec) {
    case HP_PREC_FP64: S = 192; L = 144; st = hp_wilson_bench_fp64(ctx, g, nrhs, iters, ms); break;
    case HP_PREC_MIXED_FP32: S = 96; L = 48; st = hp_wilson_bench_fp32(ctx, g, nrhs, iters, ms); break;
    case HP_PREC_MIXED_FP16: S = 52; L = 24; st = hp_wilson_bench_fp16(ctx, g, nrhs, iters, ms); break;
    case HP_PREC_MIXED_BF16: S = 52; L = 24; st = hp_wilson_bench_bf16(ctx, g, nrhs, iters, ms); break;
    default: hp_set_error("unknown precision %d", prec); return HP_EINVAL;
  }
  if (st != HP_OK) return st;
  *bytes = (double)nrhs * g.V * (2.0 * S + 4.0 * L / nrhs);
  *flops = 1368.0 * nrhs * g.V;
  return HP_OK;
}

hp_status hp_solve_wilson(hp_ctx* ctx, SolveProblem& pb, SolveResult& res) {
  const int prec = pb.opts.precision;
  double delta = pb.opts.delta;
  bool eo = pb.opts.even_odd != 0, clover = false;
  for (auto& g : pb.lats) {
    if (!eo_lattice(g)) eo = false;   // odd or padded extents: no red-black split, full-lattice iteration
    clover = clover || g.clover;
  }
  // default group-update thresholds per iteration precision (measured on the 32^3x64 workload)
  switch (prec) {
    case HP_PREC_FP64: return hp_wilson_solve_fp64(ctx, pb, res, eo, clover, delta > 0 ? delta : 0.0);
    case HP_PREC_MIXED_FP32: return hp_wilson_solve_fp32(ctx, pb, res, eo, clover, delta > 0 ? delta : 0.001);
    case HP_PREC_MIXED_FP16: return hp_wilson_solve_fp16(ctx, pb, res, eo, clover, delta > 0 ? delta : 0.03);
    case HP_PREC_MIXED_BF16: return hp_wilson_solve_bf16(ctx, pb, res, eo, clover, delta > 0 ? delta : 0.03);
  }
  hp_set_error("unknown precision %d", prec);
  return HP_EINVAL;
}
