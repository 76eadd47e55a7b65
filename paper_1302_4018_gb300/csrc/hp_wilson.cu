// Wilson-Dirac operator: link preparation, the stencil in FP64/FP32/FP16/BF16,
// and the multi-right-hand-side BiCGStab with FP64 reliable updates that
// computes the quadratures v^H D^-1 v of the probing sources (Section 1.1.2:
// quadrature through a linear solve; Section 5.3: full spin-colour dilution).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "hp_fields.cuh"

// ============================================================ link preparation
// canonical complex128 [V][4][3][3]  ->  internal layouts
__global__ void k_links_convert(const double2* __restrict__ in, int V, double2* __restrict__ U64,
                                float4* __restrict__ U32, uint2* __restrict__ U16) {
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
  }
}

static int blocks_for(hp_ctx* ctx, long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  long long cap = (long long)ctx->num_sms * 16;
  return (int)std::max(1LL, std::min(b, cap));
}

hp_status hp_prepare_mass(hp_ctx* ctx, const hp_operator* op, LatGeom* g, const char* tag) {
  g->mass = op->mass;
  g->kappa = op->kappa;
  g->mass_field = nullptr;
  if (op->mass_field) {
    std::string n = std::string(tag) + ".mass";
    const void* d = nullptr;
    HP_TRY(hp_device_view(ctx, op->mass_field, sizeof(double) * (size_t)g->V, n.c_str(), &d));
    g->mass_field = (const double*)d;
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
  HP_TRY(hp_device_view(ctx, op->links, sizeof(double) * 72 * V, (base + ".links_in").c_str(), &src));
  void *u64 = nullptr, *u32 = nullptr, *u16 = nullptr;
  HP_TRY(hp_ws(ctx, (base + ".U64").c_str(), sizeof(double2) * 36 * V, &u64));   // always: true residual
  if (need_prec & (1 << PR32)) HP_TRY(hp_ws(ctx, (base + ".U32").c_str(), sizeof(float4) * 12 * V, &u32));
  if (need_prec & (1 << PR16)) HP_TRY(hp_ws(ctx, (base + ".U16").c_str(), sizeof(uint2) * 12 * V, &u16));
  {
    ProfScope ps(ctx, "k_links_convert");
    k_links_convert<<<blocks_for(ctx, 4LL * V, 256), 256, 0, ctx->stream>>>(
        (const double2*)src, (int)V, (double2*)u64, (float4*)u32, (uint2*)u16);
  }
  HP_LAUNCH_CHECK();
  g->U64 = (const double2*)u64;
  g->U32 = (const float4*)u32;
  g->U16 = (const uint2*)u16;
  return HP_OK;
}

// ================================================================ plain apply
template <int SPR>
__global__ void k_w_from_canonical(const double2* __restrict__ in, FieldPtr f, int V, int nrhs) {
  const long long total = (long long)nrhs * V;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int slot = (int)(t / V), site = (int)(t - (long long)slot * V);
    typedef typename Real_of<SPR>::T R;
    cplx<R> s[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 v = in[((size_t)slot * V + site) * 12 + k];
      s[k] = {(R)v.x, (R)v.y};
    }
    SpinorIO<SPR>::store(f, V, slot, site, s);
  }
}

template <int SPR>
__global__ void k_w_to_canonical(FieldPtr f, int V, int nrhs, double2* __restrict__ out) {
  const long long total = (long long)nrhs * V;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int slot = (int)(t / V), site = (int)(t - (long long)slot * V);
    typedef typename Real_of<SPR>::T R;
    cplx<R> s[12];
    SpinorIO<SPR>::load(f, V, slot, site, s);
#pragma unroll
    for (int k = 0; k < 12; ++k) out[((size_t)slot * V + site) * 12 + k] = make_double2((double)s[k].x, (double)s[k].y);
  }
}

// one launch: grid (nrhs, tiles); every thread one site of one right-hand side
template <int SPR, int NT>
__global__ void __launch_bounds__(NT) k_w_dslash(LatGeom g, FieldPtr in, FieldPtr out, int Vmax) {
  typedef typename Real_of<SPR>::T R;
  constexpr int LPR = LinkPrecOf<SPR>::v;
  const int slot = blockIdx.x;
  const int ntiles = (g.V + NT - 1) / NT;
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    cplx<R> o[12], c[12];
    wilson_site<SPR, LPR, R>(g, in, Vmax, slot, site, o, c);
    SpinorIO<SPR>::store(out, Vmax, slot, site, o);
  }
}

template <int SPR>
static size_t spinor_bytes_of() {
  return SPR == PR64 ? 192 : (SPR == PR32 ? 96 : 48);
}

static size_t field_bytes(int spr, int nslots, int Vmax, size_t* norm_bytes) {
  size_t per = spr == PR64 ? 192 : (spr == PR32 ? 96 : 48);
  *norm_bytes = (spr == PR16 || spr == PRB16) ? sizeof(float) * (size_t)nslots * Vmax : 0;
  return per * (size_t)nslots * Vmax;
}

static hp_status alloc_field(hp_ctx* ctx, const std::string& name, int spr, int nslots, int Vmax, FieldPtr* f) {
  size_t nb = 0;
  size_t b = field_bytes(spr, nslots, Vmax, &nb);
  HP_TRY(hp_ws(ctx, name.c_str(), b, &f->p));
  f->nrm = nullptr;
  if (nb) {
    void* q = nullptr;
    HP_TRY(hp_ws(ctx, (name + ".nrm").c_str(), nb, &q));
    f->nrm = (float*)q;
  }
  return HP_OK;
}

static int dslash_gridy(hp_ctx* ctx, int V, int NT, int nslots) {
  int ntiles = (V + NT - 1) / NT;
  int want = (ctx->num_sms * 16 + nslots - 1) / nslots;
  return std::max(1, std::min(std::min(ntiles, want), 65535));
}

template <int SPR>
static hp_status launch_dslash(hp_ctx* ctx, const LatGeom& g, FieldPtr in, FieldPtr out, int nrhs, int Vmax) {
  constexpr int NT = 128;
  dim3 grid(nrhs, dslash_gridy(ctx, g.V, NT, nrhs));
  {
    ProfScope ps(ctx, SPR == PR64 ? "k_w_dslash<fp64>" : SPR == PR32 ? "k_w_dslash<fp32>" : SPR == PR16 ? "k_w_dslash<fp16>" : "k_w_dslash<bf16>");
    k_w_dslash<SPR, NT><<<grid, NT, 0, ctx->stream>>>(g, in, out, Vmax);
  }
  HP_LAUNCH_CHECK();
  return HP_OK;
}

template <int SPR>
static hp_status apply_wilson_t(hp_ctx* ctx, const LatGeom& g, int nrhs, const double* in, double* out) {
  const int V = g.V;
  FieldPtr fi, fo;
  HP_TRY(alloc_field(ctx, "apply.in", SPR, nrhs, V, &fi));
  HP_TRY(alloc_field(ctx, "apply.out", SPR, nrhs, V, &fo));
  const size_t cbytes = sizeof(double2) * 12 * (size_t)nrhs * V;
  const void* din = nullptr;
  HP_TRY(hp_device_view(ctx, in, cbytes, "apply.canon_in", &din));
  double* dout = out;
  bool out_host = !hp_is_device_ptr(out);
  if (out_host) {
    void* p = nullptr;
    HP_TRY(hp_ws(ctx, "apply.canon_out", cbytes, &p));
    dout = (double*)p;
  }
  k_w_from_canonical<SPR><<<blocks_for(ctx, (long long)nrhs * V, 256), 256, 0, ctx->stream>>>((const double2*)din, fi, V, nrhs);
  HP_LAUNCH_CHECK();
  HP_TRY(launch_dslash<SPR>(ctx, g, fi, fo, nrhs, V));
  k_w_to_canonical<SPR><<<blocks_for(ctx, (long long)nrhs * V, 256), 256, 0, ctx->stream>>>(fo, V, nrhs, (double2*)dout);
  HP_LAUNCH_CHECK();
  if (out_host) {
    HP_CUDA(cudaMemcpyAsync(out, dout, cbytes, cudaMemcpyDeviceToHost, ctx->stream));
    HP_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  return HP_OK;
}

hp_status hp_apply_wilson(hp_ctx* ctx, const hp_operator* op, LatGeom g, int nrhs, int prec, const double* in,
                          double* out) {
  HP_TRY(hp_prepare_mass(ctx, op, &g, "apply"));
  HP_TRY(hp_prepare_wilson(ctx, op, &g, "apply", (1 << PR64) | (1 << PR32) | (1 << PR16)));
  switch (prec) {
    case HP_PREC_FP64: return apply_wilson_t<PR64>(ctx, g, nrhs, in, out);
    case HP_PREC_MIXED_FP32: return apply_wilson_t<PR32>(ctx, g, nrhs, in, out);
    case HP_PREC_MIXED_FP16: return apply_wilson_t<PR16>(ctx, g, nrhs, in, out);
    case HP_PREC_MIXED_BF16: return apply_wilson_t<PRB16>(ctx, g, nrhs, in, out);
  }
  hp_set_error("unknown precision %d", prec);
  return HP_EINVAL;
}

// fills a field with deterministic pseudo-random values (benchmark input)
template <int SPR>
__global__ void k_w_fill(FieldPtr f, int V, int nrhs, unsigned long long seed) {
  const long long total = (long long)nrhs * V;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int slot = (int)(t / V), site = (int)(t - (long long)slot * V);
    typedef typename Real_of<SPR>::T R;
    cplx<R> s[12];
    unsigned long long z = seed ^ (unsigned long long)t * 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      z = z * 6364136223846793005ull + 1442695040888963407ull;
      s[k] = {(R)((double)(z >> 40) / 16777216.0 - 0.5), (R)((double)((z >> 16) & 0xffffff) / 16777216.0 - 0.5)};
    }
    SpinorIO<SPR>::store(f, V, slot, site, s);
  }
}

template <int SPR>
static hp_status bench_wilson_t(hp_ctx* ctx, const LatGeom& g, int nrhs, int iters, double* ms) {
  const int V = g.V;
  FieldPtr fi, fo;
  HP_TRY(alloc_field(ctx, "bench.in", SPR, nrhs, V, &fi));
  HP_TRY(alloc_field(ctx, "bench.out", SPR, nrhs, V, &fo));
  k_w_fill<SPR><<<blocks_for(ctx, (long long)nrhs * V, 256), 256, 0, ctx->stream>>>(fi, V, nrhs, 12345ull);
  HP_LAUNCH_CHECK();
  for (int w = 0; w < 3; ++w) HP_TRY(launch_dslash<SPR>(ctx, g, fi, fo, nrhs, V));
  cudaEvent_t a, b;
  HP_CUDA(cudaEventCreate(&a));
  HP_CUDA(cudaEventCreate(&b));
  HP_CUDA(cudaEventRecord(a, ctx->stream));
  for (int i = 0; i < iters; ++i) HP_TRY(launch_dslash<SPR>(ctx, g, fi, fo, nrhs, V));
  HP_CUDA(cudaEventRecord(b, ctx->stream));
  HP_CUDA(cudaEventSynchronize(b));
  float t = 0.f;
  HP_CUDA(cudaEventElapsedTime(&t, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = (double)t / iters;
  return HP_OK;
}

hp_status hp_bench_wilson(hp_ctx* ctx, const hp_operator* op, LatGeom g, int prec, int nrhs, int iters, double* ms,
                          double* bytes, double* flops) {
  HP_TRY(hp_prepare_mass(ctx, op, &g, "bench"));
  HP_TRY(hp_prepare_wilson(ctx, op, &g, "bench", (1 << PR64) | (1 << PR32) | (1 << PR16)));
  double S = 0, L = 0;
  hp_status st = HP_EINVAL;
  switch (prec) {
    case HP_PREC_FP64: S = 192; L = 144; st = bench_wilson_t<PR64>(ctx, g, nrhs, iters, ms); break;
    case HP_PREC_MIXED_FP32: S = 96; L = 48; st = bench_wilson_t<PR32>(ctx, g, nrhs, iters, ms); break;
    case HP_PREC_MIXED_FP16: S = 52; L = 24; st = bench_wilson_t<PR16>(ctx, g, nrhs, iters, ms); break;
    case HP_PREC_MIXED_BF16: S = 52; L = 24; st = bench_wilson_t<PRB16>(ctx, g, nrhs, iters, ms); break;
    default: hp_set_error("unknown precision %d", prec); return HP_EINVAL;
  }
  if (st != HP_OK) return st;
  *bytes = (double)nrhs * g.V * (2.0 * S + 4.0 * L / nrhs);
  *flops = 1368.0 * nrhs * g.V;
  return HP_OK;
}

// ==================================================================== solver
// Per slot (right-hand side) BiCGStab, x_0 = 0, shadow r^ = b:
//   v = D p; alpha = rho / (r^, v); s = r - alpha v; t = D s;
//   omega = (t, s) / (t, t); e += alpha p + omega s; r = s - omega t;
//   rho' = (r^, r); beta = (rho'/rho)(alpha/omega); p = r + beta (p - omega v)
// in the iteration precision.  Reliable update (FP64) whenever ||r|| drops
// below delta * (largest ||r|| since the last update) or below tol ||b||:
//   x += e; e = 0; r = b - D x (FP64 stencil, FP64 links); stop when that
//   true residual <= tol ||b||.
// All scalars live per slot in device memory; reductions are deterministic
// (fixed shuffle trees, per-block partials summed in block order by the
// block that finishes last).
struct WArgs {
  const LatGeom* lats;
  SlotState* st;
  double* part;          // [nslots][4][gy]
  unsigned int* cnt;     // [nslots]
  int Vmax, gy;
  FieldPtr r, rh, p, v, s, t, e;
  double2* x;            // FP64 solution [slot][12][Vmax]
  double* grad;          // unused here
  double tol2, delta2;
  int maxiter;
};

#define SLOT_PREAMBLE(COND)                                        \
  const int slot = blockIdx.x;                                     \
  SlotState* S = a.st + slot;                                      \
  if (!(COND)) return;                                             \
  const LatGeom& g = a.lats[S->lat];                               \
  const int ntiles = (g.V + NT - 1) / NT;                          \
  if ((int)blockIdx.y >= ntiles) return;                           \
  const int nparts = min((int)gridDim.y, ntiles);                  \
  double* part = a.part + (size_t)slot * 4 * a.gy;                 \
  (void)nparts;                                                    \
  (void)part;

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  if (d == 0.0) return make_double2(0.0, 0.0);
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 dmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <typename R, int NQ, int NT>
__device__ __forceinline__ void reduce_partials(R (&v)[NQ], double* part, int gy) {
  double dv[NQ];
  // warp level in the iteration precision, across warps in FP64
  __shared__ double sh[NQ][NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    R t = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[q][warp] = (double)t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += sh[q][w];
      dv[q] = t;
      part[(size_t)q * gy + blockIdx.y] = t;
    }
  }
}

// ---- init: x = 0, e = 0, r = r^ = p = b, ||b||^2
template <int SPR, int EPR, int NT>
__global__ void __launch_bounds__(NT) k_bicg_init(WArgs a) {
  SLOT_PREAMBLE(S->status == SLOT_INIT)
  typedef typename Real_of<SPR>::T R;
  double acc[1] = {0.0};
  const int comp = S->a, m = S->m;
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    double2 bv = source_value(g, site, m);
    cplx<R> b[12];
    cplx<double> z[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      b[k] = {(R)0, (R)0};
      z[k] = {0.0, 0.0};
    }
#pragma unroll
    for (int k = 0; k < 12; ++k)
      if (k == comp) b[k] = {(R)bv.x, (R)bv.y};
    SpinorIO<PR64>::store(FieldPtr{a.x, nullptr}, a.Vmax, slot, site, z);
    {
      cplx<float> zf[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) zf[k] = {0.f, 0.f};
      if (EPR == PR64) SpinorIO<PR64>::store(a.e, a.Vmax, slot, site, z);
      else SpinorIO<PR32>::store(a.e, a.Vmax, slot, site, zf);
    }
    SpinorIO<SPR>::store(a.r, a.Vmax, slot, site, b);
    SpinorIO<SPR>::store(a.rh, a.Vmax, slot, site, b);
    SpinorIO<SPR>::store(a.p, a.Vmax, slot, site, b);
    acc[0] += bv.x * bv.x + bv.y * bv.y;
  }
  reduce_partials<double, 1, NT>(acc, part, a.gy);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[1];
    block_sum_partials<1, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      S->bnorm2 = tot[0];
      S->rnorm2 = tot[0];
      S->rmax2 = tot[0];
      S->rho = make_double2(tot[0], 0.0);
      S->alpha = make_double2(1.0, 0.0);
      S->omega = make_double2(1.0, 0.0);
      S->beta = make_double2(0.0, 0.0);
      S->iters = 0;
      S->updates = 0;
      S->need_update = 0;
      S->restart = 0;
      S->sloppy_mv = 0;
      S->fp64_mv = 0;
      S->true_res2 = tot[0];
      S->status = tot[0] > 0.0 ? SLOT_RUN : SLOT_DONE;
      a.cnt[slot] = 0;
    }
  }
}

// ---- v = D p ; sigma = (r^, v) ; alpha = rho / sigma
template <int SPR, int NT>
__global__ void __launch_bounds__(NT) k_bicg_v(WArgs a) {
  SLOT_PREAMBLE(S->status == SLOT_RUN)
  typedef typename Real_of<SPR>::T R;
  constexpr int LPR = LinkPrecOf<SPR>::v;
  R acc[2] = {0, 0};
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    cplx<R> o[12], c[12], rh[12];
    wilson_site<SPR, LPR, R>(g, a.p, a.Vmax, slot, site, o, c);
    SpinorIO<SPR>::store(a.v, a.Vmax, slot, site, o);
    SpinorIO<SPR>::load(a.rh, a.Vmax, slot, site, rh);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      cplx<R> d = cconjmul(rh[k], o[k]);
      acc[0] += d.x;
      acc[1] += d.y;
    }
  }
  reduce_partials<R, 2, NT>(acc, part, a.gy);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[2];
    block_sum_partials<2, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      double2 sigma = make_double2(tot[0], tot[1]);
      S->alpha = cdiv(S->rho, sigma);
      S->restart = 0;
      S->sloppy_mv += 1;
      a.cnt[slot] = 0;
    }
  }
}

// ---- s = r - alpha v
template <int SPR, int NT>
__global__ void __launch_bounds__(NT) k_bicg_s(WArgs a) {
  SLOT_PREAMBLE(S->status == SLOT_RUN)
  typedef typename Real_of<SPR>::T R;
  const double2 al = S->alpha;
  const R ax = (R)al.x, ay = (R)al.y;
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    cplx<R> r[12], v[12];
    SpinorIO<SPR>::load(a.r, a.Vmax, slot, site, r);
    SpinorIO<SPR>::load(a.v, a.Vmax, slot, site, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      r[k].x -= ax * v[k].x - ay * v[k].y;
      r[k].y -= ax * v[k].y + ay * v[k].x;
    }
    SpinorIO<SPR>::store(a.s, a.Vmax, slot, site, r);
  }
}

// ---- t = D s ; (t, s), (t, t) ; omega = (t, s) / (t, t)
template <int SPR, int NT>
__global__ void __launch_bounds__(NT) k_bicg_t(WArgs a) {
  SLOT_PREAMBLE(S->status == SLOT_RUN)
  typedef typename Real_of<SPR>::T R;
  constexpr int LPR = LinkPrecOf<SPR>::v;
  R acc[3] = {0, 0, 0};
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    cplx<R> o[12], c[12];
    wilson_site<SPR, LPR, R>(g, a.s, a.Vmax, slot, site, o, c);
    SpinorIO<SPR>::store(a.t, a.Vmax, slot, site, o);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      cplx<R> d = cconjmul(o[k], c[k]);
      acc[0] += d.x;
      acc[1] += d.y;
      acc[2] += o[k].x * o[k].x + o[k].y * o[k].y;
    }
  }
  reduce_partials<R, 3, NT>(acc, part, a.gy);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[3];
    block_sum_partials<3, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      S->omega = tot[2] > 0.0 ? make_double2(tot[0] / tot[2], tot[1] / tot[2]) : make_double2(0.0, 0.0);
      S->sloppy_mv += 1;
      a.cnt[slot] = 0;
    }
  }
}

// ---- e += alpha p + omega s ; r = s - omega t ; rho' = (r^, r) ; ||r||^2
template <int SPR, int EPR, int NT>
__global__ void __launch_bounds__(NT) k_bicg_xr(WArgs a) {
  SLOT_PREAMBLE(S->status == SLOT_RUN)
  typedef typename Real_of<SPR>::T R;
  typedef typename Real_of<EPR>::T RE;
  const double2 al = S->alpha, om = S->omega;
  R acc[3] = {0, 0, 0};
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    cplx<R> p[12], s[12], t[12], rh[12];
    cplx<RE> e[12];
    SpinorIO<SPR>::load(a.p, a.Vmax, slot, site, p);
    SpinorIO<SPR>::load(a.s, a.Vmax, slot, site, s);
    SpinorIO<SPR>::load(a.t, a.Vmax, slot, site, t);
    SpinorIO<SPR>::load(a.rh, a.Vmax, slot, site, rh);
    SpinorIO<EPR>::load(a.e, a.Vmax, slot, site, e);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      RE px = (RE)p[k].x, py = (RE)p[k].y, sx = (RE)s[k].x, sy = (RE)s[k].y;
      e[k].x += (RE)al.x * px - (RE)al.y * py + (RE)om.x * sx - (RE)om.y * sy;
      e[k].y += (RE)al.x * py + (RE)al.y * px + (RE)om.x * sy + (RE)om.y * sx;
      cplx<R> rn;
      rn.x = s[k].x - ((R)om.x * t[k].x - (R)om.y * t[k].y);
      rn.y = s[k].y - ((R)om.x * t[k].y + (R)om.y * t[k].x);
      s[k] = rn;
    }
    SpinorIO<EPR>::store(a.e, a.Vmax, slot, site, e);
    SpinorIO<SPR>::store(a.r, a.Vmax, slot, site, s);
    // dot products of the stored (rounded) residual
    if (SPR == PR16 || SPR == PRB16) SpinorIO<SPR>::load(a.r, a.Vmax, slot, site, s);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      cplx<R> d = cconjmul(rh[k], s[k]);
      acc[0] += d.x;
      acc[1] += d.y;
      acc[2] += s[k].x * s[k].x + s[k].y * s[k].y;
    }
  }
  reduce_partials<R, 3, NT>(acc, part, a.gy);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[3];
    block_sum_partials<3, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      double2 rho_new = make_double2(tot[0], tot[1]);
      double rr = tot[2];
      double2 om2 = S->omega, rho = S->rho;
      bool bad = (om2.x == 0.0 && om2.y == 0.0) || (rho.x == 0.0 && rho.y == 0.0) ||
                 (rho_new.x * rho_new.x + rho_new.y * rho_new.y) < 1e-28 * rr * S->rmax2 || !(rr == rr);
      if (bad) {
        S->restart = 1;               // r^ := r, p := r
        S->rho = make_double2(rr, 0.0);
        S->beta = make_double2(0.0, 0.0);
      } else {
        S->beta = dmul(cdiv(rho_new, rho), cdiv(S->alpha, om2));
        S->rho = rho_new;
      }
      S->rnorm2 = rr;
      S->iters += 1;
      if (S->iters >= a.maxiter) {
        S->status = SLOT_FAIL;
        S->need_update = 1;
      } else if (rr <= a.tol2 * S->bnorm2 || rr < a.delta2 * S->rmax2 || !(rr == rr)) {
        S->need_update = 1;
      }
      a.cnt[slot] = 0;
    }
  }
}

// ---- reliable update, part 1: x += e ; e = 0  (FP64)
template <int EPR, int NT>
__global__ void __launch_bounds__(NT) k_ru_accum(WArgs a) {
  SLOT_PREAMBLE(S->need_update)
  typedef typename Real_of<EPR>::T RE;
  FieldPtr xf{a.x, nullptr};
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    cplx<double> x[12];
    cplx<RE> e[12];
    SpinorIO<PR64>::load(xf, a.Vmax, slot, site, x);
    SpinorIO<EPR>::load(a.e, a.Vmax, slot, site, e);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      x[k].x += (double)e[k].x;
      x[k].y += (double)e[k].y;
      e[k] = {(RE)0, (RE)0};
    }
    SpinorIO<PR64>::store(xf, a.Vmax, slot, site, x);
    SpinorIO<EPR>::store(a.e, a.Vmax, slot, site, e);
  }
}

// ---- reliable update, part 2: r = b - D x in FP64, stored in the iteration precision
template <int SPR, int NT>
__global__ void __launch_bounds__(NT) k_ru_residual(WArgs a) {
  SLOT_PREAMBLE(S->need_update)
  typedef typename Real_of<SPR>::T R;
  double acc[3] = {0.0, 0.0, 0.0};
  const int comp = S->a, m = S->m;
  FieldPtr xf{a.x, nullptr};
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    cplx<double> o[12], c[12];
    wilson_site<PR64, PR64, double>(g, xf, a.Vmax, slot, site, o, c);
    double2 bv = source_value(g, site, m);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      o[k].x = -o[k].x;
      o[k].y = -o[k].y;
      if (k == comp) {
        o[k].x += bv.x;
        o[k].y += bv.y;
      }
    }
    cplx<R> rs[12], rh[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) rs[k] = {(R)o[k].x, (R)o[k].y};
    SpinorIO<SPR>::store(a.r, a.Vmax, slot, site, rs);
    SpinorIO<SPR>::load(a.rh, a.Vmax, slot, site, rh);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      acc[0] += o[k].x * o[k].x + o[k].y * o[k].y;
      acc[1] += (double)rh[k].x * o[k].x + (double)rh[k].y * o[k].y;
      acc[2] += (double)rh[k].x * o[k].y - (double)rh[k].y * o[k].x;
    }
  }
  reduce_partials<double, 3, NT>(acc, part, a.gy);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[3];
    block_sum_partials<3, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      double rr = tot[0];
      S->true_res2 = rr;
      S->updates += 1;
      S->fp64_mv += 1;
      S->need_update = 0;
      if (S->status == SLOT_RUN) {
        if (rr <= a.tol2 * S->bnorm2) {
          S->status = SLOT_DONE;
        } else {
          S->rnorm2 = rr;
          S->rmax2 = rr;
          S->rho = S->restart ? make_double2(rr, 0.0) : make_double2(tot[1], tot[2]);
        }
      }
      a.cnt[slot] = 0;
    }
  }
}

// ---- p = r + beta (p - omega v)   (restart: p = r^ = r)
template <int SPR, int NT>
__global__ void __launch_bounds__(NT) k_bicg_p(WArgs a) {
  SLOT_PREAMBLE(S->status == SLOT_RUN)
  typedef typename Real_of<SPR>::T R;
  const double2 be = S->beta, om = S->omega;
  const int restart = S->restart;
  const R bx = (R)be.x, by = (R)be.y, ox = (R)om.x, oy = (R)om.y;
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    cplx<R> r[12], p[12], v[12];
    SpinorIO<SPR>::load(a.r, a.Vmax, slot, site, r);
    if (restart) {
      SpinorIO<SPR>::store(a.p, a.Vmax, slot, site, r);
      SpinorIO<SPR>::store(a.rh, a.Vmax, slot, site, r);
      continue;
    }
    SpinorIO<SPR>::load(a.p, a.Vmax, slot, site, p);
    SpinorIO<SPR>::load(a.v, a.Vmax, slot, site, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      R dx = p[k].x - (ox * v[k].x - oy * v[k].y);
      R dy = p[k].y - (ox * v[k].y + oy * v[k].x);
      p[k].x = r[k].x + (bx * dx - by * dy);
      p[k].y = r[k].y + (bx * dy + by * dx);
    }
    SpinorIO<SPR>::store(a.p, a.Vmax, slot, site, p);
  }
}

// ---- harvest: q = v^H x = sum_site conj(v(site)) x(site, a)   (FP64)
template <int NT>
__global__ void __launch_bounds__(NT) k_quad(WArgs a) {
  SLOT_PREAMBLE(S->status == SLOT_DONE || S->status == SLOT_FAIL)
  double acc[2] = {0.0, 0.0};
  const int comp = S->a, m = S->m;
  const double2* x = a.x + ((size_t)slot * 12 + comp) * a.Vmax;
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    double2 bv = source_value(g, site, m);
    double2 xv = x[site];
    acc[0] += bv.x * xv.x + bv.y * xv.y;
    acc[1] += bv.x * xv.y - bv.y * xv.x;
  }
  reduce_partials<double, 2, NT>(acc, part, a.gy);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[2];
    block_sum_partials<2, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      S->q = make_double2(tot[0], tot[1]);
      a.cnt[slot] = 0;
    }
  }
}

// ---- gradient: g(site) += g5_a sum_c g5_c |x_{slot}(site, c)|^2 over the harvested
// slots of one lattice, in slot order (deterministic)
__global__ void k_w_grad(WArgs a, int lat, const int* __restrict__ slots, int nsl, double* __restrict__ grad, int V) {
  for (int site = blockIdx.x * blockDim.x + threadIdx.x; site < V; site += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < nsl; ++i) {
      const int slot = slots[i];
      const SlotState* S = a.st + slot;
      if (S->lat != lat) continue;
      const double sa = S->a < 6 ? 1.0 : -1.0;
      const double2* x = a.x + (size_t)slot * 12 * a.Vmax + site;
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        double2 v = x[(size_t)k * a.Vmax];
        t += (k < 6 ? 1.0 : -1.0) * (v.x * v.x + v.y * v.y);
      }
      acc += sa * t;
    }
    grad[site] += acc;
  }
}

// ================================================================ the engine
template <int SPR>
struct WilsonEngine {
  static constexpr int EPR = SPR == PR64 ? PR64 : PR32;
  static constexpr int NT = 128;
  static constexpr int KERNELS_PER_ITERATION = 7;
  hp_ctx* ctx;
  WArgs a;
  int nslots, gy;
  dim3 grid() const { return dim3(nslots, gy); }

  hp_status setup(int ns, int Vmax, const LatGeom* lats_dev, SlotState* st, const hp_solver_opts& o, double tol,
                  double delta) {
    nslots = ns;
    memset(&a, 0, sizeof(a));
    a.lats = lats_dev;
    a.st = st;
    a.Vmax = Vmax;
    gy = dslash_gridy(ctx, Vmax, NT, ns);
    a.gy = gy;
    void* p = nullptr;
    HP_TRY(hp_ws(ctx, "solve.part", sizeof(double) * 4 * (size_t)ns * gy, &p));
    a.part = (double*)p;
    HP_TRY(hp_ws(ctx, "solve.cnt", sizeof(unsigned int) * ns, &p));
    a.cnt = (unsigned int*)p;
    HP_CUDA(cudaMemsetAsync(a.cnt, 0, sizeof(unsigned int) * ns, ctx->stream));
    HP_TRY(alloc_field(ctx, "solve.r", SPR, ns, Vmax, &a.r));
    HP_TRY(alloc_field(ctx, "solve.rh", SPR, ns, Vmax, &a.rh));
    HP_TRY(alloc_field(ctx, "solve.p", SPR, ns, Vmax, &a.p));
    HP_TRY(alloc_field(ctx, "solve.v", SPR, ns, Vmax, &a.v));
    HP_TRY(alloc_field(ctx, "solve.s", SPR, ns, Vmax, &a.s));
    HP_TRY(alloc_field(ctx, "solve.t", SPR, ns, Vmax, &a.t));
    HP_TRY(alloc_field(ctx, "solve.e", EPR, ns, Vmax, &a.e));
    HP_TRY(hp_ws(ctx, "solve.x", sizeof(double2) * 12 * (size_t)ns * Vmax, &p));
    a.x = (double2*)p;
    a.tol2 = tol * tol;
    a.delta2 = delta * delta;
    a.maxiter = o.maxiter > 0 ? o.maxiter : 10000;
    return HP_OK;
  }
  hp_status init() {
    {
      ProfScope ps(ctx, "k_bicg_init");
      k_bicg_init<SPR, EPR, NT><<<grid(), NT, 0, ctx->stream>>>(a);
    }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  hp_status iteration() {
    const char* nv = SPR == PR64 ? "k_bicg_v<fp64>" : SPR == PR32 ? "k_bicg_v<fp32>" : SPR == PR16 ? "k_bicg_v<fp16>" : "k_bicg_v<bf16>";
    const char* nt = SPR == PR64 ? "k_bicg_t<fp64>" : SPR == PR32 ? "k_bicg_t<fp32>" : SPR == PR16 ? "k_bicg_t<fp16>" : "k_bicg_t<bf16>";
    { ProfScope ps(ctx, nv); k_bicg_v<SPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    { ProfScope ps(ctx, "k_bicg_s"); k_bicg_s<SPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    { ProfScope ps(ctx, nt); k_bicg_t<SPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    { ProfScope ps(ctx, "k_bicg_xr"); k_bicg_xr<SPR, EPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    { ProfScope ps(ctx, "k_ru_accum"); k_ru_accum<EPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    { ProfScope ps(ctx, "k_ru_residual<fp64>"); k_ru_residual<SPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    { ProfScope ps(ctx, "k_bicg_p"); k_bicg_p<SPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  hp_status harvest(const std::vector<int>& done_slots, const SolveProblem& pb, int* dev_slots) {
    {
      ProfScope ps(ctx, "k_quad");
      k_quad<NT><<<grid(), NT, 0, ctx->stream>>>(a);
    }
    HP_LAUNCH_CHECK();
    if (pb.want_grad && !done_slots.empty()) {
      HP_CUDA(cudaMemcpyAsync(dev_slots, done_slots.data(), sizeof(int) * done_slots.size(), cudaMemcpyHostToDevice,
                              ctx->stream));
      for (size_t L = 0; L < pb.lats.size(); ++L) {
        ProfScope ps(ctx, "k_w_grad");
        k_w_grad<<<blocks_for(ctx, pb.lats[L].V, 256), 256, 0, ctx->stream>>>(a, (int)L, dev_slots,
                                                                               (int)done_slots.size(), pb.grad_dev[L],
                                                                               pb.lats[L].V);
      }
      HP_LAUNCH_CHECK();
    }
    return HP_OK;
  }
};

// generic slot scheduler shared by both operator families
#include "hp_schedule.cuh"

hp_status hp_solve_wilson(hp_ctx* ctx, SolveProblem& pb, SolveResult& res) {
  const int prec = pb.opts.precision;
  double delta = pb.opts.delta;
  switch (prec) {
    case HP_PREC_FP64: {
      WilsonEngine<PR64> e{ctx};
      return run_schedule(ctx, e, pb, res, 12, delta > 0 ? delta : 0.0);
    }
    case HP_PREC_MIXED_FP32: {
      WilsonEngine<PR32> e{ctx};
      return run_schedule(ctx, e, pb, res, 12, delta > 0 ? delta : 1e-3);
    }
    case HP_PREC_MIXED_FP16: {
      WilsonEngine<PR16> e{ctx};
      return run_schedule(ctx, e, pb, res, 12, delta > 0 ? delta : 0.1);
    }
    case HP_PREC_MIXED_BF16: {
      WilsonEngine<PRB16> e{ctx};
      return run_schedule(ctx, e, pb, res, 12, delta > 0 ? delta : 0.1);
    }
  }
  hp_set_error("unknown precision %d", prec);
  return HP_EINVAL;
}
